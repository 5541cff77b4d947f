// Once-per-load-step mesh build: octree adaptivity and 2:1 balance (Sec. 5),
// nodes, hanging classification and constraints (Sec. 3.1), GIMP refinement
// (Sec. 5), the discrete GIMP basis (Sec. 3.2, Eq. GIMP numerical), ghost
// faces and the ghost matrix (Sec. 4), the 3x3 block pattern, the gravity
// force and the contact candidates.  Compiled with --fmad=false so that the
// box and grid arithmetic that decides discrete events rounds like the plain
// IEEE expressions of the method.
#include <algorithm>
#include <vector>

#include "mpm_internal.cuh"

namespace mpm {
namespace {

// ------------------------------------------------------------------ octree

__global__ void k_tree_uniform(int n, int shift, int lev, uint64_t* key, int* levs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = (uint64_t)i << shift;
  levs[i] = lev;
}

// Sec. 5, Steps 1-2: mark leaves meeting the body or with a corner within dx_region
__global__ void k_mark_refine(int n, const uint64_t* __restrict__ key, const int* __restrict__ lev,
                              Geo g, Body b, double dxr, int dmax, int* flag, int* any) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  if (lev[i] < dmax) {
    int a[3];
    demorton(key[i], a);
    int s = 1 << (g.D - lev[i]);
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = (double)a[d] * g.unit;
      hi[d] = (double)(a[d] + s) * g.unit;
    }
    if (body_meets_box(b, lo, hi)) {
      f = 1;
    } else {
      for (int c = 0; c < 8 && !f; ++c) {
        double xc[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]};
        if (body_distance(b, xc, dxr) <= dxr) f = 1;
      }
    }
  }
  flag[i] = f;
  if (f) *any = 1;
}

__global__ void k_child_count(int n, const int* flag, int* cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = flag[i] ? 8 : 1;
}

// children of a leaf are contiguous in Morton order: the sorted order survives
__global__ void k_refine_write(int n, const uint64_t* __restrict__ key, const int* __restrict__ lev,
                               const int* __restrict__ flag, const int* __restrict__ pos, int D,
                               uint64_t* okey, int* olev) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = pos[i];
  if (flag[i]) {
    int sh = 3 * (D - lev[i] - 1);
    for (int c = 0; c < 8; ++c) {
      okey[p + c] = key[i] + ((uint64_t)c << sh);
      olev[p + c] = lev[i] + 1;
    }
  } else {
    okey[p] = key[i];
    olev[p] = lev[i];
  }
}

// 2:1 balance across faces and edges (Sec. 5: one hanging node per edge/face)
__global__ void k_balance_mark(int n, const uint64_t* __restrict__ key, const int* __restrict__ lev,
                               Geo g, int* flag, int* any) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a[3];
  demorton(key[i], a);
  int s = 1 << (g.D - lev[i]);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz == 0 || nz == 3) continue;
        int dd[3] = {dx, dy, dz}, q[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          q[d] = dd[d] == 1 ? a[d] + s : (dd[d] == -1 ? a[d] - 1 : a[d]);
          ok = ok && q[d] >= 0 && q[d] < g.N;
        }
        if (!ok) continue;
        int nb = locate(key, n, q[0], q[1], q[2]);
        if (lev[nb] < lev[i] - 1) {
          flag[nb] = 1;
          *any = 1;
        }
      }
}

// ------------------------------------------------------------------ nodes

__global__ void k_corner_keys(int n, const uint64_t* __restrict__ key, const int* __restrict__ lev,
                              int D, uint64_t* ck) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a[3];
  demorton(key[i], a);
  int s = 1 << (D - lev[i]);
  for (int c = 0; c < 8; ++c)
    ck[8 * (size_t)i + c] = morton(a[0] + (c & 1) * s, a[1] + ((c >> 1) & 1) * s, a[2] + ((c >> 2) & 1) * s);
}

__device__ inline int find_exact(const uint64_t* __restrict__ key, int n, uint64_t k) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    uint64_t v = key[mid];
    if (v == k) return mid;
    if (v < k)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

__global__ void k_corner_ids(int n, const uint64_t* __restrict__ key, const int* __restrict__ lev,
                             int D, const uint64_t* __restrict__ nkey, int nn, int* corner) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a[3];
  demorton(key[i], a);
  int s = 1 << (D - lev[i]);
  for (int c = 0; c < 8; ++c)
    corner[8 * (size_t)i + c] = find_exact(
        nkey, nn, morton(a[0] + (c & 1) * s, a[1] + ((c >> 1) & 1) * s, a[2] + ((c >> 2) & 1) * s));
}

// Sec. 3.1: n hangs when it lies on the boundary of a leaf without being one of
// its vertices; K_n is the largest such leaf (ties: lowest Morton key)
__global__ void k_hang(int nn, const uint64_t* __restrict__ nkey, const uint64_t* __restrict__ lkey,
                       const int* __restrict__ llev, int nl, Geo g, int* hang, int* owner) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  int X[3];
  demorton(nkey[n], X);
  int best = -1;
  for (int sc = 0; sc < 8; ++sc) {
    int q[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
      q[d] = X[d] - 1 + ((sc >> d) & 1);
      ok = ok && q[d] >= 0 && q[d] < g.N;
    }
    if (!ok) continue;
    int K = locate(lkey, nl, q[0], q[1], q[2]);
    int s = 1 << (g.D - llev[K]);
    int a[3];
    demorton(lkey[K], a);
    bool corner = true;
    for (int d = 0; d < 3; ++d) {
      int r = X[d] - a[d];
      corner = corner && (r == 0 || r == s);
    }
    if (corner) continue;
    if (best < 0 || llev[K] < llev[best] || (llev[K] == llev[best] && lkey[K] < lkey[best])) best = K;
  }
  hang[n] = best >= 0 ? 1 : 0;
  owner[n] = best;
}

struct NodeView {
  const uint64_t* nkey;
  const uint64_t* lkey;
  const int* llev;
  const int* corner;
  const int* hang;
  const int* owner;
  int D;
};

// Eq. (constraint equation reduced): weights phi_{i,K_n}(x_n) of the owner's corners
__device__ int direct_constraint(const NodeView& v, int h, int* ids, double* ws) {
  int K = v.owner[h];
  int s = 1 << (v.D - v.llev[K]);
  int a[3], X[3];
  demorton(v.lkey[K], a);
  demorton(v.nkey[h], X);
  double xi[3];
  for (int d = 0; d < 3; ++d) {
    int t = 2 * (X[d] - a[d]);
    if (t != 0 && t != s && t != 2 * s) return -1;
    xi[d] = (double)t / (2.0 * s);
  }
  int cnt = 0;
  for (int c = 0; c < 8; ++c) {
    double w = 1.0;
    for (int d = 0; d < 3; ++d) w *= ((c >> d) & 1) ? xi[d] : 1.0 - xi[d];
    if (w != 0.0) {
      ids[cnt] = v.corner[8 * (size_t)K + c];
      ws[cnt] = w;
      ++cnt;
    }
  }
  return cnt;
}

// transitive substitution of hanging supports; returns the count or -1
__device__ int resolve_node(const NodeView& v, int n, int* ids, double* ws) {
  int cnt = 1;
  ids[0] = n;
  ws[0] = 1.0;
  for (int round = 0; round < 128; ++round) {
    int i = -1;
    for (int k = 0; k < cnt; ++k)
      if (v.hang[ids[k]]) {
        i = k;
        break;
      }
    if (i < 0) {
      for (int a = 1; a < cnt; ++a)
        for (int b = a; b > 0 && ids[b - 1] > ids[b]; --b) {
          int t = ids[b]; ids[b] = ids[b - 1]; ids[b - 1] = t;
          double tw = ws[b]; ws[b] = ws[b - 1]; ws[b - 1] = tw;
        }
      return cnt;
    }
    int h = ids[i];
    double wh = ws[i];
    ids[i] = ids[cnt - 1];
    ws[i] = ws[cnt - 1];
    --cnt;
    int dids[8];
    double dws[8];
    int nd = direct_constraint(v, h, dids, dws);
    if (nd < 0) return -2;
    for (int k = 0; k < nd; ++k) {
      int slot = -1;
      for (int q = 0; q < cnt; ++q)
        if (ids[q] == dids[k]) slot = q;
      if (slot >= 0) {
        ws[slot] += wh * dws[k];
      } else {
        if (cnt >= MAXC) return -1;
        ids[cnt] = dids[k];
        ws[cnt] = wh * dws[k];
        ++cnt;
      }
    }
  }
  return -2;
}

__global__ void k_con_count(int nn, NodeView v, int* cnt, int* err) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  int ids[MAXC];
  double ws[MAXC];
  int c = resolve_node(v, n, ids, ws);
  if (c < 0) {
    atomicOr(err, c == -1 ? EB_SUPPORT : EB_BALANCE);
    c = 0;
  }
  cnt[n] = c;
}

__global__ void k_con_fill(int nn, NodeView v, const int* __restrict__ cptr, int* cidx, double* cw) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  int ids[MAXC];
  double ws[MAXC];
  int c = resolve_node(v, n, ids, ws);
  int b = cptr[n], e = cptr[n + 1];
  for (int k = 0; k < c && b + k < e; ++k) {
    cidx[b + k] = ids[k];
    cw[b + k] = ws[k];
  }
}

// ------------------------------------------------------------------ GIMP domains and split

// GIMP domain in finest-grid units: bounds snapped, clipped; returns V_p (unclipped)
__device__ inline double domain_box(const double* x, const double* l, const Geo& g, double* Lo,
                                    double* Hi) {
  double V = 1.0, N = (double)g.N;
  for (int d = 0; d < 3; ++d) {
    double lo = snap_grid((x[d] - l[d]) * g.scale);
    double hi = snap_grid((x[d] + l[d]) * g.scale);
    V *= hi - lo;
    Lo[d] = lo < 0.0 ? 0.0 : lo;
    Hi[d] = hi > N ? N : hi;
  }
  return V;
}

// Sec. 5: split if some overlapped leaf has l_K < beta l_p (l_p: largest reference
// half-length); the leaf-by-leaf cutting stops at the first such leaf, and a
// work list overflow counts as a split
__global__ void k_split_flag(int P, const double* __restrict__ x, const double* __restrict__ lp,
                             const double* __restrict__ l0, const uint64_t* __restrict__ lkey,
                             const int* __restrict__ llev, int nl, Geo g, double beta, int* flag,
                             int* err) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double Lo[3], Hi[3];
  domain_box(x + 3 * (size_t)p, lp + 3 * (size_t)p, g, Lo, Hi);
  if (!(Hi[0] > Lo[0]) || !(Hi[1] > Lo[1]) || !(Hi[2] > Lo[2])) {
    atomicOr(err, EB_DOMAIN);
    flag[p] = 0;
    return;
  }
  double lm = l0[3 * (size_t)p];
  if (l0[3 * (size_t)p + 1] > lm) lm = l0[3 * (size_t)p + 1];
  if (l0[3 * (size_t)p + 2] > lm) lm = l0[3 * (size_t)p + 2];
  double lim = beta * lm * g.scale;
  double st[SPLIT_STACK][6];
  int ns = 1;
  for (int d = 0; d < 3; ++d) {
    st[0][d] = Lo[d];
    st[0][3 + d] = Hi[d];
  }
  int f = 0;
  while (ns > 0) {
    --ns;
    double a[3], b[3], kh[3], e[3];
    int q[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = st[ns][d];
      b[d] = st[ns][3 + d];
      q[d] = (int)floor(a[d]);
      q[d] = q[d] > g.N - 1 ? g.N - 1 : (q[d] < 0 ? 0 : q[d]);
    }
    int K = locate(lkey, nl, q[0], q[1], q[2]);
    int s = 1 << (g.D - llev[K]);
    if (0.5 * (double)s < lim) {
      f = 1;
      break;
    }
    int ka[3];
    demorton(lkey[K], ka);
    for (int d = 0; d < 3; ++d) {
      kh[d] = (double)(ka[d] + s);
      e[d] = b[d] < kh[d] ? b[d] : kh[d];
    }
    if (ns + 3 > SPLIT_STACK) {
      f = 1;
      break;
    }
    if (b[0] > kh[0]) {
      double* r = st[ns++];
      r[0] = kh[0]; r[1] = a[1]; r[2] = a[2]; r[3] = b[0]; r[4] = b[1]; r[5] = b[2];
    }
    if (b[1] > kh[1]) {
      double* r = st[ns++];
      r[0] = a[0]; r[1] = kh[1]; r[2] = a[2]; r[3] = e[0]; r[4] = b[1]; r[5] = b[2];
    }
    if (b[2] > kh[2]) {
      double* r = st[ns++];
      r[0] = a[0]; r[1] = a[1]; r[2] = kh[2]; r[3] = e[0]; r[4] = e[1]; r[5] = b[2];
    }
  }
  flag[p] = f;
}

// children: child 0 keeps the parent slot, children 1..7 go to P + 7 rank + c - 1
__global__ void k_split_write(int P, const int* __restrict__ flag, const int* __restrict__ rank,
                              mpm_points pts) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P || !flag[p]) return;
  double xc[3], lc[3], l0c[3];
  for (int d = 0; d < 3; ++d) {
    xc[d] = pts.x[3 * (size_t)p + d];
    lc[d] = pts.lp[3 * (size_t)p + d];
    l0c[d] = pts.l0[3 * (size_t)p + d];
  }
  for (int c = 0; c < 8; ++c) {
    size_t q = c == 0 ? (size_t)p : (size_t)P + 7 * (size_t)rank[p] + (c - 1);
    for (int d = 0; d < 3; ++d) {
      double sg = ((c >> d) & 1) ? 0.5 : -0.5;
      pts.x[3 * q + d] = xc[d] + sg * lc[d];
      pts.lp[3 * q + d] = 0.5 * lc[d];
      pts.l0[3 * q + d] = 0.5 * l0c[d];
    }
    if (c) {
      for (int i = 0; i < 9; ++i) pts.F[9 * q + i] = pts.F[9 * (size_t)p + i];
      for (int i = 0; i < 6; ++i) pts.be[6 * q + i] = pts.be[6 * (size_t)p + i];
      pts.V0[q] = pts.V0[p] / 8.0;
      pts.mass[q] = pts.mass[p] / 8.0;
      pts.E[q] = pts.E[p];
      pts.ys[q] = pts.ys[p];
      if (pts.v)
        for (int d = 0; d < 3; ++d) pts.v[3 * q + d] = pts.v[3 * (size_t)p + d];
    }
  }
  pts.V0[p] /= 8.0;
  pts.mass[p] /= 8.0;
}

// ------------------------------------------------------------------ cell sort

__global__ void k_point_cell(int P, const double* __restrict__ x, Geo g,
                             const uint64_t* __restrict__ lkey, int nl, int* cell, int* idx) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int q[3];
  for (int d = 0; d < 3; ++d) {
    double v = floor(x[3 * (size_t)p + d] * g.scale);
    q[d] = v < 0 ? 0 : (v > g.N - 1 ? g.N - 1 : (int)v);
  }
  cell[p] = locate(lkey, nl, q[0], q[1], q[2]);
  idx[p] = p;
}

__global__ void k_gather_points(int P, const int* __restrict__ perm, mpm_points pts, double* x,
                                double* lp, double* l0, double* F, double* be, double* V0,
                                double* mass, double* E, double* ys, double* v) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  size_t p = perm[w];
  for (int d = 0; d < 3; ++d) {
    x[3 * (size_t)w + d] = pts.x[3 * p + d];
    lp[3 * (size_t)w + d] = pts.lp[3 * p + d];
    l0[3 * (size_t)w + d] = pts.l0[3 * p + d];
    if (v) v[3 * (size_t)w + d] = pts.v[3 * p + d];
  }
  for (int i = 0; i < 9; ++i) F[9 * (size_t)w + i] = pts.F[9 * p + i];
  for (int i = 0; i < 6; ++i) be[6 * (size_t)w + i] = pts.be[6 * p + i];
  V0[w] = pts.V0[p];
  mass[w] = pts.mass[p];
  E[w] = pts.E[p];
  ys[w] = pts.ys[p];
}

// ------------------------------------------------------------------ discrete GIMP basis

struct SubBox {
  double xi[3];  // centroid in the leaf's local coordinates
  double w;      // V_Kp / V_p
  double is;     // 1 / leaf size (a power of two, exact)
  int K, s;
};

__device__ inline int warp_excl_scan(int v, int lane) {
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

constexpr int BW = 4;  // warps per block of the basis kernel

constexpr int BH = 512;  // per-warp hash set of the basis kernel's node ids (at most MAXS distinct)

__device__ inline unsigned basis_hash(int j) { return ((unsigned)j * 2654435761u) >> 23; }

// Eq. (GIMP numerical), one warp per point (cell-sorted order):
//  1. lane 0 cuts the domain into its leaf intersections (centre, volume);
//  2. the (leaf corner, constraint entry) pairs are listed in a fixed order;
//  3. the distinct independent nodes are found by a shared-memory hash set and
//     ranked by id (support sorted by node id); the entries are grouped by
//     node, each group keeping list order;
//  4. lane k sums the contributions of support node k in list order, so the
//     result does not depend on scheduling.
__global__ void __launch_bounds__(32 * BW)
    k_basis(int P, Geo g, const double* __restrict__ px, const double* __restrict__ plp,
            const double* __restrict__ pE, const uint64_t* __restrict__ lkey,
            const int* __restrict__ llev, int nl, const int* __restrict__ corner,
            const int* __restrict__ cptr, const int* __restrict__ cidx,
            const double* __restrict__ cw, int* nsup, int* sidx, double* S, double* dS,
            int* populated, unsigned long long* betaK, int* err) {
  __shared__ SubBox sb[BW][MAXK];
  __shared__ int e_node[BW][MAXE];
  __shared__ short e_q[BW][MAXE];
  __shared__ short e_ord[BW][MAXE];
  __shared__ float e_w[BW][MAXE];  // constraint weights are products of 1/2 and 1/4: exact
  __shared__ unsigned char e_rk[BW][MAXE];
  __shared__ int sup[BW][MAXS];
  __shared__ int hkey[BW][BH];
  __shared__ unsigned char hslot[BW][BH];
  __shared__ int uid[BW][MAXS];
  __shared__ unsigned char urank[BW][MAXS];
  __shared__ int ucnt[BW][MAXS], ubase[BW][MAXS], ustart[BW][MAXS];
  __shared__ int nsub_s[BW], nu_s[BW];
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int w = blockIdx.x * BW + wi;
  if (w >= P) return;
  // 1. the domain cut into its leaf intersections.  Every cut face is a leaf
  // face, an integer in grid units, so lane 0 walks the leaves in integer
  // arithmetic: a bound is either the domain's own (code -1) or a face.
  // The walk's FP64 work (volumes, centroids) then runs one sub-box per
  // lane: a warp's FP64 instruction costs the same pipe time whatever the
  // number of active lanes.
  double Lo[3], Hi[3];
  double Vp = domain_box(px + 3 * (size_t)w, plp + 3 * (size_t)w, g, Lo, Hi);
  if (lane == 0) {
    int n = 0;
    if (!(Hi[0] > Lo[0]) || !(Hi[1] > Lo[1]) || !(Hi[2] > Lo[2])) {
      atomicOr(err, EB_DOMAIN);
      n = -1;
    } else {
      int fLo[3], fHi[3];
      bool iHi[3];
      for (int d = 0; d < 3; ++d) {
        fLo[d] = (int)floor(Lo[d]);
        fHi[d] = (int)floor(Hi[d]);
        iHi[d] = Hi[d] == (double)fHi[d];
      }
      int st[3 * MAXK + 8][6];
      int ns = 1;
      for (int d = 0; d < 6; ++d) st[0][d] = -1;
      while (ns > 0) {
        --ns;
        int a[3], b[3], kh[3], e[3], q[3];
        for (int d = 0; d < 3; ++d) {
          a[d] = st[ns][d];
          b[d] = st[ns][3 + d];
          q[d] = a[d] < 0 ? fLo[d] : a[d];
          q[d] = q[d] > g.N - 1 ? g.N - 1 : (q[d] < 0 ? 0 : q[d]);
        }
        int K = locate(lkey, nl, q[0], q[1], q[2]);
        int s = 1 << (g.D - llev[K]);
        int ka[3];
        demorton(lkey[K], ka);
        bool gt[3];
        for (int d = 0; d < 3; ++d) {
          kh[d] = ka[d] + s;
          if (b[d] < 0) {
            // the domain's upper bound against the face kh: Hi < kh iff
            // floor(Hi) < kh; Hi > kh iff floor(Hi) > kh, or equal and Hi
            // is not an integer
            e[d] = fHi[d] < kh[d] ? -1 : kh[d];
            gt[d] = fHi[d] > kh[d] || (!iHi[d] && fHi[d] == kh[d]);
          } else {
            e[d] = b[d] < kh[d] ? b[d] : kh[d];
            gt[d] = b[d] > kh[d];
          }
        }
        if (n >= MAXK || ns + 3 > 3 * MAXK + 8) {
          atomicOr(err, EB_SUPPORT);
          n = -1;
          break;
        }
        SubBox& o = sb[wi][n++];
        int* cd = reinterpret_cast<int*>(o.xi);  // bound codes until step 1b
        for (int d = 0; d < 3; ++d) {
          cd[d] = a[d];
          cd[3 + d] = e[d];
        }
        o.K = K;
        o.s = s;
        if (gt[0]) {
          int* r = st[ns++];
          r[0] = kh[0]; r[1] = a[1]; r[2] = a[2]; r[3] = b[0]; r[4] = b[1]; r[5] = b[2];
        }
        if (gt[1]) {
          int* r = st[ns++];
          r[0] = a[0]; r[1] = kh[1]; r[2] = a[2]; r[3] = e[0]; r[4] = b[1]; r[5] = b[2];
        }
        if (gt[2]) {
          int* r = st[ns++];
          r[0] = a[0]; r[1] = a[1]; r[2] = kh[2]; r[3] = e[0]; r[4] = e[1]; r[5] = b[2];
        }
      }
    }
    nsub_s[wi] = n;
  }
  __syncwarp();
  // 1b. one lane per sub-box: volume fraction, centroid in leaf coordinates
  if (lane < nsub_s[wi]) {
    SubBox& o = sb[wi][lane];
    const int* cd = reinterpret_cast<const int*>(o.xi);
    int ca[3], ce[3];
    for (int d = 0; d < 3; ++d) {
      ca[d] = cd[d];
      ce[d] = cd[3 + d];
    }
    int ka[3];
    demorton(lkey[o.K], ka);
    double vol = 1.0, xi[3];
    // the leaf size is a power of two: multiplying by its exact reciprocal
    // equals the division and keeps the FP64 pipe (slow on this part) free
    double is = ldexp(1.0, llev[o.K] - g.D);
    for (int d = 0; d < 3; ++d) {
      double a = ca[d] < 0 ? Lo[d] : (double)ca[d];
      double e = ce[d] < 0 ? Hi[d] : (double)ce[d];
      vol *= e - a;
      xi[d] = (0.5 * (a + e) - (double)ka[d]) * is;
    }
    for (int d = 0; d < 3; ++d) o.xi[d] = xi[d];
    o.is = is;
    o.w = vol / Vp;
  }
  __syncwarp();
  int nsub = nsub_s[wi];
  if (nsub < 0) {
    if (lane == 0) nsup[w] = 0;
    return;
  }
  if (lane < nsub) {
    int K = sb[wi][lane].K;
    populated[K] = 1;
    atomicMax(betaK + K, (unsigned long long)__double_as_longlong(pE[w]));
  }
  // 2. list the (corner, constraint) entries in pair order
  int npair = 8 * nsub;
  int per = (npair + 31) / 32;
  int q0 = lane * per, q1 = min(q0 + per, npair);
  int len = 0;
  for (int q = q0; q < q1; ++q) {
    int node = corner[8 * (size_t)sb[wi][q >> 3].K + (q & 7)];
    len += cptr[node + 1] - cptr[node];
  }
  int off = warp_excl_scan(len, lane);
  int total = __shfl_sync(0xffffffffu, off + len, 31);
  if (total > MAXE) {
    if (lane == 0) {
      atomicOr(err, EB_SUPPORT);
      nsup[w] = 0;
    }
    return;
  }
  int pos = off;
  for (int q = q0; q < q1; ++q) {
    int node = corner[8 * (size_t)sb[wi][q >> 3].K + (q & 7)];
    for (int t = cptr[node]; t < cptr[node + 1]; ++t) {
      e_node[wi][pos] = cidx[t];
      e_q[wi][pos] = (short)q;
      e_w[wi][pos] = (float)cw[t];
      ++pos;
    }
  }
  __syncwarp();
  // 3. distinct nodes (hash set), ranked by id, entries grouped by node
  for (int i = lane; i < BH; i += 32) hkey[wi][i] = -1;
  if (lane == 0) nu_s[wi] = 0;
  __syncwarp();
  for (int e = lane; e < total; e += 32) {
    int j = e_node[wi][e];
    unsigned h = basis_hash(j);
    for (int probe = 0; probe < BH; ++probe) {
      int prev = atomicCAS(&hkey[wi][h], -1, j);
      if (prev == -1) {
        int slot = atomicAdd(&nu_s[wi], 1);
        if (slot < MAXS) uid[wi][slot] = j;
        hslot[wi][h] = (unsigned char)min(slot, 255);
        break;
      }
      if (prev == j) break;
      h = (h + 1) & (BH - 1);
    }
  }
  __syncwarp();
  int ns = nu_s[wi];
  if (ns > MAXS) {
    if (lane == 0) {
      atomicOr(err, EB_SUPPORT);
      nsup[w] = 0;
    }
    return;
  }
  for (int u = lane; u < ns; u += 32) {
    int j = uid[wi][u], r = 0;
    for (int u2 = 0; u2 < ns; ++u2) r += uid[wi][u2] < j ? 1 : 0;
    urank[wi][u] = (unsigned char)r;
    sup[wi][r] = j;
  }
  for (int u = lane; u < MAXS; u += 32) ucnt[wi][u] = 0;
  __syncwarp();
  // rank of every entry (hash lookup) and the count per rank
  for (int e = lane; e < total; e += 32) {
    int j = e_node[wi][e];
    unsigned h = basis_hash(j);
    while (hkey[wi][h] != j) h = (h + 1) & (BH - 1);
    int r = urank[wi][hslot[wi][h]];
    e_rk[wi][e] = (unsigned char)r;
    atomicAdd(&ucnt[wi][r], 1);
  }
  __syncwarp();
  {
    int c0 = lane < ns ? ucnt[wi][lane] : 0, c1 = lane + 32 < ns ? ucnt[wi][lane + 32] : 0;
    int x0 = warp_excl_scan(c0, lane), x1 = warp_excl_scan(c1, lane);
    int t0 = __shfl_sync(0xffffffffu, x0 + c0, 31);
    if (lane < ns) ubase[wi][lane] = ustart[wi][lane] = x0;
    if (lane + 32 < ns) ubase[wi][lane + 32] = ustart[wi][lane + 32] = t0 + x1;
  }
  __syncwarp();
  // stable grouping: chunks of 32 entries in list order, positions inside a
  // chunk by lane order among the lanes of the same rank
  for (int c0 = 0; c0 < total; c0 += 32) {
    int e = c0 + lane;
    bool valid = e < total;
    int r = valid ? (int)e_rk[wi][e] : -1 - lane;
    unsigned grp = __match_any_sync(0xffffffffu, r);
    int before = __popc(grp & ((1u << lane) - 1u));
    int pos = valid ? ubase[wi][r] + before : 0;
    __syncwarp();
    if (valid) {
      e_ord[wi][pos] = (short)e;
      if (before == 0) ubase[wi][r] += __popc(grp);
    }
    __syncwarp();
  }
  // 4. values and gradients of S_vp
  for (int k = lane; k < ns; k += 32) {
    int j = sup[wi][k];
    double s0 = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int t = ustart[wi][k]; t < ustart[wi][k] + ucnt[wi][k]; ++t) {
      int e = e_ord[wi][t];
      int q = e_q[wi][e];
      const SubBox& o = sb[wi][q >> 3];
      int c = q & 7;
      double f0 = (c & 1) ? o.xi[0] : 1.0 - o.xi[0];
      double f1 = (c & 2) ? o.xi[1] : 1.0 - o.xi[1];
      double f2 = (c & 4) ? o.xi[2] : 1.0 - o.xi[2];
      double inv = o.is;
      double d0 = (c & 1) ? inv : -inv, d1 = (c & 2) ? inv : -inv, d2 = (c & 4) ? inv : -inv;
      double ww = e_w[wi][e] * o.w;
      s0 += ww * (f0 * f1 * f2);
      g0 += ww * (d0 * f1 * f2);
      g1 += ww * (f0 * d1 * f2);
      g2 += ww * (f0 * f1 * d2);
    }
    size_t o = (size_t)w * MAXS + k;
    sidx[o] = j;
    S[o] = s0;
    dS[3 * o] = g0 * g.scale;
    dS[3 * o + 1] = g1 * g.scale;
    dS[3 * o + 2] = g2 * g.scale;
  }
  if (lane == 0) nsup[w] = ns;
}

__global__ void k_mark_active(int P, const int* __restrict__ nsup, const int* __restrict__ sidx,
                              int* active) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)P * MAXS) return;
  int w = (int)(i / MAXS), k = (int)(i % MAXS);
  if (k < nsup[w]) active[sidx[i]] = 1;
}

__global__ void k_number_dofs(int nn, const int* __restrict__ active, const int* __restrict__ pos,
                              int* node_dof, int* dof_node) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  if (active[n]) {
    node_dof[n] = pos[n];
    dof_node[pos[n]] = n;
  } else {
    node_dof[n] = -1;
  }
}

__global__ void k_sidx_to_dof(int P, const int* __restrict__ nsup, const int* __restrict__ node_dof,
                              int* sidx) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)P * MAXS) return;
  int w = (int)(i / MAXS), k = (int)(i % MAXS);
  if (k < nsup[w]) sidx[i] = node_dof[sidx[i]];
}

struct Planes {
  int n;
  int axis[8];
  int pos[8];
  int mask[8];
};

__global__ void k_dof_mask(int nd, const int* __restrict__ dof_node, const uint64_t* __restrict__ nkey,
                           Planes pl, int* mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  int X[3];
  demorton(nkey[dof_node[i]], X);
  int m = 0;
  for (int b = 0; b < pl.n; ++b)
    if (X[pl.axis[b]] == pl.pos[b]) m |= pl.mask[b];
  mask[i] = m;
}

// ------------------------------------------------------------------ ghost faces (Sec. 4)

__device__ inline int across(const uint64_t* lkey, const int* llev, int nl, const Geo& g, int K,
                             int axis, int sign, int o1, int o2) {
  int a[3];
  demorton(lkey[K], a);
  int s = 1 << (g.D - llev[K]);
  a[axis] = sign > 0 ? a[axis] + s : a[axis] - 1;
  if (a[axis] < 0 || a[axis] >= g.N) return -1;
  a[(axis + 1) % 3] += o1;
  a[(axis + 2) % 3] += o2;
  return locate(lkey, nl, a[0], a[1], a[2]);
}

// T^B: populated leaves sharing a face with an unpopulated leaf
__global__ void k_boundary_elements(int nl, const uint64_t* __restrict__ lkey,
                                    const int* __restrict__ llev, Geo g,
                                    const int* __restrict__ pop, int* isB) {
  int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nl) return;
  int b = 0;
  if (pop[K]) {
    int s = 1 << (g.D - llev[K]);
    for (int f = 0; f < 6 && !b; ++f) {
      int axis = f >> 1, sign = (f & 1) ? 1 : -1;
      int nb = across(lkey, llev, nl, g, K, axis, sign, 0, 0);
      if (nb < 0) continue;
      if (llev[nb] <= llev[K]) {
        if (!pop[nb]) b = 1;
      } else {
        for (int o = 0; o < 4; ++o) {
          int nb2 = across(lkey, llev, nl, g, K, axis, sign, (o & 1) * (s >> 1), ((o >> 1) & 1) * (s >> 1));
          if (!pop[nb2]) b = 1;
        }
      }
    }
  }
  isB[K] = b;
}

// F_B: both leaves populated and one of them in T^B; each face once, from its
// smaller leaf (equal leaves: from the lower one)
__global__ void k_ghost_face_flag(int nl, const uint64_t* __restrict__ lkey,
                                  const int* __restrict__ llev, Geo g, const int* __restrict__ pop,
                                  const int* __restrict__ isB, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * nl) return;
  int K = i / 6, f = i % 6;
  int axis = f >> 1, sign = (f & 1) ? 1 : -1;
  int ok = 0;
  if (pop[K]) {
    int nb = across(lkey, llev, nl, g, K, axis, sign, 0, 0);
    if (nb >= 0 && llev[nb] <= llev[K] && !(llev[nb] == llev[K] && sign < 0) && pop[nb] &&
        (isB[K] || isB[nb]))
      ok = 1;
  }
  flag[i] = ok;
}

__global__ void k_ghost_face_write(int nl, const uint64_t* __restrict__ lkey,
                                   const int* __restrict__ llev, Geo g, const int* __restrict__ flag,
                                   const int* __restrict__ pos, int* face) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * nl || !flag[i]) return;
  int K = i / 6, f = i % 6;
  int axis = f >> 1, sign = (f & 1) ? 1 : -1;
  int p = pos[i];
  face[4 * p] = K;
  face[4 * p + 1] = across(lkey, llev, nl, g, K, axis, sign, 0, 0);
  face[4 * p + 2] = axis;
  face[4 * p + 3] = sign;
}

// dofs of I(K+) u I(K-) of each ghost face
__global__ void k_ghost_face_dofs(int nf, const int* __restrict__ face, const int* __restrict__ corner,
                                  const int* __restrict__ cptr, const int* __restrict__ cidx,
                                  const int* __restrict__ node_dof, int* gdof, int* gn, int* err) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int n = 0;
  int* out = gdof + (size_t)f * MAXG;
  for (int side = 0; side < 2; ++side) {
    int K = face[4 * f + side];
    for (int c = 0; c < 8; ++c) {
      int node = corner[8 * (size_t)K + c];
      for (int t = cptr[node]; t < cptr[node + 1]; ++t) {
        int j = node_dof[cidx[t]];
        bool have = false;
        for (int q = 0; q < n; ++q) have = have || out[q] == j;
        if (have) continue;
        if (n >= MAXG || j < 0) {
          atomicOr(err, EB_SUPPORT);
          continue;
        }
        out[n++] = j;
      }
    }
  }
  gn[f] = n;
}

__device__ inline int find_slot(const int* __restrict__ row_ptr, const int* __restrict__ col, int r,
                                int c) {
  int lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = col[mid];
    if (v == c) return mid;
    if (v < c)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

// derivative along `axis` (grid units) of phi~_j in leaf K at xi
__device__ double leaf_dphi(int K, int s, const double* xi, int axis, int j,
                            const int* __restrict__ corner, const int* __restrict__ cptr,
                            const int* __restrict__ cidx, const double* __restrict__ cw,
                            const int* __restrict__ node_dof) {
  double r = 0.0;
  for (int c = 0; c < 8; ++c) {
    double f[3];
    for (int d = 0; d < 3; ++d) f[d] = ((c >> d) & 1) ? xi[d] : 1.0 - xi[d];
    f[axis] = (((c >> axis) & 1) ? 1.0 : -1.0) / (double)s;
    double dp = f[0] * f[1] * f[2];
    int node = corner[8 * (size_t)K + c];
    for (int t = cptr[node]; t < cptr[node + 1]; ++t)
      if (node_dof[cidx[t]] == j) r += cw[t] * dp;
  }
  return r;
}

// Eq. (ghost): 2x2 Gauss points on the smaller face, mapped into the larger
// leaf; k_G(i,j) = sum over faces and Gauss points of w (h_F beta_F / kappa)
// J_i J_j with J the normal-derivative jump.  One warp per face stores the
// face's coefficient w h_F beta_F / kappa and its jumps J (4 x MAXG); the
// rows are summed by k_ghost_rows.
__global__ void k_ghost_jumps(int nf, Geo g, double kappa, const int* __restrict__ face,
                              const uint64_t* __restrict__ lkey, const int* __restrict__ llev,
                              const double* __restrict__ betaK, const int* __restrict__ gdof,
                              const int* __restrict__ gn, const int* __restrict__ corner,
                              const int* __restrict__ cptr, const int* __restrict__ cidx,
                              const double* __restrict__ cw, const int* __restrict__ node_dof,
                              double* gJ, double* gcoef) {
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int f = blockIdx.x * 4 + wi;
  if (f >= nf) return;
  int K = face[4 * f], Nb = face[4 * f + 1], axis = face[4 * f + 2], sign = face[4 * f + 3];
  int sK = 1 << (g.D - llev[K]), sN = 1 << (g.D - llev[Nb]);
  int aK[3], aN[3];
  demorton(lkey[K], aK);
  demorton(lkey[Nb], aN);
  double hF = (double)(sK > sN ? sK : sN) * g.unit;
  double bF = betaK[K] > betaK[Nb] ? betaK[K] : betaK[Nb];
  double area = ((double)sK * g.unit) * ((double)sK * g.unit);
  if (lane == 0) gcoef[f] = hF * bF / kappa * area / 4.0;
  const double gq = 0.5 / sqrt(3.0);
  int t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
  int n = gn[f];
  const int* ids = gdof + (size_t)f * MAXG;
  for (int gp = 0; gp < 4; ++gp) {
    double X[3];
    X[axis] = (double)aK[axis] + (sign > 0 ? (double)sK : 0.0);
    X[t1] = (double)aK[t1] + (double)sK * ((gp & 1) ? 0.5 + gq : 0.5 - gq);
    X[t2] = (double)aK[t2] + (double)sK * ((gp & 2) ? 0.5 + gq : 0.5 - gq);
    double xiK[3], xiN[3];
    for (int d = 0; d < 3; ++d) {
      xiK[d] = (X[d] - (double)aK[d]) / (double)sK;
      xiN[d] = (X[d] - (double)aN[d]) / (double)sN;
    }
    for (int e = lane; e < n; e += 32) {
      int j = ids[e];
      double jk = leaf_dphi(K, sK, xiK, axis, j, corner, cptr, cidx, cw, node_dof);
      double jn = leaf_dphi(Nb, sN, xiN, axis, j, corner, cptr, cidx, cw, node_dof);
      gJ[((size_t)f * 4 + gp) * MAXG + e] = (double)sign * (jk - jn) * g.scale;
    }
  }
}

// k_G row r: one warp; the row's ghost-face sources (face f, local index a of
// r in the face's dofs) in key order, and for each the face's dofs b over the
// lanes: k_G(r, b) += coef_f sum over Gauss points of J_a J_b.  The lanes of
// one source write distinct columns and the sources follow one another, so
// every entry is summed in a fixed order (no atomics).
__global__ void k_ghost_rows(int nd, int P, const long long* __restrict__ sptr,
                             const uint64_t* __restrict__ skeys, const int* __restrict__ gdof,
                             const int* __restrict__ gn, const double* __restrict__ gJ,
                             const double* __restrict__ gcoef, const int* __restrict__ row_ptr,
                             const int* __restrict__ col, double* kg) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nd) return;
  for (long long q = sptr[r]; q < sptr[r + 1]; ++q) {
    uint32_t sid = (uint32_t)skeys[q];
    int f = (int)(sid >> 6) - P, a = (int)(sid & 63);
    if (f < 0) continue;  // a point source
    double cf = gcoef[f];
    const double* J = gJ + (size_t)f * 4 * MAXG;
    double ja[4] = {J[a], J[MAXG + a], J[2 * MAXG + a], J[3 * MAXG + a]};
    int n = gn[f];
    for (int b = lane; b < n; b += 32) {
      double v = cf * (ja[0] * J[b] + ja[1] * J[MAXG + b] + ja[2] * J[2 * MAXG + b] +
                       ja[3] * J[3 * MAXG + b]);
      if (v == 0.0) continue;
      int sl = find_slot(row_ptr, col, r, gdof[(size_t)f * MAXG + b]);
      if (sl >= 0) kg[sl] += v;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ block pattern

// sum over the points of (support size)^2: the (source, column) pairs of the
// tangent gather, for the benchmark's operation counts (integer, exact)
__global__ void k_support_pairs(int P, const int* __restrict__ nsup, unsigned long long* out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = w < P ? (unsigned long long)nsup[w] * (unsigned long long)nsup[w] : 0ULL;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// source keys: row dof << 32 | source << 6 | local index (points, then ghost faces)
__global__ void k_src_keys_points(int P, const int* __restrict__ nsup, const int* __restrict__ sidx,
                                  const int* __restrict__ off, uint64_t* keys) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)P * MAXS) return;
  int w = (int)(i / MAXS), k = (int)(i % MAXS);
  if (k >= nsup[w]) return;
  keys[off[w] + k] = ((uint64_t)(uint32_t)sidx[i] << 32) | ((uint64_t)(uint32_t)w << 6) | (uint32_t)k;
}

__global__ void k_src_keys_faces(int nf, int P, const int* __restrict__ gn, const int* __restrict__ gdof,
                                 long long base, uint64_t* keys) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nf * MAXG) return;
  int f = (int)(i / MAXG), k = (int)(i % MAXG);
  if (k >= gn[f]) return;
  keys[base + (long long)f * MAXG + k] =
      ((uint64_t)(uint32_t)gdof[i] << 32) | ((uint64_t)(uint32_t)(P + f) << 6) | (uint32_t)k;
}

__global__ void k_src_ptr(long long n, const uint64_t* __restrict__ keys, int ndof, long long* ptr) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t r = (uint32_t)(keys[i] >> 32);
  if (r >= (uint32_t)ndof) return;  // unused padding keys sort last
  if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != r) ptr[r] = i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != r) ptr[r + 1] = i + 1;
}

__device__ inline int hash_insert(int* h, int key) {
  unsigned s = ((unsigned)key * 2654435761u) & (HASH - 1);
  for (int probe = 0; probe < HASH; ++probe) {
    int prev = atomicCAS(h + s, -1, key);
    if (prev == -1) return 1;
    if (prev == key) return 0;
    s = (s + 1) & (HASH - 1);
  }
  return -1;
}

constexpr int PW = 2;  // warps per block of the pattern kernel

// one warp per row: the columns of row r are the union of the supports of
// every source (point or ghost face) touching r; count, then write sorted
__global__ void __launch_bounds__(32 * PW)
    k_pattern_rows(int ndof, int P, int mode, const long long* __restrict__ sptr,
                   const uint64_t* __restrict__ keys, const int* __restrict__ nsup,
                   const int* __restrict__ sidx, const int* __restrict__ gn,
                   const int* __restrict__ gdof, int* rowcnt, const int* __restrict__ row_ptr,
                   int* col, int* err) {
  __shared__ int h[PW][HASH];
  __shared__ int lst[PW][MAXROW];
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int r = blockIdx.x * PW + wi;
  if (r >= ndof) return;
  for (int i = lane; i < HASH; i += 32) h[wi][i] = -1;
  __syncwarp();
  int cnt = 0, bad = 0;
  for (long long i = sptr[r]; i < sptr[r + 1]; ++i) {
    uint32_t sid = (uint32_t)keys[i] >> 6;
    int n;
    const int* base;
    if ((int)sid < P) {
      n = nsup[sid];
      base = sidx + (size_t)sid * MAXS;
    } else {
      n = gn[sid - P];
      base = gdof + (size_t)(sid - P) * MAXG;
    }
    for (int l = lane; l < n; l += 32) {
      int rv = hash_insert(h[wi], base[l]);
      if (rv > 0) ++cnt;
      if (rv < 0) bad = 1;
    }
  }
  cnt = warp_sum_int(cnt);
  bad = __any_sync(0xffffffffu, bad);
  if (cnt > MAXROW || bad) {
    if (lane == 0) atomicOr(err, EB_ROW);
    if (mode == 0 && lane == 0) rowcnt[r] = 0;
    return;
  }
  if (mode == 0) {
    if (lane == 0) rowcnt[r] = cnt;
    return;
  }
  __syncwarp();
  // compact the occupied slots, then rank
  int mine = 0;
  for (int i = lane * (HASH / 32); i < (lane + 1) * (HASH / 32); ++i) mine += h[wi][i] >= 0;
  int off = warp_excl_scan(mine, lane);
  for (int i = lane * (HASH / 32); i < (lane + 1) * (HASH / 32); ++i)
    if (h[wi][i] >= 0) lst[wi][off++] = h[wi][i];
  __syncwarp();
  int b = row_ptr[r];
  for (int e = lane; e < cnt; e += 32) {
    int v = lst[wi][e], rk = 0;
    for (int e2 = 0; e2 < cnt; ++e2) rk += lst[wi][e2] < v;
    col[b + rk] = v;
  }
}

// ------------------------------------------------------------------ gravity, contact candidates

// f_ext,r = sum over the point sources (p, k) of row r of S_pk m_p g: one warp
// per row, lanes strided over the sources in key order, then the fixed
// shuffle tree (the same sums on every run)
__global__ void k_fext_rows(int nd, int P, const long long* __restrict__ sptr,
                            const uint64_t* __restrict__ skeys, const double* __restrict__ S,
                            const double* __restrict__ mass, double g0, double g1, double g2,
                            double* fext) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nd) return;
  double a = 0.0;
  for (long long q = sptr[r] + lane; q < sptr[r + 1]; q += 32) {
    uint32_t sid = (uint32_t)skeys[q];
    int w = (int)(sid >> 6), k = (int)(sid & 63);
    if (w >= P) continue;
    a += S[(size_t)w * MAXS + k] * mass[w];
  }
  a = warp_sum(a);
  if (lane < 3) fext[3 * (size_t)r + lane] = a * (lane == 0 ? g0 : (lane == 1 ? g1 : g2));
}

__global__ void k_cand_flag(int P, const double* __restrict__ px, const double* __restrict__ plp,
                            Body b, double margin, int* flag) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  int f = 0;
  for (int c = 0; c < 8 && !f; ++c) {
    double y[3];
    for (int d = 0; d < 3; ++d)
      y[d] = px[3 * (size_t)w + d] + (((c >> d) & 1) ? 1.0 : -1.0) * plp[3 * (size_t)w + d];
    if (body_distance(b, y, margin) <= margin) f = 1;
  }
  flag[w] = f;
}

__global__ void k_cand_write(int P, const int* __restrict__ flag, const int* __restrict__ pos,
                             int* cand) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < P && flag[w]) cand[pos[w]] = w;
}

// background basis of each candidate corner, in the leaf on the inside of the domain
__global__ void k_cand_basis(int nc, const int* __restrict__ cand, Geo g,
                             const double* __restrict__ px, const double* __restrict__ plp,
                             const uint64_t* __restrict__ lkey, const int* __restrict__ llev, int nl,
                             const int* __restrict__ corner, const int* __restrict__ cptr,
                             const int* __restrict__ cidx, const double* __restrict__ cw,
                             const int* __restrict__ node_dof, int* cb_n, int* cb_idx,
                             double* cb_phi, double* cb_y0, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * nc) return;
  int w = cand[i >> 3], c = i & 7;
  double Lo[3], Hi[3];
  domain_box(px + 3 * (size_t)w, plp + 3 * (size_t)w, g, Lo, Hi);
  int q[3];
  double X[3];
  for (int d = 0; d < 3; ++d) {
    int side = (c >> d) & 1;
    X[d] = side ? Hi[d] : Lo[d];
    int v = side ? (int)ceil(X[d]) - 1 : (int)floor(X[d]);
    q[d] = v < 0 ? 0 : (v > g.N - 1 ? g.N - 1 : v);
    cb_y0[3 * (size_t)i + d] = px[3 * (size_t)w + d] + (side ? 1.0 : -1.0) * plp[3 * (size_t)w + d];
  }
  int K = locate(lkey, nl, q[0], q[1], q[2]);
  int s = 1 << (g.D - llev[K]);
  int a[3];
  demorton(lkey[K], a);
  double xi[3];
  for (int d = 0; d < 3; ++d) xi[d] = (X[d] - (double)a[d]) / (double)s;
  int n = 0;
  int* ids = cb_idx + (size_t)i * MAXCB;
  double* ph = cb_phi + (size_t)i * MAXCB;
  for (int cc = 0; cc < 8; ++cc) {
    double f = 1.0;
    for (int d = 0; d < 3; ++d) f *= ((cc >> d) & 1) ? xi[d] : 1.0 - xi[d];
    int node = corner[8 * (size_t)K + cc];
    for (int t = cptr[node]; t < cptr[node + 1]; ++t) {
      int j = node_dof[cidx[t]];
      int slot = -1;
      for (int e = 0; e < n; ++e)
        if (ids[e] == j) slot = e;
      if (slot < 0) {
        if (n >= MAXCB || j < 0) {
          atomicOr(err, EB_SUPPORT);
          continue;
        }
        slot = n++;
        ids[slot] = j;
        ph[slot] = 0.0;
      }
      ph[slot] += cw[t] * f;
    }
  }
  cb_n[i] = n;
}

// the transpose of the corner basis: keys (dof << 32 | corner << 5 | entry),
// unused entries last
__global__ void k_ct_keys(int nc8, const int* __restrict__ cb_n, const int* __restrict__ cb_idx,
                          uint64_t* keys) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nc8 * MAXCB) return;
  int i = (int)(t / MAXCB), e = (int)(t % MAXCB);
  keys[t] = e < cb_n[i] ? ((uint64_t)(uint32_t)cb_idx[t] << 32) | ((uint64_t)i << 5) | (uint64_t)e
                        : ~0ULL;
}

// first entry of each row in the sorted keys
__global__ void k_ct_flag(long long n, const uint64_t* __restrict__ keys, int* flag) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint64_t k = keys[q];
  flag[q] = k != ~0ULL && (q == 0 || (keys[q - 1] >> 32) != (k >> 32));
}

__global__ void k_ct_write(long long n, const uint64_t* __restrict__ keys, const int* __restrict__ flag,
                           const int* __restrict__ pos, int nrow, int* crow, int* cptr, int* cent) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint64_t k = keys[q];
  if (k == ~0ULL) return;
  cent[q] = (int)(k & 0xffffffffULL);
  if (flag[q]) {
    crow[pos[q]] = (int)(k >> 32);
    cptr[pos[q]] = (int)q;
  }
  if (q == n - 1 || keys[q + 1] == ~0ULL) cptr[nrow] = (int)(q + 1);
}

// ------------------------------------------------------------------ triangulated body

// unit normal of every triangle (body frame)
__global__ void k_tri_fn(int nt, const double* __restrict__ v, const int* __restrict__ t, double* fn) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const double *a = v + 3 * (size_t)t[3 * i], *b = v + 3 * (size_t)t[3 * i + 1],
               *c = v + 3 * (size_t)t[3 * i + 2];
  double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) fn[3 * (size_t)i + d] = n[d] / l;
}

// edge pseudo-normals: the face normal plus that of the first other triangle
// (in index order) holding both ends of the edge
__global__ void k_tri_en(int nt, const int* __restrict__ t, const double* __restrict__ fn, double* en) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * nt) return;
  int i = e / 3, k = e % 3;
  int a = t[3 * i + k], b = t[3 * i + (k + 1) % 3];
  double N[3] = {fn[3 * (size_t)i], fn[3 * (size_t)i + 1], fn[3 * (size_t)i + 2]};
  for (int u = 0; u < nt; ++u) {
    if (u == i) continue;
    int ha = 0, hb = 0;
    for (int q = 0; q < 3; ++q) {
      ha |= t[3 * u + q] == a;
      hb |= t[3 * u + q] == b;
    }
    if (ha && hb) {
      for (int d = 0; d < 3; ++d) N[d] += fn[3 * (size_t)u + d];
      break;
    }
  }
  for (int d = 0; d < 3; ++d) en[3 * (size_t)e + d] = N[d];
}

// vertex pseudo-normals: angle-weighted sum of the face normals around the
// vertex (triangles in index order)
__global__ void k_tri_vn(int nv, int nt, const double* __restrict__ v, const int* __restrict__ t,
                         const double* __restrict__ fn, double* vn) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  double N[3] = {0.0, 0.0, 0.0};
  const double* a = v + 3 * (size_t)p;
  for (int u = 0; u < nt; ++u)
    for (int k = 0; k < 3; ++k) {
      if (t[3 * u + k] != p) continue;
      const double* b = v + 3 * (size_t)t[3 * u + (k + 1) % 3];
      const double* c = v + 3 * (size_t)t[3 * u + (k + 2) % 3];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cs = (e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2]) /
                  sqrt((e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) *
                       (e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
      double ang = acos(fmin(fmax(cs, -1.0), 1.0));
      for (int d = 0; d < 3; ++d) N[d] += ang * fn[3 * (size_t)u + d];
    }
  for (int d = 0; d < 3; ++d) vn[3 * (size_t)p + d] = N[d];
}

// ------------------------------------------------------------------ sliced storage

// storage order: one block per window of SLICE_WINDOW storage rows, a thread
// per dof row of the window; the window's dof rows by decreasing length, ties
// by dof (a rank by counting, so the order is the same on every run); rows at
// or beyond nd stay in place
__global__ void k_slice_order(int nd, int npad, const int* __restrict__ rp, int* row, int* pos) {
  __shared__ int len[SLICE_WINDOW];
  int w0 = blockIdx.x * SLICE_WINDOW, t = threadIdx.x, r = w0 + t;
  int n = min(SLICE_WINDOW, max(0, nd - w0));
  len[t] = t < n ? rp[r + 1] - rp[r] : -1;
  __syncthreads();
  if (r >= npad) return;
  if (t >= n) {
    row[r] = r;
    pos[r] = r;
    return;
  }
  int L = len[t], rank = 0;
  for (int j = 0; j < n; ++j) rank += (len[j] > L) || (len[j] == L && j < t);
  pos[r] = w0 + rank;
  row[w0 + rank] = r;
}

// width of each slice of 32 storage rows: longest row, rounded up to 4 blocks
__global__ void k_slice_width(int nd, int ns, const int* __restrict__ rp, const int* __restrict__ row, int* w) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  int m = 0;
  for (int sr = 32 * s; sr < 32 * s + 32; ++sr) {
    int r = row[sr];
    if (r < nd) m = max(m, rp[r + 1] - rp[r]);
  }
  w[s] = (m + 3) & ~3;
}

__global__ void k_slice_slots(int ns, const int* __restrict__ w, int* slots) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns) slots[s] = 32 * w[s];
}

__global__ void k_slice_base64(int ns, const int* __restrict__ pos, long long* base) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns) base[s] = pos[s];
}

// slot columns of each storage row: its dof row's sorted columns, then padding
// slots pointing at that row
__global__ void k_slice_cols(int nd, int ns, const int* __restrict__ rp, const int* __restrict__ col,
                             const int* __restrict__ w, const long long* __restrict__ base,
                             const int* __restrict__ row, int* scol) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int sr = (int)(t >> 5), lane = (int)(t & 31);
  if (sr >= 32 * ns) return;
  int s = sr >> 5, r = row[sr];
  int nb = r < nd ? rp[r + 1] - rp[r] : 0;
  for (int idx = lane; idx < w[s]; idx += 32)
    scol[sliced_slot(base[s], sr, idx)] = idx < nb ? col[rp[r] + idx] : (r < nd ? r : 0);
}

// ------------------------------------------------------------------ host helpers

int read_total(mpm_ctx* c, const int* scan_out, const int* cnt, int n) {
  if (n == 0) return 0;
  MPM_CUDA(cudaMemcpyAsync(c->h_int + 2, scan_out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaMemcpyAsync(c->h_int + 3, cnt + n - 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_int[2] + c->h_int[3];
}

int read_flag(mpm_ctx* c, int* d_any) {
  MPM_CUDA(cudaMemcpyAsync(c->h_int + 4, d_any, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  return c->h_int[4];
}

void tree_refine(mpm_ctx* c, mpm_mesh* m, const int* flag) {
  int n = m->nleaf;
  int* cnt = grow<int>(c, c->tmp[0], n);
  int* pos = grow<int>(c, m->scan, n);
  MPM_LAUNCH(k_child_count<<<grid_for(n, 256), 256, 0, c->stream>>>(n, flag, cnt));
  cub_exclusive_sum_int(c, cnt, pos, n);
  int total = read_total(c, pos, cnt, n);
  uint64_t* okey = grow<uint64_t>(c, m->leaf_tmp_key, total);
  int* olev = grow<int>(c, m->leaf_tmp_lev, total);
  MPM_LAUNCH(k_refine_write<<<grid_for(n, 256), 256, 0, c->stream>>>(n, ptr<uint64_t>(m->leaf_key),
                                                          ptr<int>(m->leaf_lev), flag, pos, m->g.D,
                                                          okey, olev));
  std::swap(m->leaf_key, m->leaf_tmp_key);
  std::swap(m->leaf_lev, m->leaf_tmp_lev);
  m->nleaf = total;
}

void tree_balance(mpm_ctx* c, mpm_mesh* m) {
  int* any = (int*)(c->d_red + 8);
  for (int it = 0; it < 4 * m->g.D + 8; ++it) {
    int n = m->nleaf;
    int* flag = grow<int>(c, m->flag, n);
    MPM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * n, c->stream));
    MPM_CUDA(cudaMemsetAsync(any, 0, sizeof(int), c->stream));
    MPM_LAUNCH(k_balance_mark<<<grid_for(n, 256), 256, 0, c->stream>>>(n, ptr<uint64_t>(m->leaf_key),
                                                            ptr<int>(m->leaf_lev), m->g, flag, any));
    if (!read_flag(c, any)) return;
    tree_refine(c, m, flag);
  }
  throw CudaError(MPM_ERR_BALANCE, "octree balance did not settle");
}

int bits_for(long long v) {
  int b = 1;
  while ((1LL << b) <= v) ++b;
  return b;
}

}  // namespace

// ------------------------------------------------------------------ the build

// a triangulated body: check its arrays, then its pseudo-normals and bounding box
void tri_setup(mpm_ctx* c, mpm_mesh* m, const mpm_rigid& b) {
  cudaStream_t st = c->stream;
  if (b.ntri <= 0 || b.nvert <= 0 || !b.tri_v || !b.tri_t)
    throw CudaError(MPM_ERR_ARG, "triangulated body: need ntri > 0, nvert > 0 and both arrays");
  std::vector<double> v(3 * (size_t)b.nvert);
  std::vector<int> t(3 * (size_t)b.ntri);
  MPM_CUDA(cudaMemcpyAsync(v.data(), b.tri_v, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, st));
  MPM_CUDA(cudaMemcpyAsync(t.data(), b.tri_t, sizeof(int) * t.size(), cudaMemcpyDeviceToHost, st));
  MPM_CUDA(cudaStreamSynchronize(st));
  for (int i : t)
    if (i < 0 || i >= b.nvert) throw CudaError(MPM_ERR_ARG, "triangulated body: vertex index out of range");
  for (int d = 0; d < 3; ++d) {
    m->tri_lo[d] = 1e300;
    m->tri_hi[d] = -1e300;
  }
  for (int i = 0; i < b.nvert; ++i)
    for (int d = 0; d < 3; ++d) {
      m->tri_lo[d] = std::min(m->tri_lo[d], v[3 * (size_t)i + d]);
      m->tri_hi[d] = std::max(m->tri_hi[d], v[3 * (size_t)i + d]);
    }
  double* fn = grow<double>(c, m->tri_fn, 3 * (size_t)b.ntri);
  double* en = grow<double>(c, m->tri_en, 9 * (size_t)b.ntri);
  double* vn = grow<double>(c, m->tri_vn, 3 * (size_t)b.nvert);
  MPM_LAUNCH(k_tri_fn<<<grid_for(b.ntri, 128), 128, 0, st>>>(b.ntri, b.tri_v, b.tri_t, fn));
  MPM_LAUNCH(k_tri_en<<<grid_for(3LL * b.ntri, 128), 128, 0, st>>>(b.ntri, b.tri_t, fn, en));
  MPM_LAUNCH(k_tri_vn<<<grid_for(b.nvert, 128), 128, 0, st>>>(b.nvert, b.ntri, b.tri_v, b.tri_t, fn, vn));
}

void build_mesh(mpm_ctx* c, mpm_mesh* m, const mpm_domain& dom, const mpm_rigid& body,
                const mpm_adapt& ad, const mpm_material& mat, mpm_points* pts, int flags,
                double cand_extra) {
  cudaStream_t st = c->stream;
  m->built = 0;
  ++m->gen;
  m->dom = dom;
  m->body = body;
  m->ad = ad;
  m->mat = mat;
  Geo& g = m->g;
  g.D = dom.depth_max;
  g.N = 1 << g.D;
  g.L = dom.L;
  g.unit = dom.L / ldexp(1.0, g.D);
  g.scale = ldexp(1.0, g.D) / dom.L;
  int* d_err = c->d_err;
  if (body.kind == 3) tri_setup(c, m, body);
  const Body bv = body_view(m, body);

  // ---- a1: uniform tree at depth_min, then Sec. 5 refinement + balance
  {
    int n = 1 << (3 * dom.depth_min);
    grow<uint64_t>(c, m->leaf_key, n);
    grow<int>(c, m->leaf_lev, n);
    MPM_LAUNCH(k_tree_uniform<<<grid_for(n, 256), 256, 0, st>>>(n, 3 * (g.D - dom.depth_min), dom.depth_min,
                                                     ptr<uint64_t>(m->leaf_key), ptr<int>(m->leaf_lev)));
    m->nleaf = n;
    if (body.kind != 0 && dom.depth_max > dom.depth_min) {
      int* any = (int*)(c->d_red + 8);
      bool settled = false;
      for (int it = 0; it < 4 * g.D + 8; ++it) {
        int nl = m->nleaf;
        int* flag = grow<int>(c, m->flag, nl);
        MPM_CUDA(cudaMemsetAsync(any, 0, sizeof(int), st));
        MPM_LAUNCH(k_mark_refine<<<grid_for(nl, 256), 256, 0, st>>>(nl, ptr<uint64_t>(m->leaf_key),
                                                         ptr<int>(m->leaf_lev), g, bv, ad.dx_region,
                                                         dom.depth_max, flag, any));
        if (!read_flag(c, any)) {
          settled = true;
          break;
        }
        tree_refine(c, m, flag);
        tree_balance(c, m);
      }
      if (!settled) throw CudaError(MPM_ERR_BALANCE, "octree refinement did not settle");
    }
  }
  int nl = m->nleaf;
  const uint64_t* lkey = ptr<uint64_t>(m->leaf_key);
  const int* llev = ptr<int>(m->leaf_lev);

  // ---- a3: GIMP refinement, in the caller's arrays
  for (SplitRound& r : m->split_log) {
    free_buf(c, r.flag);
    free_buf(c, r.rank);
  }
  m->split_log.clear();
  if (!(flags & 1)) {
    for (int round = 0; round < 32; ++round) {
      int P = pts->count;
      int* flag = grow<int>(c, c->tmp[1], P);
      int* rank = grow<int>(c, c->tmp[2], P);
      MPM_LAUNCH(k_split_flag<<<grid_for(P, 128), 128, 0, st>>>(P, pts->x, pts->lp, pts->l0, lkey, llev, nl, g,
                                                     ad.beta, flag, d_err));
      cub_exclusive_sum_int(c, flag, rank, P);
      int cnt = read_total(c, rank, flag, P);
      if (cnt == 0) break;
      long long np = (long long)P + 7LL * cnt;
      if (np > pts->capacity)
        throw CudaError(MPM_ERR_CAPACITY, "GIMP split needs " + std::to_string(np) +
                                              " points, capacity is " + std::to_string(pts->capacity));
      MPM_LAUNCH(k_split_write<<<grid_for(P, 128), 128, 0, st>>>(P, flag, rank, *pts));
      if (m->record_splits) {
        m->split_log.emplace_back();
        SplitRound& r = m->split_log.back();
        r.P = P;
        r.cnt = cnt;
        MPM_CUDA(cudaMemcpyAsync(grow<int>(c, r.flag, P), flag, sizeof(int) * P, cudaMemcpyDeviceToDevice, st));
        MPM_CUDA(cudaMemcpyAsync(grow<int>(c, r.rank, P), rank, sizeof(int) * P, cudaMemcpyDeviceToDevice, st));
      }
      pts->count = (int)np;
      if (round == 31) throw CudaError(MPM_ERR_SUPPORT, "GIMP split did not settle");
    }
  }
  int P = pts->count;
  m->np = P;

  // ---- a2: nodes, hanging classification, constraints
  {
    uint64_t* ck = grow<uint64_t>(c, c->tmp[3], 8 * (size_t)nl);
    uint64_t* alt = grow<uint64_t>(c, c->tmp[4], 8 * (size_t)nl);
    MPM_LAUNCH(k_corner_keys<<<grid_for(nl, 256), 256, 0, st>>>(nl, lkey, llev, g.D, ck));
    cub_sort_u64(c, ck, alt, 8 * nl, 3 * (g.D + 1));
    uint64_t* nkey = grow<uint64_t>(c, m->node_key, 8 * (size_t)nl);
    int nn = cub_unique_u64(c, ck, nkey, 8 * nl);
    m->nnode = nn;
    int* corner = grow<int>(c, m->corner, 8 * (size_t)nl);
    MPM_LAUNCH(k_corner_ids<<<grid_for(nl, 256), 256, 0, st>>>(nl, lkey, llev, g.D, nkey, nn, corner));
    int* hang = grow<int>(c, m->hang, nn);
    int* owner = grow<int>(c, m->owner, nn);
    MPM_LAUNCH(k_hang<<<grid_for(nn, 256), 256, 0, st>>>(nn, nkey, lkey, llev, nl, g, hang, owner));
    NodeView v{nkey, lkey, llev, corner, hang, owner, g.D};
    int* cnt = grow<int>(c, c->tmp[0], nn + 1);
    int* cptr = grow<int>(c, m->cptr, nn + 1);
    MPM_LAUNCH(k_con_count<<<grid_for(nn, 128), 128, 0, st>>>(nn, v, cnt, d_err));
    MPM_CUDA(cudaMemsetAsync(cnt + nn, 0, sizeof(int), st));
    cub_exclusive_sum_int(c, cnt, cptr, nn + 1);
    int ncon = read_total(c, cptr, cnt, nn + 1);
    m->ncon = ncon;
    int* cidx = grow<int>(c, m->cidx, ncon);
    double* cw = grow<double>(c, m->cw, ncon);
    MPM_LAUNCH(k_con_fill<<<grid_for(nn, 128), 128, 0, st>>>(nn, v, cptr, cidx, cw));
    int st2 = check_device_error(c, "node constraints");
    if (st2) throw CudaError(st2, c->err);
  }
  const int* corner = ptr<int>(m->corner);
  const int* cptr = ptr<int>(m->cptr);
  const int* cidx = ptr<int>(m->cidx);
  const double* cw = ptr<double>(m->cw);
  int nn = m->nnode;

  // ---- points: sort by leaf of the centre, gather the step-start state
  {
    int* cell = grow<int>(c, c->tmp[1], P);
    int* idx = grow<int>(c, c->tmp[2], P);
    int* perm = grow<int>(c, m->perm, P);
    int* pcell = grow<int>(c, m->pcell, P);
    MPM_LAUNCH(k_point_cell<<<grid_for(P, 256), 256, 0, st>>>(P, pts->x, g, lkey, nl, cell, idx));
    cub_sort_pairs_int(c, cell, pcell, idx, perm, P, bits_for(nl));
    MPM_LAUNCH(k_gather_points<<<grid_for(P, 256), 256, 0, st>>>(
        P, perm, *pts, grow<double>(c, m->px, 3 * (size_t)P), grow<double>(c, m->plp, 3 * (size_t)P),
        grow<double>(c, m->pl0, 3 * (size_t)P), grow<double>(c, m->pF, 9 * (size_t)P),
        grow<double>(c, m->pbe, 6 * (size_t)P), grow<double>(c, m->pV0, P),
        grow<double>(c, m->pmass, P), grow<double>(c, m->pE, P), grow<double>(c, m->pys, P),
        pts->v ? grow<double>(c, m->pv, 3 * (size_t)P) : nullptr));
    m->has_v = pts->v != nullptr;
  }

  // ---- a4: discrete GIMP basis
  int* nsup = grow<int>(c, m->nsup, P);
  int* sidx = grow<int>(c, m->sidx, (size_t)P * MAXS);
  double* S = grow<double>(c, m->S, (size_t)P * MAXS);
  double* dS = grow<double>(c, m->dS, (size_t)P * MAXS * 3);
  int* pop = grow<int>(c, m->populated, nl);
  double* betaK = grow<double>(c, m->betaK, nl);
  MPM_CUDA(cudaMemsetAsync(pop, 0, sizeof(int) * nl, st));
  MPM_CUDA(cudaMemsetAsync(betaK, 0, sizeof(double) * nl, st));
  MPM_LAUNCH_P(MPM_PROF_BASIS, k_basis<<<grid_for(P, BW), 32 * BW, 0, st>>>(P, g, ptr<double>(m->px), ptr<double>(m->plp),
                                               ptr<double>(m->pE), lkey, llev, nl, corner, cptr, cidx,
                                               cw, nsup, sidx, S, dS, pop,
                                               (unsigned long long*)betaK, d_err));
  {
    int e = check_device_error(c, "GIMP basis");
    if (e) throw CudaError(e, c->err);
  }
  // active nodes -> dofs (Morton order)
  {
    int* active = grow<int>(c, c->tmp[0], nn);
    int* pos = grow<int>(c, c->tmp[1], nn);
    MPM_CUDA(cudaMemsetAsync(active, 0, sizeof(int) * nn, st));
    MPM_LAUNCH(k_mark_active<<<grid_for((long long)P * MAXS, 256), 256, 0, st>>>(P, nsup, sidx, active));
    cub_exclusive_sum_int(c, active, pos, nn);
    int nd = read_total(c, pos, active, nn);
    m->ndof = nd;
    int* node_dof = grow<int>(c, m->node_dof, nn);
    int* dof_node = grow<int>(c, m->dof_node, nd);
    MPM_LAUNCH(k_number_dofs<<<grid_for(nn, 256), 256, 0, st>>>(nn, active, pos, node_dof, dof_node));
    MPM_LAUNCH(k_sidx_to_dof<<<grid_for((long long)P * MAXS, 256), 256, 0, st>>>(P, nsup, node_dof, sidx));
    Planes pl{};
    pl.n = dom.nbc;
    for (int b = 0; b < dom.nbc; ++b) {
      pl.axis[b] = dom.bc_axis[b];
      pl.pos[b] = (int)floor(dom.bc_pos[b] * g.scale + 0.5);
      pl.mask[b] = dom.bc_mask[b];
    }
    MPM_LAUNCH(k_dof_mask<<<grid_for(nd, 256), 256, 0, st>>>(nd, dof_node, ptr<uint64_t>(m->node_key), pl,
                                                  grow<int>(c, m->dof_mask, nd)));
  }
  int nd = m->ndof;
  const int* node_dof = ptr<int>(m->node_dof);

  // ---- a6 (faces): boundary elements and ghost faces
  int nf = 0;
  {
    int* isB = grow<int>(c, m->isB, nl);
    MPM_LAUNCH(k_boundary_elements<<<grid_for(nl, 256), 256, 0, st>>>(nl, lkey, llev, g, pop, isB));
    if (mat.ghost_on) {
      int* flag = grow<int>(c, c->tmp[0], 6 * (size_t)nl);
      int* pos = grow<int>(c, c->tmp[1], 6 * (size_t)nl);
      MPM_LAUNCH(k_ghost_face_flag<<<grid_for(6LL * nl, 256), 256, 0, st>>>(nl, lkey, llev, g, pop, isB, flag));
      cub_exclusive_sum_int(c, flag, pos, 6 * nl);
      nf = read_total(c, pos, flag, 6 * nl);
      int* face = grow<int>(c, m->gface, 4 * (size_t)nf);
      MPM_LAUNCH(k_ghost_face_write<<<grid_for(6LL * nl, 256), 256, 0, st>>>(nl, lkey, llev, g, flag, pos, face));
      MPM_LAUNCH(k_ghost_face_dofs<<<grid_for(nf, 128), 128, 0, st>>>(nf, face, corner, cptr, cidx, node_dof,
                                                          grow<int>(c, m->gdof, (size_t)nf * MAXG),
                                                          grow<int>(c, m->gn, nf), d_err));
    }
    m->nghost = nf;
  }

  // ---- a5: sources of every row, then the pattern
  {
    int* off = grow<int>(c, c->tmp[0], P + 1);
    MPM_CUDA(cudaMemsetAsync(off + P, 0, sizeof(int), st));
    // nsup[P] is not defined: scan P entries and read the total
    cub_exclusive_sum_int(c, nsup, off, P);
    long long npt = read_total(c, off, nsup, P);
    long long total = npt + (long long)nf * MAXG;
    uint64_t* keys = grow<uint64_t>(c, m->src_key, total);
    uint64_t* alt = grow<uint64_t>(c, c->tmp[3], total);
    MPM_LAUNCH(k_src_keys_points<<<grid_for((long long)P * MAXS, 256), 256, 0, st>>>(P, nsup, sidx, off, keys));
    if (nf) {
      // unused face slots keep an out-of-range row so that they sort last
      MPM_CUDA(cudaMemsetAsync(keys + npt, 0xff, sizeof(uint64_t) * (size_t)nf * MAXG, st));
      MPM_LAUNCH(k_src_keys_faces<<<grid_for((long long)nf * MAXG, 256), 256, 0, st>>>(
          nf, P, ptr<int>(m->gn), ptr<int>(m->gdof), npt, keys));
    }
    cub_sort_u64(c, keys, alt, (int)total, 64);
    long long* sptr = grow<long long>(c, m->src_ptr, nd + 1);
    MPM_CUDA(cudaMemsetAsync(sptr, 0, sizeof(long long) * (nd + 1), st));
    MPM_LAUNCH(k_src_ptr<<<grid_for(total, 256), 256, 0, st>>>(total, keys, nd, sptr));
    m->nsrc = total;
    {
      unsigned long long* np2 = (unsigned long long*)(c->d_red + 50);
      MPM_CUDA(cudaMemsetAsync(np2, 0, sizeof(unsigned long long), st));
      MPM_LAUNCH(k_support_pairs<<<grid_for(P, 256), 256, 0, st>>>(P, nsup, np2));
      MPM_CUDA(cudaMemcpyAsync(&m->npair, np2, sizeof(long long), cudaMemcpyDeviceToHost, st));
    }
    int* rowcnt = grow<int>(c, m->rowcnt, nd + 1);
    int* rp = grow<int>(c, m->row_ptr, nd + 1);
    MPM_CUDA(cudaMemsetAsync(rowcnt + nd, 0, sizeof(int), st));
    MPM_LAUNCH_P(MPM_PROF_PATTERN, k_pattern_rows<<<grid_for(nd, PW), 32 * PW, 0, st>>>(nd, P, 0, sptr, keys, nsup, sidx,
                                                         ptr<int>(m->gn), ptr<int>(m->gdof), rowcnt,
                                                         nullptr, nullptr, d_err));
    cub_exclusive_sum_int(c, rowcnt, rp, nd + 1);
    int nnzb = read_total(c, rp, rowcnt, nd + 1);
    {
      int e = check_device_error(c, "block pattern");
      if (e) throw CudaError(e, c->err);
    }
    m->nnzb = nnzb;
    int* col = grow<int>(c, m->col, nnzb);
    MPM_LAUNCH_P(MPM_PROF_PATTERN, k_pattern_rows<<<grid_for(nd, PW), 32 * PW, 0, st>>>(nd, P, 1, sptr, keys, nsup, sidx,
                                                         ptr<int>(m->gn), ptr<int>(m->gdof), rowcnt,
                                                         rp, col, d_err));
    // longest row (for the solver's launch shapes)
    std::vector<int> h(nd + 1);
    MPM_CUDA(cudaMemcpyAsync(h.data(), rp, sizeof(int) * (nd + 1), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    int mr = 0;
    for (int r = 0; r < nd; ++r) mr = std::max(mr, h[r + 1] - h[r]);
    m->maxrow = mr;
    // sliced storage of the stiffness
    int ns = (nd + 31) / 32;
    m->nslice = ns;
    int* sw = grow<int>(c, m->slice_w, ns + 1);
    int* slots = grow<int>(c, c->tmp[1], ns + 1);
    int* spos = grow<int>(c, c->tmp[2], ns + 1);
    int* srow = grow<int>(c, m->srow, 32 * (size_t)ns);
    int* rpos = grow<int>(c, m->spos, 32 * (size_t)ns);
    MPM_LAUNCH(k_slice_order<<<(32 * ns + SLICE_WINDOW - 1) / SLICE_WINDOW, SLICE_WINDOW, 0, st>>>(nd, 32 * ns, rp, srow, rpos));
    MPM_LAUNCH(k_slice_width<<<grid_for(ns, 256), 256, 0, st>>>(nd, ns, rp, srow, sw));
    MPM_LAUNCH(k_slice_slots<<<grid_for(ns, 256), 256, 0, st>>>(ns, sw, slots));
    MPM_CUDA(cudaMemsetAsync(slots + ns, 0, sizeof(int), st));
    cub_exclusive_sum_int(c, slots, spos, ns + 1);
    m->nslot = read_total(c, spos, slots, ns + 1);
    long long* sb = grow<long long>(c, m->slice_base, ns + 1);
    MPM_LAUNCH(k_slice_base64<<<grid_for(ns + 1, 256), 256, 0, st>>>(ns + 1, spos, sb));
    int* scol = grow<int>(c, m->scol, m->nslot);
    MPM_LAUNCH(k_slice_cols<<<grid_for(32LL * 32 * ns, 256), 256, 0, st>>>(nd, ns, rp, col, sw, sb, srow, scol));
  }
  const int* rp = ptr<int>(m->row_ptr);
  const int* col = ptr<int>(m->col);

  // ---- a6 (matrix): ghost coefficients
  {
    double* kg = grow<double>(c, m->kg, m->nnzb);
    MPM_CUDA(cudaMemsetAsync(kg, 0, sizeof(double) * m->nnzb, st));
    if (nf) {
      double* gJ = grow<double>(c, m->gJ, 4 * (size_t)nf * MAXG);
      double* gco = grow<double>(c, m->gcoef, nf);
      MPM_LAUNCH(k_ghost_jumps<<<grid_for(nf, 4), 128, 0, st>>>(nf, g, mat.kappa, ptr<int>(m->gface), lkey, llev,
                                                               betaK, ptr<int>(m->gdof), ptr<int>(m->gn),
                                                               corner, cptr, cidx, cw, node_dof, gJ, gco));
      MPM_LAUNCH(k_ghost_rows<<<grid_for(nd, 8), 256, 0, st>>>(nd, P, ptr<long long>(m->src_ptr),
                                                              ptr<uint64_t>(m->src_key), ptr<int>(m->gdof),
                                                              ptr<int>(m->gn), gJ, gco, rp, col, kg));
    }
  }

  // ---- gravity force at load 1: f_ext,v = sum_p S_vp m_p g
  {
    double* fext = grow<double>(c, m->fext, 3 * (size_t)nd);
    MPM_CUDA(cudaMemsetAsync(fext, 0, sizeof(double) * 3 * nd, st));
    if (mat.g[0] != 0.0 || mat.g[1] != 0.0 || mat.g[2] != 0.0)
      MPM_LAUNCH(k_fext_rows<<<grid_for(nd, 8), 256, 0, st>>>(nd, P, ptr<long long>(m->src_ptr),
                                                             ptr<uint64_t>(m->src_key), S,
                                                             ptr<double>(m->pmass), mat.g[0], mat.g[1],
                                                             mat.g[2], fext));
  }

  // ---- contact candidates: domains with a corner within 4 finest cells of the
  // body (plus cand_extra: a free body's motion over the step)
  m->ncand = 0;
  m->nct = 0;
  if (mat.contact_on && body.kind != 0) {
    int* flag = grow<int>(c, c->tmp[0], P);
    int* pos = grow<int>(c, c->tmp[1], P);
    MPM_LAUNCH(k_cand_flag<<<grid_for(P, 256), 256, 0, st>>>(P, ptr<double>(m->px), ptr<double>(m->plp), bv,
                                                  4.0 * g.unit + cand_extra, flag));
    cub_exclusive_sum_int(c, flag, pos, P);
    int nc = read_total(c, pos, flag, P);
    m->ncand = nc;
    if (nc) {
      int* cand = grow<int>(c, m->cand, nc);
      MPM_LAUNCH(k_cand_write<<<grid_for(P, 256), 256, 0, st>>>(P, flag, pos, cand));
      MPM_LAUNCH(k_cand_basis<<<grid_for(8LL * nc, 128), 128, 0, st>>>(
          nc, cand, g, ptr<double>(m->px), ptr<double>(m->plp), lkey, llev, nl, corner, cptr, cidx,
          cw, node_dof, grow<int>(c, m->cb_n, 8 * (size_t)nc),
          grow<int>(c, m->cb_idx, 8 * (size_t)nc * MAXCB),
          grow<double>(c, m->cb_phi, 8 * (size_t)nc * MAXCB),
          grow<double>(c, m->cb_y0, 24 * (size_t)nc), d_err));
      // the transpose of the corner basis, rows with their (corner, entry)
      // lists in sorted order, for the contact row gather
      long long nk = 8LL * nc * MAXCB;
      uint64_t* keys = grow<uint64_t>(c, c->tmp[4], nk);
      uint64_t* alt = grow<uint64_t>(c, c->tmp[5], nk);
      MPM_LAUNCH(k_ct_keys<<<grid_for(nk, 256), 256, 0, st>>>(8 * nc, ptr<int>(m->cb_n), ptr<int>(m->cb_idx), keys));
      cub_sort_u64(c, keys, alt, (int)nk, 64);
      int* cflag = grow<int>(c, c->tmp[6], nk + 1);
      int* cpos = grow<int>(c, c->tmp[7], nk + 1);
      MPM_LAUNCH(k_ct_flag<<<grid_for(nk, 256), 256, 0, st>>>(nk, keys, cflag));
      cub_exclusive_sum_int(c, cflag, cpos, (int)nk);
      int nrow = read_total(c, cpos, cflag, (int)nk);
      m->nct = nrow;
      MPM_LAUNCH(k_ct_write<<<grid_for(nk, 256), 256, 0, st>>>(
          nk, keys, cflag, cpos, nrow, grow<int>(c, m->ct_row, nrow + 1), grow<int>(c, m->ct_ptr, nrow + 1),
          grow<int>(c, m->ct_ent, nk)));
    }
  }

  // FP32 copies of the basis for the mixed-precision path are made on demand
  // by the assembly; count the largest support
  {
    std::vector<int> h(P);
    MPM_CUDA(cudaMemcpyAsync(h.data(), nsup, sizeof(int) * P, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    int mx = 0;
    for (int v : h) mx = std::max(mx, v);
    m->maxs = mx;
  }
  int nh = 0;
  {
    std::vector<int> h(nn);
    MPM_CUDA(cudaMemcpyAsync(h.data(), ptr<int>(m->hang), sizeof(int) * nn, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    for (int v : h) nh += v;
  }
  m->nhang = nh;
  m->built = 1;
}

Body body_view(const mpm_mesh* m, const mpm_rigid& b) {
  Body v{};
  v.b = b;
  if (b.kind == 3) {
    v.fn = ptr<double>(m->tri_fn);
    v.en = ptr<double>(m->tri_en);
    v.vn = ptr<double>(m->tri_vn);
    for (int d = 0; d < 3; ++d) {
      v.lo[d] = m->tri_lo[d];
      v.hi[d] = m->tri_hi[d];
    }
  }
  return v;
}

}  // namespace mpm
