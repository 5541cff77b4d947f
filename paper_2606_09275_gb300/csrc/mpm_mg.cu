// Geometric multigrid preconditioner for the symmetric stiffness: a V-cycle
// used inside PCG, the multilevel counterpart of the Jacobi-type
// preconditioning that Sec. 1 names for Krylov solvers.
//
// Levels: the octree dofs (fine), then the active nodes of uniform grids of
// depth d1 > d2 > ... > 1.  d1 is at most the coarsest leaf depth, so every
// coarse trilinear field lies in the fine octree space and the prolongation P
// is plain trilinear interpolation at the fine node positions (components
// fixed by a Dirichlet plane are dropped from P).  Coarse operators are
// Galerkin products A_c = P^T A P, accumulated by one warp per finer-level row
// into the coarse rows by 64-bit integer atomics on a fixed-point copy (exact
// integer sums, so the operator is the same bit for bit whatever the order of
// the atomics), and stored per stencil offset on the uniform grid.
// Restrictions gather the stored residual of the finer level in a fixed
// order (level 1 through the transpose of P, sorted by fine dof);
// prolongations gather.  The
// smoother is l1 block Jacobi, M = D + diag(sum over the row's off-diagonal
// |entries|), damped by a fixed weight w < 2 (kSmoothW), which is convergent
// without eigenvalue estimates; one sweep before and one after the coarse
// correction, so the V-cycle is symmetric positive definite.  The depth-1
// level is solved with a dense inverse.
#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>

#include "mpm_internal.cuh"
#include "mpm_sliced.cuh"

namespace mpm {
namespace {

constexpr int MGW = 4;  // warps per block of the warp-per-row level kernels

// packed grid coordinates (coarse grids have at most 2^7 + 1 nodes per axis)
__host__ __device__ inline int pack3(int x, int y, int z) { return x | (y << 10) | (z << 20); }
__host__ __device__ inline void unpack3(int v, int* c) {
  c[0] = v & 1023;
  c[1] = (v >> 10) & 1023;
  c[2] = v >> 20;
}

// k < 0 (BiCGStab): only the solve's `done` flag stops the work
__device__ inline bool skip(const Scal* sk, int k) {
  return sk && (sk->done || (k >= 0 && sk->rr[(k + 1) % 3] <= sk->thr));
}

// ---------------------------------------------------------------- structure

// level-1 interpolation weights of every fine dof; marks the coarse nodes used
__global__ void k_mg_p1(int nd, int D, int d1, const int* __restrict__ dof_node,
                        const uint64_t* __restrict__ nkey, const int* __restrict__ mask, int* pidx,
                        float* pw, int* active, int* freeb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  int X[3];
  demorton(nkey[dof_node[i]], X);
  int sh = D - d1, n = 1 << d1, n1 = n + 1;
  int cc[3];
  float t[3];
  for (int d = 0; d < 3; ++d) {
    cc[d] = min(X[d] >> sh, n - 1);
    t[d] = (float)(X[d] - (cc[d] << sh)) / (float)(1 << sh);
  }
  int fr = 7 & ~mask[i];
  int q = 0;
  for (int c = 0; c < 8; ++c) {
    float w = 1.0f;
    for (int d = 0; d < 3; ++d) w *= ((c >> d) & 1) ? t[d] : 1.0f - t[d];
    if (w == 0.0f) continue;
    int lin = (cc[0] + (c & 1)) + n1 * ((cc[1] + ((c >> 1) & 1)) + n1 * (cc[2] + ((c >> 2) & 1)));
    pidx[8 * (size_t)i + q] = lin;
    pw[8 * (size_t)i + q] = w;
    ++q;
    active[lin] = 1;
    if (fr) atomicOr(freeb + lin, fr);
  }
  for (; q < 8; ++q) pidx[8 * (size_t)i + q] = -1;
}

// coarse nodes used by the interpolation from the active rows of a uniform level
__global__ void k_mg_mark_u(int nrow, const int* __restrict__ xyz, const int* __restrict__ mask,
                            int n1c, int* active, int* freeb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrow) return;
  int c[3];
  unpack3(xyz[i], c);
  int fr = 7 & ~mask[i];
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = c[d] >> 1;
    hi[d] = (c[d] + 1) >> 1;
  }
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        int lin = x + n1c * (y + n1c * z);
        active[lin] = 1;
        if (fr) atomicOr(freeb + lin, fr);
      }
}

// compact numbering of the active grid nodes
__global__ void k_mg_compact(int ng, int n1, const int* __restrict__ active,
                             const int* __restrict__ scan, const int* __restrict__ freeb, int* gid,
                             int* xyz, int* mask) {
  int lin = blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= ng) return;
  if (!active[lin]) {
    gid[lin] = -1;
    return;
  }
  int r = scan[lin];
  gid[lin] = r;
  int x = lin % n1, y = (lin / n1) % n1, z = lin / (n1 * n1);
  xyz[r] = pack3(x, y, z);
  mask[r] = 7 & ~freeb[lin];
}

// fine -> level-1 entries: grid ids to rows
__global__ void k_mg_p1_rows(int nd, const int* __restrict__ gid, int* pidx) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8LL * nd) return;
  int lin = pidx[e];
  if (lin >= 0) pidx[e] = gid[lin];
}

// the transpose of the level-1 interpolation: keys (level-1 row << 35 | the
// entry's position 8 i + q in pidx), unused entries last
__global__ void k_mg_tkeys(int nd, const int* __restrict__ pidx, uint64_t* keys) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8LL * nd) return;
  int a = pidx[e];
  keys[e] = a < 0 ? ~0ULL : ((uint64_t)a << 35) | (uint64_t)e;
}

// first entry of each level-1 row among the sorted keys (row nrow: the count)
__global__ void k_mg_tptr(int nrow, long long n, const uint64_t* __restrict__ keys, int* tptr,
                          int* tmax) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a > nrow) return;
  auto first = [&](uint64_t k) {
    long long lo = 0, hi = n;
    while (lo < hi) {
      long long mid = (lo + hi) >> 1;
      if (keys[mid] < k)
        lo = mid + 1;
      else
        hi = mid;
    }
    return lo;
  };
  long long b = first((uint64_t)a << 35);
  tptr[a] = (int)b;
  if (a < nrow) atomicMax(tmax, (int)(first((uint64_t)(a + 1) << 35) - b));
}

// (fine dof, weight) of each entry of the transpose
__global__ void k_mg_tent(long long n, const uint64_t* __restrict__ keys, const float* __restrict__ pw,
                          int* tidx, float* tw) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint64_t k = keys[e];
  if (k == ~0ULL) return;
  long long f = (long long)(k & ((1ULL << 35) - 1));
  tidx[e] = (int)(f >> 3);
  tw[e] = pw[f];
}

// largest level-1 cell distance between the two dofs of any stored block
__global__ void k_mg_reach(int nd, int D, int d1, const int* __restrict__ rp,
                           const int* __restrict__ col, const int* __restrict__ dof_node,
                           const uint64_t* __restrict__ nkey, int* reach) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nd) return;
  int sh = D - d1, n = 1 << d1;
  int X[3], ci[3];
  demorton(nkey[dof_node[r]], X);
  for (int d = 0; d < 3; ++d) ci[d] = min(X[d] >> sh, n - 1);
  int m = 0;
  for (int s = rp[r] + lane; s < rp[r + 1]; s += 32) {
    int Y[3];
    demorton(nkey[dof_node[col[s]]], Y);
    for (int d = 0; d < 3; ++d) m = max(m, abs(min(Y[d] >> sh, n - 1) - ci[d]));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && m > 0) atomicMax(reach, m);
}

// ---------------------------------------------------------------- Galerkin products

// Fixed-point scale of a Galerkin product whose entries are sums of terms
// with sum |term| <= B: 2^(60 - floor(log2 B)), so that every partial sum
// stays below 2^61 in magnitude and the 64-bit integer accumulation cannot
// overflow; one unit is at most 2^-60 B (below FP64 rounding of the sum).
// 64-bit accumulators (FP64 operators): partial sums below 2^61; 32-bit
// (FP32 operators, 24-bit significands): below 2^30, one unit at most
// 2^-29 B, below FP32 rounding of the larger entries
template <class ACC>
__device__ inline double fixed_scale(double B) {
  if (!(B > 0.0) || !isfinite(B)) return 1.0;
  return ldexp(1.0, (sizeof(ACC) == 8 ? 60 : 29) - ilogb(B));
}

__device__ inline void fixed_add(unsigned long long* a, double v, double sc) {
  if (v != 0.0) atomicAdd(a, (unsigned long long)__double2ll_rn(v * sc));
}
__device__ inline void fixed_add(unsigned int* a, double v, double sc) {
  if (v != 0.0) atomicAdd(a, (unsigned int)__double2int_rn(v * sc));
}
__device__ inline double fixed_value(unsigned long long v) { return (double)(long long)v; }
__device__ inline double fixed_value(unsigned int v) { return (double)(int)v; }

// fixed point -> operator values
template <class T, class ACC>
__global__ void k_mg_from_fixed(long long n, const ACC* __restrict__ acc,
                                const unsigned long long* __restrict__ bnd, double cnt, T* A) {
  double inv = 1.0 / fixed_scale<ACC>(__longlong_as_double((long long)*bnd) * cnt);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    A[i] = (T)(fixed_value(acc[i]) * inv);
}

__device__ inline int stencil_index(const int* cb, const int* ca, int R) {
  int S1 = 2 * R + 1;
  int dx = cb[0] - ca[0] + R, dy = cb[1] - ca[1] + R, dz = cb[2] - ca[2] + R;
  if ((unsigned)dx >= (unsigned)S1 || (unsigned)dy >= (unsigned)S1 || (unsigned)dz >= (unsigned)S1)
    return -1;
  return dx + S1 * (dy + S1 * dz);
}

// Dirichlet components of a coarse row: identity on the diagonal (their rows
// and columns receive no contribution from the Galerkin products)
template <class T>
__global__ void k_mg_fix_masked(int nrow, int S, int R, const int* __restrict__ cmask, T* A) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nrow) return;
  int cm = cmask[a];
  if (!cm) return;
  int S1 = 2 * R + 1, center = R + S1 * (R + S1 * R);
  for (int c = 0; c < 3; ++c)
    if ((cm >> c) & 1) A[((size_t)a * S + center) * 9 + 4 * c] = (T)1;
}

// level 1: one warp per fine dof i; its block row, weighted by P_ia for every
// coarse row a it interpolates from, spread to the coarse columns of each
// column dof j.  The terms go to the zeroed fixed-point operator by integer
// atomics (resolved in L2; 32-bit for an FP32 operator, 64-bit for FP64); a
// warp per fine row keeps the work
// balanced when the coarse grid is much coarser than the finest leaves.  The
// bound: every entry sums terms P_ia |K_ij| P_jb with sum over j, b at most
// the l1 norm of row i (bnd, from the fine smoother kernel) and at most cnt
// fine rows i per coarse row a.
template <class T, class ACC>
__global__ void k_mg_rap1(int nd, int R, int S, const float* __restrict__ pw,
                          const int* __restrict__ pidx, const int* __restrict__ fmask,
                          const int* __restrict__ rp, const int* __restrict__ col, Sliced SK,
                          const T* __restrict__ K, const int* __restrict__ xyz,
                          ACC* A, const unsigned long long* __restrict__ bnd,
                          double cnt, int* err) {
  int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= nd) return;
  double sc = fixed_scale<ACC>(__longlong_as_double((long long)*bnd) * cnt);
  int mi = fmask[i];
  int s0 = rp[i], nb = rp[i + 1] - s0;
  int si = SK.pos[i], sl = si >> 5, W = SK.w[sl];
  long long b0 = SK.base[sl];
  for (int idx = lane; idx < nb; idx += 32) {
    int j = col[s0 + idx];
    int mj = fmask[j];
    long long slot = sliced_slot(b0, si, idx);
    T v[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      int ci = e / 3, ck = e - 3 * (e / 3);
      v[e] = (((mi >> ci) & 1) || ((mj >> ck) & 1)) ? (T)0 : K[sliced_entry(b0, W, slot, e)];
    }
    for (int qa = 0; qa < 8; ++qa) {
      int a = pidx[8 * (size_t)i + qa];
      if (a < 0) break;
      double wa = (double)pw[8 * (size_t)i + qa];
      int ca[3];
      unpack3(xyz[a], ca);
      ACC* row = A + (size_t)a * S * 9;
      for (int q = 0; q < 8; ++q) {
        int b = pidx[8 * (size_t)j + q];
        if (b < 0) break;
        double f = wa * (double)pw[8 * (size_t)j + q];
        int cb[3];
        unpack3(xyz[b], cb);
        int o = stencil_index(cb, ca, R);
        if (o < 0) {
          atomicOr(err, EB_ROW);
          continue;
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) fixed_add(row + 9 * o + e, f * (double)v[e], sc);
      }
    }
  }
}

// Level 1 in two gathers, in plain arithmetic and free of atomics, for the
// usual stencil radius R = 2 (the fine blocks reach one level-1 cell):
// (1) k_mg_kp, one warp per fine row i: (K P)_iJ = sum_j K_ij P_jJ for the
//     4 x 4 x 4 level-1 nodes J = c_i + (-1..2) around the level-1 cell c_i
//     of dof i (every P_jJ of a column j of the row lands there), the
//     columns j taken in row order, accumulated in shared memory and written
//     out as kp[i][9][64];
// (2) k_mg_ptkp, one warp per level-1 row a: A_ab = sum_i P_ia (K P)_ib over
//     the fine dofs i of the transpose of P, in dof order, lanes over the
//     125 stencil offsets b - a.
// Every sum runs in a fixed order, so the operator is the same bit for bit
// on every run, like the fixed-point product it replaces where it applies.
constexpr int KP_NS = 64;  // (2R)^3 level-1 nodes around a fine dof's cell, R = 2
// warps per block of k_mg_kp: its shared memory (44 KB FP32, 36 KB FP64)
// stays under the 48 KB of a static allocation
template <class T>
__host__ __device__ constexpr int kp_warps() {
  return sizeof(T) == 4 ? 8 : 4;
}

template <class T>
struct KpShared {
  static constexpr int NW = kp_warps<T>();
  T tab[NW][KP_NS * 9];     // (K P)_i, [slot][9]
  T sv[NW][32][9];          // a chunk of 32 blocks K_ij (masked)
  int ss[NW][32][8];        // their P_j entries: slot (-1: none) ...
  float sw[NW][32][8];      // ... and weight
};

template <class T>
__global__ void __launch_bounds__(32 * kp_warps<T>())
    k_mg_kp(int nd, int D, int d1, const int* __restrict__ dof_node, const uint64_t* __restrict__ nkey,
            const float* __restrict__ pw, const int* __restrict__ pidx, const int* __restrict__ fmask,
            const int* __restrict__ rp, const int* __restrict__ col, Sliced SK, const T* __restrict__ K,
            const int* __restrict__ xyz, T* kp, int* kpc, int* err) {
  __shared__ KpShared<T> sh;
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int i = blockIdx.x * kp_warps<T>() + wi;
  if (i >= nd) return;
  T* tab = sh.tab[wi];
  for (int f = lane; f < KP_NS * 9; f += 32) tab[f] = (T)0;
  int X[3], ci[3];
  demorton(nkey[dof_node[i]], X);
  int shf = D - d1, n = 1 << d1;
  for (int d = 0; d < 3; ++d) ci[d] = min(X[d] >> shf, n - 1);
  if (lane == 0) kpc[i] = pack3(ci[0], ci[1], ci[2]);
  int mi = fmask[i];
  int s0 = rp[i], nb = rp[i + 1] - s0;
  int si = SK.pos[i], sl = si >> 5, W = SK.w[sl];
  long long b0 = SK.base[sl];
  bool bad = false;
  for (int base = 0; base < nb; base += 32) {
    int idx = base + lane, cnt = min(32, nb - base);
    __syncwarp();
    if (idx < nb) {
      int j = col[s0 + idx];
      int mj = fmask[j];
      long long slot = sliced_slot(b0, si, idx);
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        int ca = e / 3, ck = e - 3 * (e / 3);
        sh.sv[wi][lane][e] = (((mi >> ca) & 1) || ((mj >> ck) & 1)) ? (T)0 : K[sliced_entry(b0, W, slot, e)];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int b = pidx[8 * (size_t)j + q];
        int s = -1;
        if (b >= 0) {
          int cb[3];
          unpack3(xyz[b], cb);
          int o0 = cb[0] - ci[0] + 1, o1 = cb[1] - ci[1] + 1, o2 = cb[2] - ci[2] + 1;
          if ((unsigned)o0 < 4u && (unsigned)o1 < 4u && (unsigned)o2 < 4u)
            s = o0 + 4 * (o1 + 4 * o2);
          else
            bad = true;
          sh.sw[wi][lane][q] = pw[8 * (size_t)j + q];
        }
        sh.ss[wi][lane][q] = s;
      }
    }
    __syncwarp();
    // column by column (a fixed order per accumulator): the 8 x 9 (entry,
    // component) terms of a column go to distinct accumulators
    for (int u = 0; u < cnt; ++u) {
      for (int t = lane; t < 72; t += 32) {
        int q = t / 9, e = t - 9 * (t / 9);
        int s = sh.ss[wi][u][q];
        if (s >= 0) tab[9 * s + e] += (T)sh.sw[wi][u][q] * sh.sv[wi][u][e];
      }
      __syncwarp();
    }
  }
  if (bad) atomicOr(err, EB_ROW);
  __syncwarp();
  T* out = kp + (size_t)i * 9 * KP_NS;
  for (int f = lane; f < KP_NS * 9; f += 32) {
    int e = f / KP_NS, s = f - KP_NS * (f / KP_NS);
    out[f] = tab[9 * s + e];
  }
}

template <class T>
__global__ void k_mg_ptkp(int nrow, const int* __restrict__ xyz, const int* __restrict__ tptr,
                          const int* __restrict__ tidx, const float* __restrict__ tw,
                          const int* __restrict__ kpc, const T* __restrict__ kp, T* A) {
  constexpr int R = 2, S1 = 2 * R + 1, S = S1 * S1 * S1, NPL = (S + 31) / 32;
  int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= nrow) return;
  int ca[3];
  unpack3(xyz[a], ca);
  T acc[NPL][9];
#pragma unroll
  for (int k = 0; k < NPL; ++k)
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[k][e] = (T)0;
  for (int t = tptr[a]; t < tptr[a + 1]; ++t) {
    int i = tidx[t];
    T w = (T)tw[t];
    int ci[3];
    unpack3(kpc[i], ci);
    const T* kv = kp + (size_t)i * 9 * KP_NS;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      int o = lane + 32 * k;
      if (o >= S) continue;
      // b = a + delta(o); its slot around the cell of i
      int s0 = ca[0] + o % S1 - R - ci[0] + 1;
      int s1 = ca[1] + (o / S1) % S1 - R - ci[1] + 1;
      int s2 = ca[2] + o / (S1 * S1) - R - ci[2] + 1;
      if ((unsigned)s0 >= 4u || (unsigned)s1 >= 4u || (unsigned)s2 >= 4u) continue;
      int s = s0 + 4 * (s1 + 4 * s2);
#pragma unroll
      for (int e = 0; e < 9; ++e) acc[k][e] += w * kv[e * KP_NS + s];
    }
  }
  T* row = A + (size_t)a * S * 9;
#pragma unroll
  for (int k = 0; k < NPL; ++k) {
    int o = lane + 32 * k;
    if (o >= S) continue;
#pragma unroll
    for (int e = 0; e < 9; ++e) row[9 * o + e] = acc[k][e];
  }
}

// uniform level -> next coarser: one warp per row i of the finer level; its
// operator row, weighted by the trilinear weights prod(1 - |delta|/2) of the
// coarse rows a around it, spread to the coarse columns of each column j, by
// fixed-point integer atomics as above (at most 27 finer rows per coarse row)
template <class T, class ACC>
__global__ void k_mg_rapu(int nrow_f, int Rc, int Sc, int n1c, const int* __restrict__ gid_c,
                          int Rf, int Sf, int n1f, const int* __restrict__ gid_f,
                          const int* __restrict__ xyz_f, const int* __restrict__ fmask,
                          const T* __restrict__ Af, ACC* A,
                          const unsigned long long* __restrict__ bnd, int* err) {
  int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= nrow_f) return;
  double sc = fixed_scale<ACC>(__longlong_as_double((long long)*bnd) * 27.0);
  int fi[3];
  unpack3(xyz_f[i], fi);
  int mi = fmask[i];
  int S1f = 2 * Rf + 1;
  int alo[3], ahi[3];
  for (int d = 0; d < 3; ++d) {
    alo[d] = fi[d] >> 1;
    ahi[d] = (fi[d] + 1) >> 1;
  }
  const T* frow = Af + (size_t)i * Sf * 9;
  for (int of = lane; of < Sf; of += 32) {
    int fj[3] = {fi[0] + of % S1f - Rf, fi[1] + (of / S1f) % S1f - Rf, fi[2] + of / (S1f * S1f) - Rf};
    if (fj[0] < 0 || fj[1] < 0 || fj[2] < 0 || fj[0] >= n1f || fj[1] >= n1f || fj[2] >= n1f) continue;
    int j = gid_f[fj[0] + n1f * (fj[1] + n1f * fj[2])];
    if (j < 0) continue;
    int mj = fmask[j];
    T v[9];
    bool any = false;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      int ci = e / 3, ck = e - 3 * (e / 3);
      v[e] = (((mi >> ci) & 1) || ((mj >> ck) & 1)) ? (T)0 : frow[9 * of + e];
      any = any || v[e] != (T)0;
    }
    if (!any) continue;
    int blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) {
      blo[d] = fj[d] >> 1;
      bhi[d] = (fj[d] + 1) >> 1;
    }
    for (int az = alo[2]; az <= ahi[2]; ++az)
      for (int ay = alo[1]; ay <= ahi[1]; ++ay)
        for (int ax = alo[0]; ax <= ahi[0]; ++ax) {
          int a = gid_c[ax + n1c * (ay + n1c * az)];
          if (a < 0) continue;
          double wa = 1.0;
          if (alo[0] != ahi[0]) wa *= 0.5;
          if (alo[1] != ahi[1]) wa *= 0.5;
          if (alo[2] != ahi[2]) wa *= 0.5;
          ACC* row = A + (size_t)a * Sc * 9;
          int ca[3] = {ax, ay, az};
          for (int z = blo[2]; z <= bhi[2]; ++z)
            for (int y = blo[1]; y <= bhi[1]; ++y)
              for (int x = blo[0]; x <= bhi[0]; ++x) {
                double f = wa;
                if (blo[0] != bhi[0]) f *= 0.5;
                if (blo[1] != bhi[1]) f *= 0.5;
                if (blo[2] != bhi[2]) f *= 0.5;
                int cb[3] = {x, y, z};
                int o = stencil_index(cb, ca, Rc);
                if (o < 0) {
                  atomicOr(err, EB_ROW);
                  continue;
                }
#pragma unroll
                for (int e = 0; e < 9; ++e) fixed_add(row + 9 * o + e, f * (double)v[e], sc);
              }
        }
  }
}

// ---------------------------------------------------------------- smoother inverses

// w times the inverse of D + diag(l1 sums of the off-diagonal blocks), 12 per row
template <class T>
__device__ inline void store_inv(const double* a, T* o, int* err, double w) {
  double c0 = a[4] * a[8] - a[5] * a[7], c1 = a[5] * a[6] - a[3] * a[8], c2 = a[3] * a[7] - a[4] * a[6];
  double det = a[0] * c0 + a[1] * c1 + a[2] * c2;
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    atomicOr(err, EB_KRYLOV);
    det = 1.0;
  }
  double id = w / det;
  o[0] = (T)(c0 * id);
  o[1] = (T)((a[2] * a[7] - a[1] * a[8]) * id);
  o[2] = (T)((a[1] * a[5] - a[2] * a[4]) * id);
  o[3] = (T)0;
  o[4] = (T)(c1 * id);
  o[5] = (T)((a[0] * a[8] - a[2] * a[6]) * id);
  o[6] = (T)((a[2] * a[3] - a[0] * a[5]) * id);
  o[7] = (T)0;
  o[8] = (T)(c2 * id);
  o[9] = (T)((a[1] * a[6] - a[0] * a[7]) * id);
  o[10] = (T)((a[0] * a[4] - a[1] * a[3]) * id);
  o[11] = (T)0;
}

// also the largest l1 norm of a row (all 9 entries of every block), the bound
// of the level-1 Galerkin product (a maximum of non-negative doubles, by the
// ordering of their bit patterns: the same whatever the order)
template <class T>
__global__ void k_mg_dinv_fine(int nd, int npad, Sliced SK, const T* __restrict__ K, T* Dinv, int* err,
                               double w, unsigned long long* bnd) {
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  if (sr >= npad) return;
  int r = SK.row[sr];
  T* o = Dinv + 12 * (size_t)r;
  if (r >= nd) {
    for (int e = 0; e < 12; ++e) o[e] = (T)0;
    return;
  }
  // the row in the access pattern of the SpMV: four slots per 16-byte load
  int sl = sr >> 5, ln = sr & 31, W = SK.w[sl];
  long long b0 = SK.base[sl];
  const T* Kb = K + 9 * b0;
  const int* cb = SK.scol + b0;
  size_t plane = (size_t)32 * W;
  // (the l1 sums, a smoother parameter, accumulate in the matrix precision)
  double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  T s[3] = {0, 0, 0};
  for (int k4 = 0; k4 < (W >> 2); ++k4) {
    size_t off = ((size_t)k4 * 32 + ln) * 4;
    int4 c = *reinterpret_cast<const int4*>(cb + off);
    int cc[4] = {c.x, c.y, c.z, c.w};
    T v[9][4];
#pragma unroll
    for (int e = 0; e < 9; ++e) ld4(Kb + e * plane + off, v[e]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (cc[j] == r) {
#pragma unroll
        for (int e = 0; e < 9; ++e) a[e] += (double)v[e][j];
      } else {
#pragma unroll
        for (int e = 0; e < 9; ++e) s[e / 3] += v[e][j] < (T)0 ? -v[e][j] : v[e][j];
      }
    }
  }
  double l1 = (double)s[0] + (double)s[1] + (double)s[2];
  for (int e = 0; e < 9; ++e) l1 += fabs(a[e]);
  atomicMax(bnd, (unsigned long long)__double_as_longlong(l1));
  for (int d = 0; d < 3; ++d) a[4 * d] += (double)s[d];
  store_inv<T>(a, o, err, w);
}

template <class T>
__global__ void k_mg_dinv(int nrow, int npad, int S, int R, const T* __restrict__ A, T* Dinv, int* err,
                          double w, unsigned long long* bnd) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= npad) return;
  T* o = Dinv + 12 * (size_t)r;
  if (r >= nrow) {
    for (int e = 0; e < 12; ++e) o[e] = (T)0;
    return;
  }
  int S1 = 2 * R + 1, center = R + S1 * (R + S1 * R);
  const T* row = A + (size_t)r * S * 9;
  double a[9], s[3] = {0, 0, 0};
  for (int e = 0; e < 9; ++e) a[e] = (double)row[9 * center + e];
  for (int oo = 0; oo < S; ++oo) {
    if (oo == center) continue;
    for (int e = 0; e < 9; ++e) s[e / 3] += fabs((double)row[9 * oo + e]);
  }
  double l1 = s[0] + s[1] + s[2];
  for (int e = 0; e < 9; ++e) l1 += fabs(a[e]);
  atomicMax(bnd, (unsigned long long)__double_as_longlong(l1));
  for (int d = 0; d < 3; ++d) a[4 * d] += s[d];
  store_inv<T>(a, o, err, w);
}

// dense inverse of the coarsest operator (one block; n3 = 3 nrow <= 81),
// Gauss-Jordan without pivoting on the symmetric positive semi-definite
// matrix, in FP64.  A pivot below 1e-12 of the largest diagonal entry marks a
// direction the coarse space does not resolve (interpolation columns that
// coincide on a thin active region): its row and column are dropped, which
// leaves the pseudo-inverse on the rest and keeps the V-cycle positive
// definite (the smoother part alone is).
template <class T>
__global__ void k_mg_dense(int nrow, int S, int R, const int* __restrict__ xyz, int n1,
                           const int* __restrict__ gid, const T* __restrict__ A, T* Cinv) {
  extern __shared__ double M[];  // [n3][2 n3]
  __shared__ double dmax;
  int n3 = 3 * nrow, w2 = 2 * n3;
  for (int u = threadIdx.x; u < n3 * w2; u += blockDim.x) M[u] = 0.0;
  __syncthreads();
  int S1 = 2 * R + 1;
  for (int u = threadIdx.x; u < nrow * S; u += blockDim.x) {
    int a = u / S, o = u - S * a;
    int ca[3];
    unpack3(xyz[a], ca);
    int cb[3] = {ca[0] + o % S1 - R, ca[1] + (o / S1) % S1 - R, ca[2] + o / (S1 * S1) - R};
    if (cb[0] < 0 || cb[1] < 0 || cb[2] < 0 || cb[0] >= n1 || cb[1] >= n1 || cb[2] >= n1) continue;
    int b = gid[cb[0] + n1 * (cb[1] + n1 * cb[2])];
    if (b < 0) continue;
    const T* blk = A + ((size_t)a * S + o) * 9;
    for (int e = 0; e < 9; ++e) M[(3 * a + e / 3) * w2 + 3 * b + e % 3] = (double)blk[e];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int i = 0; i < n3; ++i) d = fmax(d, M[i * w2 + i]);
    dmax = d;
  }
  for (int i = threadIdx.x; i < n3; i += blockDim.x) M[i * w2 + n3 + i] = 1.0;
  __syncthreads();
  double tiny = 1e-12 * dmax;
  for (int k = 0; k < n3; ++k) {
    double piv = M[k * w2 + k];
    __syncthreads();
    if (!(piv > tiny) || !isfinite(piv)) {
      // drop direction k: zero its row and column in both halves
      for (int j = threadIdx.x; j < w2; j += blockDim.x) M[k * w2 + j] = 0.0;
      for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        M[i * w2 + k] = 0.0;
        M[i * w2 + n3 + k] = 0.0;
      }
      __syncthreads();
      continue;
    }
    for (int j = threadIdx.x; j < w2; j += blockDim.x) M[k * w2 + j] /= piv;
    __syncthreads();
    for (int u = threadIdx.x; u < n3 * w2; u += blockDim.x) {
      int i = u / w2, j = u - w2 * i;
      if (i == k || j == k) continue;
      M[u] -= M[i * w2 + k] * M[k * w2 + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x)
      if (i != k) M[i * w2 + k] = 0.0;
    __syncthreads();
  }
  for (int u = threadIdx.x; u < n3 * n3; u += blockDim.x) {
    int i = u / n3, j = u - n3 * i;
    Cinv[u] = (T)M[i * w2 + n3 + j];
  }
}

// ---------------------------------------------------------------- FP16 smoothing copy

// largest |K| (as ordered bits of a non-negative float)
__global__ void k_absmax(long long n, const float* __restrict__ K, unsigned* out) {
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(K[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// FP16 copy of K scaled by 2^e (the largest |entry| maps below 2^14, clear of
// the FP16 limit 65504); scaling by a power of two keeps the copy exactly as
// symmetric as K.  kscale receives 2^-e.
__global__ void k_to_half(int nslice, Sliced SK, const float* __restrict__ K, const unsigned* amax,
                          __half* Kh, float* kscale) {
  float m = __uint_as_float(*amax);
  int e = 14 - (m > 0.f ? (int)ceilf(log2f(m)) : 0);
  float sc = ldexpf(1.f, e);
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *kscale = ldexpf(1.f, -e);
  // one warp per slice, a lane per row; the plane-pair layout of sliced_row_h
  int sl = (int)(t >> 5), ln = (int)(t & 31);
  if (sl >= nslice) return;
  int W = SK.w[sl];
  long long b0 = SK.base[sl];
  const float* Kb = K + 9 * b0;
  __half* Hb = Kh + 9 * b0;
  size_t plane = (size_t)32 * W;
  auto pack = [sc](float a, float b) {
    __half2 h = __floats2half2_rn(a * sc, b * sc);
    return *reinterpret_cast<unsigned*>(&h);
  };
  for (int k4 = 0; k4 < (W >> 2); ++k4) {
    size_t off = ((size_t)k4 * 32 + ln) * 4;
    float4 v[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] = *reinterpret_cast<const float4*>(Kb + q * plane + off);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 o = {pack(v[2 * q].x, v[2 * q].y), pack(v[2 * q].z, v[2 * q].w),
                 pack(v[2 * q + 1].x, v[2 * q + 1].y), pack(v[2 * q + 1].z, v[2 * q + 1].w)};
      *reinterpret_cast<uint4*>(Hb + 2 * q * plane + 2 * off) = o;
    }
    uint2 o8 = {pack(v[8].x, v[8].y), pack(v[8].z, v[8].w)};
    *reinterpret_cast<uint2*>(Hb + 8 * plane + off) = o8;
  }
}

// ---------------------------------------------------------------- V-cycle kernels

// x = Dinv b (rows padded to 4 components)
template <class T>
__global__ void k_mg_jac0(int n, const T* __restrict__ Dinv, const T* __restrict__ b, T* x,
                          const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T bv[4], xv[4];
  ld4(b + 4 * (size_t)i, bv);
  apply_dinv(Dinv, i, bv, xv);
  st4(x + 4 * (size_t)i, xv);
}

// fine level: MODE 0, out = b - K x with the Dirichlet components zeroed (the
// residual that k_mg_restrict1 gathers to level 1); MODE 1, out = x + Dinv
// (b - K x) with r.z += b.out by a fixed-order grid sum (rz non-null).
// Bounded to 2 resident blocks of 256 per SM: with the FP16 row product's two
// groups of loads in flight the kernel needs about 96 registers; at 4 blocks
// (64 registers) it spilled and ran 10 % slower (0.120 against 0.108 ms at
// 248 k rows)
template <class T, int MODE, class TK>
__global__ void __launch_bounds__(256, 2) k_mg_fine(int nd, int npad, Sliced SK, const TK* __restrict__ K, const float* kscale,
                          const T* __restrict__ b, const T* __restrict__ x, const T* __restrict__ Dinv,
                          T* out, const int* __restrict__ fmask, double* rz, const Scal* sk, int k,
                          GridRed gr) {
  if (skip(sk, k)) return;
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  double part = 0.0;
  if (sr < npad) {
    int r = SK.row[sr];
    T y[3];
    if constexpr (sizeof(TK) == 2) {
      float yf[3];
      sliced_row_h(sr, SK, (const __half*)K, (const float*)x, yf);
      float ks = *kscale;
      for (int c = 0; c < 3; ++c) y[c] = (T)(yf[c] * ks);
    } else {
      sliced_row<T, T, T, 4>(sr, SK, (const T*)K, x, y);
    }
    T bv[4], res[4];
    ld4(b + 4 * (size_t)r, bv);
    for (int c = 0; c < 3; ++c) res[c] = r < nd ? bv[c] - y[c] : (T)0;
    res[3] = (T)0;
    if (MODE == 0) {
      int mi = r < nd ? fmask[r] : 7;
      for (int c = 0; c < 3; ++c)
        if ((mi >> c) & 1) res[c] = (T)0;
      st4(out + 4 * (size_t)r, res);
    } else {
      T xv[4], d[4];
      ld4(x + 4 * (size_t)r, xv);
      apply_dinv(Dinv, r, res, d);
      for (int c = 0; c < 3; ++c) xv[c] = r < nd ? xv[c] + d[c] : (T)0;
      xv[3] = (T)0;
      st4(out + 4 * (size_t)r, xv);
      for (int c = 0; c < 3; ++c) part += (double)bv[c] * (double)xv[c];
    }
  }
  if (MODE == 1 && rz) grid_sum1(part, rz, gr);  // rz is the same for every block
}

// level-1 right-hand side b = P^T r (r: the fine residual of k_mg_fine MODE 0,
// gathered through the transpose of P in the fixed order of its entries) and
// the pre-smoothing x = Dinv b; one warp per level-1 row, padding rows zero
template <class T>
__global__ void k_mg_restrict1(int nrow, int npad, const int* __restrict__ tptr,
                               const int* __restrict__ tidx, const float* __restrict__ tw,
                               const T* __restrict__ r, const T* __restrict__ Dinv, T* b, T* x,
                               const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= npad) return;
  T s0 = (T)0, s1 = (T)0, s2 = (T)0;
  if (a < nrow) {
    int e1 = tptr[a + 1];
    for (int e = tptr[a] + lane; e < e1; e += 32) {
      T w = (T)tw[e];
      T v[4];
      ld4(r + 4 * (size_t)tidx[e], v);
      s0 += w * v[0];
      s1 += w * v[1];
      s2 += w * v[2];
    }
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    T bv[4] = {s0, s1, s2, (T)0}, xv[4];
    st4(b + 4 * (size_t)a, bv);
    apply_dinv(Dinv, a, bv, xv);  // padding rows of Dinv are zero
    st4(x + 4 * (size_t)a, xv);
  }
}

// uniform level -> next coarser right-hand side: coarse node a gathers the
// residual rf of the 27 finer nodes 2a + delta (delta in {-1, 0, 1}^3) with
// the weights prod(1 - |delta|/2), then x = Dinv b; one thread per row, its
// 27 grid lookups issued before its 27 loads (two round trips, not 27)
template <class T>
__global__ void k_mg_restrictu(int nrow, int npad, const int* __restrict__ xyz, int n1f,
                               const int* __restrict__ gid_f, const T* __restrict__ rf,
                               const T* __restrict__ Dinv, T* b, T* x, const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= npad) return;
  T s[3] = {(T)0, (T)0, (T)0};
  if (a < nrow) {
    int ca[3];
    unpack3(xyz[a], ca);
    int jq[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      int fx = 2 * ca[0] + q % 3 - 1, fy = 2 * ca[1] + (q / 3) % 3 - 1, fz = 2 * ca[2] + q / 9 - 1;
      bool in = fx >= 0 && fy >= 0 && fz >= 0 && fx < n1f && fy < n1f && fz < n1f;
      jq[q] = in ? gid_f[fx + n1f * (fy + n1f * fz)] : -1;
    }
    // z, then y, then x offsets, in that order
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      if (jq[q] < 0) continue;
      int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
      T f = (T)((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
      T v[4];
      ld4(rf + 4 * (size_t)jq[q], v);
      for (int c = 0; c < 3; ++c) s[c] += f * v[c];
    }
  }
  T bv[4] = {s[0], s[1], s[2], (T)0}, xv[4];
  st4(b + 4 * (size_t)a, bv);
  apply_dinv(Dinv, a, bv, xv);
  st4(x + 4 * (size_t)a, xv);
}

// uniform level (warp per row): MODE 0, out = b - A x with the Dirichlet
// components zeroed (gathered by k_mg_restrictu of the next coarser level);
// MODE 1, out = x + Dinv (b - A x)
template <class T, int MODE>
__global__ void k_mg_lvl(int nrow, int S, int R, int n1, const int* __restrict__ xyz,
                         const int* __restrict__ gid, const T* __restrict__ A, const T* __restrict__ b,
                         const T* __restrict__ x, const T* __restrict__ Dinv, T* out,
                         const int* __restrict__ mask, const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= nrow) return;
  int ca[3];
  unpack3(xyz[a], ca);
  int S1 = 2 * R + 1;
  const T* row = A + (size_t)a * S * 9;
  T y0 = 0, y1 = 0, y2 = 0;
  // four stencil trips of the warp per round: their grid lookups, then their
  // x loads, go out together (two dependent round trips per round, not eight)
  for (int o0 = 0; o0 < S; o0 += 128) {
    int j[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int o = o0 + 32 * u + lane;
      j[u] = -1;
      if (o < S) {
        int cb[3] = {ca[0] + o % S1 - R, ca[1] + (o / S1) % S1 - R, ca[2] + o / (S1 * S1) - R};
        if (cb[0] >= 0 && cb[1] >= 0 && cb[2] >= 0 && cb[0] < n1 && cb[1] < n1 && cb[2] < n1)
          j[u] = gid[cb[0] + n1 * (cb[1] + n1 * cb[2])];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (j[u] < 0) continue;
      T xv[4];
      ld4(x + 4 * (size_t)j[u], xv);
      const T* v = row + 9 * (o0 + 32 * u + lane);
      y0 += v[0] * xv[0] + v[1] * xv[1] + v[2] * xv[2];
      y1 += v[3] * xv[0] + v[4] * xv[1] + v[5] * xv[2];
      y2 += v[6] * xv[0] + v[7] * xv[1] + v[8] * xv[2];
    }
  }
  y0 = warp_sum(y0);
  y1 = warp_sum(y1);
  y2 = warp_sum(y2);
  if (lane == 0) {
    T bv[4], res[4];
    ld4(b + 4 * (size_t)a, bv);
    res[0] = bv[0] - y0;
    res[1] = bv[1] - y1;
    res[2] = bv[2] - y2;
    res[3] = (T)0;
    if (MODE == 0) {
      int mi = mask[a];
      for (int c = 0; c < 3; ++c)
        if ((mi >> c) & 1) res[c] = (T)0;
      st4(out + 4 * (size_t)a, res);
    } else {
      T xv[4], d[4];
      ld4(x + 4 * (size_t)a, xv);
      apply_dinv(Dinv, a, res, d);
      for (int c = 0; c < 3; ++c) xv[c] += d[c];
      xv[3] = (T)0;
      st4(out + 4 * (size_t)a, xv);
    }
  }
}

// xf += P x1 (level 1 -> fine)
template <class T>
__global__ void k_mg_prolong1(int nd, const int* __restrict__ pidx, const float* __restrict__ pw,
                              const int* __restrict__ fmask, const T* __restrict__ x1, T* xf,
                              const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  T s[3] = {0, 0, 0};
  // the row's 8 weights in two 16-byte loads each, then all coarse loads
  int4 ia = *reinterpret_cast<const int4*>(pidx + 8 * (size_t)i);
  int4 ib = *reinterpret_cast<const int4*>(pidx + 8 * (size_t)i + 4);
  float4 wa = *reinterpret_cast<const float4*>(pw + 8 * (size_t)i);
  float4 wb = *reinterpret_cast<const float4*>(pw + 8 * (size_t)i + 4);
  int av[8] = {ia.x, ia.y, ia.z, ia.w, ib.x, ib.y, ib.z, ib.w};
  float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
  bool live = true;  // entries end at the first negative index
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    live = live && av[q] >= 0;
    if (!live) continue;
    T xv[4];
    ld4(x1 + 4 * (size_t)av[q], xv);
    for (int c = 0; c < 3; ++c) s[c] += (T)wv[q] * xv[c];
  }
  int mi = fmask[i];
  T xv[4];
  ld4(xf + 4 * (size_t)i, xv);
  for (int c = 0; c < 3; ++c)
    if (!((mi >> c) & 1)) xv[c] += s[c];
  st4(xf + 4 * (size_t)i, xv);
}

// xf += P xc between uniform levels
template <class T>
__global__ void k_mg_prolong_u(int nrow, const int* __restrict__ xyz_f, const int* __restrict__ fmask,
                               int n1c, const int* __restrict__ gid_c, const T* __restrict__ xc, T* xf,
                               const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrow) return;
  int c[3];
  unpack3(xyz_f[i], c);
  int lo[3], hi[3];
  T f = (T)1;
  for (int d = 0; d < 3; ++d) {
    lo[d] = c[d] >> 1;
    hi[d] = (c[d] + 1) >> 1;
    if (lo[d] != hi[d]) f *= (T)0.5;
  }
  T s[3] = {0, 0, 0};
  // the (up to) 8 coarse corners in z, y, x order: lookups first, then loads
  int bq[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int x = lo[0] + (q & 1), y = lo[1] + ((q >> 1) & 1), z = lo[2] + (q >> 2);
    bq[q] = (x <= hi[0] && y <= hi[1] && z <= hi[2]) ? gid_c[x + n1c * (y + n1c * z)] : -1;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (bq[q] < 0) continue;
    T xv[4];
    ld4(xc + 4 * (size_t)bq[q], xv);
    for (int cc = 0; cc < 3; ++cc) s[cc] += f * xv[cc];
  }
  int mi = fmask[i];
  T xv[4];
  ld4(xf + 4 * (size_t)i, xv);
  for (int cc = 0; cc < 3; ++cc)
    if (!((mi >> cc) & 1)) xv[cc] += s[cc];
  st4(xf + 4 * (size_t)i, xv);
}

// coarsest: x = Cinv b (one block, a warp per output entry, the lanes over
// the columns, combined by a fixed shuffle tree)
template <class T>
__global__ void k_mg_coarse(int nrow, const T* __restrict__ Cinv, const T* __restrict__ b, T* x,
                            const Scal* sk, int k) {
  if (skip(sk, k)) return;
  int n3 = 3 * nrow;
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = wi; i < 4 * nrow; i += nw) {
    int a = i >> 2, c = i & 3;
    T s = (T)0;
    if (c < 3) {
      const T* row = Cinv + (size_t)(3 * a + c) * n3;
      for (int j = lane; j < nrow; j += 32)
        s += row[3 * j] * b[4 * j] + row[3 * j + 1] * b[4 * j + 1] + row[3 * j + 2] * b[4 * j + 2];
    }
    s = warp_sum(s);
    if (lane == 0) x[i] = s;
  }
}

// ---------------------------------------------------------------- host side

int pad32(int n) { return (n + 31) & ~31; }

// structure for the current mesh build (once per build)
void mg_structure(mpm_ctx* c, mpm_mesh* m) {
  cudaStream_t st = c->stream;
  if (!m->mg) m->mg = new MGData();
  MGData& G = *m->mg;
  const Geo& g = m->g;
  int nd = m->ndof;
  int d1 = std::min(std::min(m->dom.depth_min, g.D - 1), 7);
  // the first coarse grid should hold at most a quarter of the fine unknowns
  while (d1 > 1 && (double)(1 << d1) * (1 << d1) * (1 << d1) > 0.25 * nd) --d1;
  if (d1 < 1) throw CudaError(MPM_ERR_ARG, "multigrid needs an octree of depth 2 or more");
  G.nlev = d1;  // depths d1, d1-1, ..., 1
  // level 1 from the fine dofs
  for (int l = 0; l < G.nlev; ++l) {
    MGLevel& L = G.lev[l];
    L.d = d1 - l;
    L.n1 = (1 << L.d) + 1;
    int ng = L.n1 * L.n1 * L.n1;
    int* active = grow<int>(c, c->tmp[1], ng);
    int* freeb = grow<int>(c, c->tmp[2], ng);
    int* scan = grow<int>(c, c->tmp[3], ng);
    MPM_CUDA(cudaMemsetAsync(active, 0, sizeof(int) * ng, st));
    MPM_CUDA(cudaMemsetAsync(freeb, 0, sizeof(int) * ng, st));
    if (l == 0) {
      int* pidx = grow<int>(c, G.p_idx, 8 * (size_t)nd);
      float* pw = grow<float>(c, G.p_w, 8 * (size_t)nd);
      MPM_LAUNCH(k_mg_p1<<<grid_for(nd, 256), 256, 0, st>>>(nd, g.D, L.d, ptr<int>(m->dof_node),
                                                            ptr<uint64_t>(m->node_key), ptr<int>(m->dof_mask),
                                                            pidx, pw, active, freeb));
    } else {
      MGLevel& F = G.lev[l - 1];
      MPM_LAUNCH(k_mg_mark_u<<<grid_for(F.nrow, 256), 256, 0, st>>>(F.nrow, ptr<int>(F.xyz), ptr<int>(F.mask),
                                                                    L.n1, active, freeb));
    }
    cub_exclusive_sum_int(c, active, scan, ng);
    int last[2];
    MPM_CUDA(cudaMemcpyAsync(&c->h_int[2], scan + ng - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaMemcpyAsync(&c->h_int[3], active + ng - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    last[0] = c->h_int[2];
    last[1] = c->h_int[3];
    L.nrow = last[0] + last[1];
    L.npad = pad32(std::max(L.nrow, 1));
    int* gid = grow<int>(c, L.gid, ng);
    grow<int>(c, L.xyz, L.npad);
    grow<int>(c, L.mask, L.npad);
    MPM_LAUNCH(k_mg_compact<<<grid_for(ng, 256), 256, 0, st>>>(ng, L.n1, active, scan, freeb, gid,
                                                              ptr<int>(L.xyz), ptr<int>(L.mask)));
    if (l == 0) {
      MPM_LAUNCH(k_mg_p1_rows<<<grid_for(8LL * nd, 256), 256, 0, st>>>(nd, gid, ptr<int>(G.p_idx)));
      // stencil radius of level 1 from the reach of the fine blocks
      int* reach = (int*)(c->d_red + 8);
      MPM_CUDA(cudaMemsetAsync(reach, 0, sizeof(int), st));
      MPM_LAUNCH(k_mg_reach<<<grid_for(nd, 8), 256, 0, st>>>(nd, g.D, L.d, ptr<int>(m->row_ptr), ptr<int>(m->col),
                                                             ptr<int>(m->dof_node), ptr<uint64_t>(m->node_key), reach));
      MPM_CUDA(cudaMemcpyAsync(&c->h_int[2], reach, sizeof(int), cudaMemcpyDeviceToHost, st));
      MPM_CUDA(cudaStreamSynchronize(st));
      L.R = std::max(2, c->h_int[2] + 1);
      // the transpose of P, for the gathered restriction: keys sorted by
      // (level-1 row, fine dof, entry)
      long long n8 = 8LL * nd;
      uint64_t* keys = grow<uint64_t>(c, c->tmp[4], n8);
      uint64_t* alt = grow<uint64_t>(c, c->tmp[5], n8);
      MPM_LAUNCH(k_mg_tkeys<<<grid_for(n8, 256), 256, 0, st>>>(nd, ptr<int>(G.p_idx), keys));
      cub_sort_u64(c, keys, alt, (int)n8, 64);
      int* tptr = grow<int>(c, G.t_ptr, L.nrow + 1);
      int* tmax = (int*)(c->d_red + 8);
      MPM_CUDA(cudaMemsetAsync(tmax, 0, sizeof(int), st));
      MPM_LAUNCH(k_mg_tptr<<<grid_for(L.nrow + 1, 256), 256, 0, st>>>(L.nrow, n8, keys, tptr, tmax));
      MPM_LAUNCH(k_mg_tent<<<grid_for(n8, 256), 256, 0, st>>>(n8, keys, ptr<float>(G.p_w),
                                                             grow<int>(c, G.t_idx, n8),
                                                             grow<float>(c, G.t_w, n8)));
      MPM_CUDA(cudaMemcpyAsync(&c->h_int[2], tmax, sizeof(int), cudaMemcpyDeviceToHost, st));
      MPM_CUDA(cudaStreamSynchronize(st));
      G.t_max = c->h_int[2];
    } else {
      L.R = std::max(2, (G.lev[l - 1].R + 2) / 2);
    }
    int S1 = 2 * L.R + 1;
    L.S = S1 * S1 * S1;
  }
  MGLevel& C = G.lev[G.nlev - 1];
  G.n3c = 3 * C.nrow;
  if (G.n3c > 81) throw CudaError(MPM_ERR_ARG, "multigrid: coarsest level too large");
  int e = check_device_error(c, "multigrid structure");
  if (e) throw CudaError(e, c->err);
  G.gen = m->gen;
  G.prec = -1;
  G.num_gen = -1;
}

// Smoother weight.  The l1 block-Jacobi M bounds the stiffness, K <= M in
// the SPD ordering (each off-diagonal coupling x_i' K_ij x_j is at most half
// of |K_ij| (x_i^2 + x_j^2), which the l1 sums put on the diagonal), so the
// spectrum of M^-1 K lies in (0, 1].  The step x += w M^-1 (b - K x) then
// converges for every w in (0, 2), and the V(1,1) cycle stays symmetric
// positive definite because 2 M / w - K is.  The bound is loose for these
// meshes (27 to 125 coupled nodes per row; the largest eigenvalue of M^-1 K
// is near 0.8), so w = 1 under-relaxes: over [0.1, 0.8] the smoothing factor
// max |1 - w lambda| falls from 0.9 to 0.81 at w = 1.9, and far more in the
// middle of that range.  Measured: a quarter fewer PCG iterations on the
// indentation workload.  2 / w leaves 5 % of margin for the FP16 rounding of
// the fine-level copy of K.
constexpr double kSmoothW = 1.9;

template <class T>
void mg_numeric(mpm_ctx* c, mpm_mesh* m, const T* K, bool coarse) {
  cudaStream_t st = c->stream;
  MGData& G = *m->mg;
  int nd = m->ndof, npad = 32 * m->nslice;
  Sliced SK = sliced_view(m);
  // fine smoother and V-cycle vectors; bnd[l]: largest row l1 norm of the
  // level-l operator (l = 0 the fine matrix), the Galerkin products' bounds
  unsigned long long* bnd = grow<unsigned long long>(c, G.bound, 16);
  MPM_CUDA(cudaMemsetAsync(bnd, 0, 16 * sizeof(unsigned long long), st));
  T* fD = grow<T>(c, G.fDinv, 12 * (size_t)npad);
  MPM_LAUNCH_P(MPM_PROF_MG_SETUP, k_mg_dinv_fine<T><<<grid_for(npad, 256), 256, 0, st>>>(nd, npad, SK, K, fD, c->d_err, kSmoothW, bnd));
  grow<T>(c, G.fr, 4 * (size_t)npad);
  grow<T>(c, G.fx, 4 * (size_t)npad);
  if constexpr (sizeof(T) == 4) {
    // FP16 copy of the fine matrix for the V-cycle's two fine-level products
    long long n9 = 9LL * m->nslot;
    unsigned* amax = (unsigned*)(c->d_red + 10);
    float* ksc = (float*)(c->d_red + 11);
    MPM_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned), st));
    MPM_LAUNCH_P(MPM_PROF_MG_SETUP, k_absmax<<<4 * 152, 256, 0, st>>>(n9, K, amax));
    MPM_LAUNCH_P(MPM_PROF_MG_SETUP, k_to_half<<<grid_for(32LL * m->nslice, 256), 256, 0, st>>>(m->nslice, SK, K, amax, grow<__half>(c, G.fKh, n9), ksc));
  }
  if (!coarse) return;
  for (int l = 0; l < G.nlev; ++l) {
    MGLevel& L = G.lev[l];
    size_t nA = (size_t)L.nrow * L.S * 9;
    T* A = grow<T>(c, L.A, nA);
    // 64-bit integer accumulator (a 32-bit one, tried for the FP32 operator,
    // was no faster and, scaled by the row bound, too coarse for the cone's
    // level 1: twice the BiCGStab iterations)
    typedef unsigned long long ACC;
    if (l == 0 && L.R == 2) {
      // the two gathers (no accumulator, no atomics)
      T* kp = grow<T>(c, G.kp, (size_t)nd * 9 * KP_NS);
      int* kpc = grow<int>(c, G.kpc, nd);
      constexpr int NW = kp_warps<T>();
      MPM_LAUNCH_P(MPM_PROF_MG_RAP, k_mg_kp<T><<<(nd + NW - 1) / NW, 32 * NW, 0, st>>>(
          nd, m->g.D, L.d, ptr<int>(m->dof_node), ptr<uint64_t>(m->node_key), ptr<float>(G.p_w),
          ptr<int>(G.p_idx), ptr<int>(m->dof_mask), ptr<int>(m->row_ptr), ptr<int>(m->col), SK, K,
          ptr<int>(L.xyz), kp, kpc, c->d_err));
      MPM_LAUNCH_P(MPM_PROF_MG_RAP, k_mg_ptkp<T><<<grid_for(L.nrow, 8), 256, 0, st>>>(
          L.nrow, ptr<int>(L.xyz), ptr<int>(G.t_ptr), ptr<int>(G.t_idx), ptr<float>(G.t_w), kpc, kp, A));
    } else {
    ACC* acc = grow<ACC>(c, G.acc, nA);
    MPM_CUDA(cudaMemsetAsync(acc, 0, sizeof(ACC) * nA, st));
    double cnt;
    if (l == 0) {
      cnt = (double)std::max(G.t_max, 1);
      MPM_LAUNCH_P(MPM_PROF_MG_RAP, (k_mg_rap1<T, ACC><<<grid_for(nd, 8), 256, 0, st>>>(
          nd, L.R, L.S, ptr<float>(G.p_w), ptr<int>(G.p_idx), ptr<int>(m->dof_mask), ptr<int>(m->row_ptr),
          ptr<int>(m->col), SK, K, ptr<int>(L.xyz), acc, bnd, cnt, c->d_err)));
    } else {
      MGLevel& F = G.lev[l - 1];
      cnt = 27.0;
      MPM_LAUNCH_P(MPM_PROF_MG_RAP, (k_mg_rapu<T, ACC><<<grid_for(F.nrow, 8), 256, 0, st>>>(
          F.nrow, L.R, L.S, L.n1, ptr<int>(L.gid), F.R, F.S, F.n1, ptr<int>(F.gid), ptr<int>(F.xyz),
          ptr<int>(F.mask), ptr<T>(F.A), acc, bnd + l, c->d_err)));
    }
    MPM_LAUNCH_P(MPM_PROF_MG_RAP, (k_mg_from_fixed<T, ACC><<<4 * 152, 256, 0, st>>>((long long)nA, acc, bnd + l, cnt, A)));
    }
    MPM_LAUNCH_P(MPM_PROF_MG_SETUP, k_mg_fix_masked<T><<<grid_for(L.nrow, 128), 128, 0, st>>>(L.nrow, L.S, L.R, ptr<int>(L.mask), A));
    MPM_LAUNCH_P(MPM_PROF_MG_SETUP, k_mg_dinv<T><<<grid_for(L.npad, 128), 128, 0, st>>>(L.nrow, L.npad, L.S, L.R, A,
                                                                   grow<T>(c, L.Dinv, 12 * (size_t)L.npad), c->d_err, kSmoothW,
                                                                   bnd + l + 1));
    // level vectors: padding rows stay zero
    MPM_CUDA(cudaMemsetAsync(grow<T>(c, L.b, 4 * (size_t)L.npad), 0, sizeof(T) * 4 * L.npad, st));
    MPM_CUDA(cudaMemsetAsync(grow<T>(c, L.x, 4 * (size_t)L.npad), 0, sizeof(T) * 4 * L.npad, st));
    MPM_CUDA(cudaMemsetAsync(grow<T>(c, L.r, 4 * (size_t)L.npad), 0, sizeof(T) * 4 * L.npad, st));
  }
  MGLevel& C = G.lev[G.nlev - 1];
  int n3 = G.n3c;
  T* Ci = grow<T>(c, G.cinv, (size_t)std::max(n3 * n3, 1));
  size_t dsm = sizeof(double) * (size_t)n3 * 2 * n3;
  MPM_CUDA(cudaFuncSetAttribute(k_mg_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
  MPM_LAUNCH_P(MPM_PROF_MG_SETUP, k_mg_dense<T><<<1, 256, dsm, st>>>(C.nrow, C.S, C.R, ptr<int>(C.xyz), C.n1, ptr<int>(C.gid),
                                                ptr<T>(C.A), Ci));
  G.prec = sizeof(T) == 4 ? MPM_MIXED : MPM_FP64;
  G.num_gen = m->gen;
}

}  // namespace

template <class T>
void mg_setup(mpm_ctx* c, mpm_mesh* m, const T* K, bool reuse) {
  if (!m->mg || m->mg->gen != m->gen) mg_structure(c, m);
  MGData& G = *m->mg;
  int prec = sizeof(T) == 4 ? MPM_MIXED : MPM_FP64;
  bool keep = reuse && G.num_gen == m->gen && G.prec == prec;
  mg_numeric<T>(c, m, K, !keep);
}

namespace {

// the launches of one V-cycle on the context stream
template <class T>
void vcycle_launch(mpm_ctx* c, const mpm_mesh* mc, const T* K, const T* r, T* z, const Scal* sk, int k,
                   double* rz) {
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  cudaStream_t st = c->stream;
  MGData& G = *m->mg;
  int nd = m->ndof, npad = 32 * m->nslice;
  Sliced SK = sliced_view(m);
  const int* fmask = ptr<int>(m->dof_mask);
  T* fx = ptr<T>(G.fx);
  const T* fD = ptr<T>(G.fDinv);
  const int FB = 8 * 32;  // rows per block of the fine row kernels
  GridRed gr = grid_red(c, 1, grid_for(npad, FB));
  // fine pre-smoothing from zero, residual, restriction (gathered)
  MGLevel& L0 = G.lev[0];
  T* fr = ptr<T>(G.fr);
  MPM_LAUNCH_P(MPM_PROF_MG, k_mg_jac0<T><<<grid_for(npad, 256), 256, 0, st>>>(npad, fD, r, fx, sk, k));
  const float* ksc = (const float*)(c->d_red + 11);
  if constexpr (sizeof(T) == 4)
    MPM_LAUNCH_P(MPM_PROF_MG_FINE, k_mg_fine<T, 0, __half><<<grid_for(npad, FB), FB, 0, st>>>(
        nd, npad, SK, ptr<__half>(G.fKh), ksc, r, fx, fD, fr, fmask, nullptr, sk, k, gr));
  else
    MPM_LAUNCH_P(MPM_PROF_MG_FINE, k_mg_fine<T, 0, T><<<grid_for(npad, FB), FB, 0, st>>>(
        nd, npad, SK, K, ksc, r, fx, fD, fr, fmask, nullptr, sk, k, gr));
  MPM_LAUNCH_P(MPM_PROF_MG, k_mg_restrict1<T><<<grid_for(L0.npad, MGW), 32 * MGW, 0, st>>>(
      L0.nrow, L0.npad, ptr<int>(G.t_ptr), ptr<int>(G.t_idx), ptr<float>(G.t_w), fr, ptr<T>(L0.Dinv),
      ptr<T>(L0.b), ptr<T>(L0.x), sk, k));
  // down the uniform levels: residual, then the next level's gathered
  // right-hand side and pre-smoothing
  T* xcur[8];
  for (int l = 0; l + 1 < G.nlev; ++l) {
    MGLevel& L = G.lev[l];
    MGLevel& N = G.lev[l + 1];
    MPM_LAUNCH_P(l == 0 ? MPM_PROF_MG_LEVEL1 : MPM_PROF_MG, k_mg_lvl<T, 0><<<grid_for(L.nrow, MGW), 32 * MGW, 0, st>>>(
        L.nrow, L.S, L.R, L.n1, ptr<int>(L.xyz), ptr<int>(L.gid), ptr<T>(L.A), ptr<T>(L.b), ptr<T>(L.x),
        ptr<T>(L.Dinv), ptr<T>(L.r), ptr<int>(L.mask), sk, k));
    MPM_LAUNCH_P(MPM_PROF_MG, k_mg_restrictu<T><<<grid_for(N.npad, 128), 128, 0, st>>>(
        N.nrow, N.npad, ptr<int>(N.xyz), L.n1, ptr<int>(L.gid), ptr<T>(L.r), ptr<T>(N.Dinv), ptr<T>(N.b),
        ptr<T>(N.x), sk, k));
  }
  MGLevel& C = G.lev[G.nlev - 1];
  MPM_LAUNCH_P(MPM_PROF_MG, k_mg_coarse<T><<<1, 1024, 0, st>>>(C.nrow, ptr<T>(G.cinv), ptr<T>(C.b), ptr<T>(C.x), sk, k));
  xcur[G.nlev - 1] = ptr<T>(C.x);
  // up: prolongate, post-smooth (into the r buffer, which becomes the iterate)
  for (int l = G.nlev - 2; l >= 0; --l) {
    MGLevel& L = G.lev[l];
    MGLevel& N = G.lev[l + 1];
    MPM_LAUNCH_P(MPM_PROF_MG, k_mg_prolong_u<T><<<grid_for(L.nrow, 128), 128, 0, st>>>(
        L.nrow, ptr<int>(L.xyz), ptr<int>(L.mask), N.n1, ptr<int>(N.gid), xcur[l + 1], ptr<T>(L.x), sk, k));
    MPM_LAUNCH_P(l == 0 ? MPM_PROF_MG_LEVEL1 : MPM_PROF_MG, k_mg_lvl<T, 1><<<grid_for(L.nrow, MGW), 32 * MGW, 0, st>>>(
        L.nrow, L.S, L.R, L.n1, ptr<int>(L.xyz), ptr<int>(L.gid), ptr<T>(L.A), ptr<T>(L.b), ptr<T>(L.x),
        ptr<T>(L.Dinv), ptr<T>(L.r), nullptr, sk, k));
    xcur[l] = ptr<T>(L.r);
  }
  MPM_LAUNCH_P(MPM_PROF_MG, k_mg_prolong1<T><<<grid_for(nd, 128), 128, 0, st>>>(nd, ptr<int>(G.p_idx), ptr<float>(G.p_w), fmask,
                                                                  xcur[0], fx, sk, k));
  if constexpr (sizeof(T) == 4)
    MPM_LAUNCH_P(MPM_PROF_MG_FINE, k_mg_fine<T, 1, __half><<<grid_for(npad, FB), FB, 0, st>>>(
        nd, npad, SK, ptr<__half>(G.fKh), ksc, r, fx, fD, z, nullptr, rz, sk, k, gr));
  else
    MPM_LAUNCH_P(MPM_PROF_MG_FINE, k_mg_fine<T, 1, T><<<grid_for(npad, FB), FB, 0, st>>>(
        nd, npad, SK, K, ksc, r, fx, fD, z, nullptr, rz, sk, k, gr));
}

// everything the launches of a V-cycle take that can change between calls:
// the graph of a V-cycle is replayed only while these stay the same
template <class T>
uint64_t vcycle_key(mpm_ctx* c, const mpm_mesh* m, const T* K, const T* r, const T* z, const Scal* sk,
                    int kk, double* rz) {
  const MGData& G = *m->mg;
  uint64_t h = 1469598103934665603ULL;
  auto mix = [&](uint64_t v) {
    h ^= v;
    h *= 1099511628211ULL;
  };
  mix((uint64_t)m->gen);
  mix((uint64_t)(int64_t)kk);
  mix(sizeof(T));
  mix((uint64_t)(uintptr_t)K);
  mix((uint64_t)(uintptr_t)r);
  mix((uint64_t)(uintptr_t)z);
  mix((uint64_t)(uintptr_t)sk);
  mix((uint64_t)(uintptr_t)rz);
  mix((uint64_t)(uintptr_t)c->part.p);
  mix((uint64_t)(uintptr_t)c->d_ticket);
  mix((uint64_t)(uintptr_t)c->d_red);
  const Buf* bs[] = {&G.fx, &G.fDinv, &G.fr, &G.fKh, &G.t_ptr, &G.t_idx, &G.t_w, &G.p_idx, &G.p_w, &G.cinv};
  for (const Buf* b : bs) mix((uint64_t)(uintptr_t)b->p);
  mix((uint64_t)G.nlev);
  for (int l = 0; l < G.nlev; ++l) {
    const MGLevel& L = G.lev[l];
    const Buf* lb[] = {&L.A, &L.Dinv, &L.b, &L.x, &L.r, &L.gid, &L.xyz, &L.mask};
    for (const Buf* b : lb) mix((uint64_t)(uintptr_t)b->p);
    mix(((uint64_t)L.nrow << 32) | (uint64_t)(unsigned)L.S);
  }
  return h;
}

}  // namespace

// z = B r, one V-cycle.  Without per-launch timing, the V-cycle's launches
// are captured once into a CUDA graph on a private stream and replayed on the
// context stream: its many small coarse-level kernels then cost one launch.
// The graphs are cached by their key (every pointer and size the launches
// take, and k % 3, which is all the kernels read of k); the least recently
// used one is replaced.  A capture that fails falls back to plain launches.
template <class T>
void mg_apply(mpm_ctx* c, const mpm_mesh* mc, const T* K, const T* r, T* z, const Scal* sk, int k,
              double* rz) {
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  MGData& G = *m->mg;
  if (c->prof_on || !c->cap_stream || G.graphs_off) {
    vcycle_launch<T>(c, m, K, r, z, sk, k, rz);
    return;
  }
  int kk = k < 0 ? -1 : k % 3;
  uint64_t key = vcycle_key<T>(c, m, K, r, z, sk, kk, rz);
  ++G.vg_clock;
  int slot = -1, lru = 0;
  for (int i = 0; i < MGData::NVG; ++i) {
    if (G.vg[i].exec && G.vg[i].key == key) slot = i;
    if (G.vg[i].used < G.vg[lru].used) lru = i;
  }
  bool fresh = slot < 0;
  if (fresh) slot = lru;
  VGraph& g = G.vg[slot];
  g.used = G.vg_clock;
  if (fresh) {
    cudaStream_t keep = c->stream;
    long long nl0 = c->nlaunch;
    cudaGraph_t graph = nullptr;
    c->stream = c->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        vcycle_launch<T>(c, m, K, r, z, sk, kk, rz);
      } catch (...) {
        cudaStreamEndCapture(c->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        c->stream = keep;
        c->nlaunch = nl0;
        throw;
      }
      e = cudaStreamEndCapture(c->stream, &graph);
    }
    c->stream = keep;
    int nk = (int)(c->nlaunch - nl0);
    c->nlaunch = nl0;
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !g.exec) {
      cudaGetLastError();  // clear a capture or instantiation error
      g.exec = nullptr;
      G.graphs_off = true;
      vcycle_launch<T>(c, m, K, r, z, sk, k, rz);
      return;
    }
    g.key = key;
    g.nkern = nk;
  }
  MPM_CUDA(cudaGraphLaunch(g.exec, c->stream));
  c->nlaunch += g.nkern;
}

void mg_release(mpm_ctx* c, mpm_mesh* m) {
  if (!m->mg) return;
  MGData& G = *m->mg;
  for (VGraph& g : G.vg)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& L : G.lev) {
    Buf* b[] = {&L.gid, &L.xyz, &L.mask, &L.A, &L.Dinv, &L.b, &L.x, &L.r};
    for (Buf* x : b) free_buf(c, *x);
  }
  Buf* b[] = {&G.p_idx, &G.p_w, &G.t_ptr, &G.t_idx, &G.t_w, &G.acc, &G.kp, &G.kpc, &G.bound, &G.fDinv, &G.fx,
              &G.fr, &G.fKh, &G.cinv};
  for (Buf* x : b) free_buf(c, *x);
  delete m->mg;
  m->mg = nullptr;
}

template void mg_setup<float>(mpm_ctx*, mpm_mesh*, const float*, bool);
template void mg_setup<double>(mpm_ctx*, mpm_mesh*, const double*, bool);
template void mg_apply<float>(mpm_ctx*, const mpm_mesh*, const float*, const float*, float*, const Scal*,
                              int, double*);
template void mg_apply<double>(mpm_ctx*, const mpm_mesh*, const double*, const double*, double*,
                               const Scal*, int, double*);

}  // namespace mpm
