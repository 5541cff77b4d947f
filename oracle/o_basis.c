/*
 * Oracle: GIMP domains, the discrete GIMP basis (Sec. 3.2, Eq. GIMP numerical),
 * GIMP refinement (Sec. 5), the block sparsity pattern and the ghost faces and
 * ghost matrix (Sec. 4).  TEST INFRASTRUCTURE ONLY: plain loops, no tuning.
 */
#include "o_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Box bounds closer than this (in finest-grid units) to a grid plane are
 * moved onto the plane, so that rounding never creates sliver overlaps. */
#define O_SNAP 1e-9

static double snap(double v) {
  double r = floor(v + 0.5);
  return fabs(v - r) < O_SNAP ? r : v;
}

/* GIMP domain of point p in finest-grid units: snapped, clipped to the domain.
 * Returns the unclipped (snapped) box volume, which is V_p of Eq. (GIMP basis);
 * reading: the box is clipped to Omega without renormalisation. */
static double point_box(const o_model* m, int p, double* Lo, double* Hi) {
  double N = (double)(1 << m->D), V = 1.0;
  for (int d = 0; d < 3; ++d) {
    double lo = snap((m->x[3 * p + d] - m->lp[3 * p + d]) * m->scale);
    double hi = snap((m->x[3 * p + d] + m->lp[3 * p + d]) * m->scale);
    V *= hi - lo;
    Lo[d] = lo < 0.0 ? 0.0 : lo;
    Hi[d] = hi > N ? N : hi;
  }
  return V;
}

typedef struct {
  int K;
  double a[3], e[3];
} subbox;

/* Partition the box [Lo,Hi] into its intersections with leaves (the set K_p
 * of Sec. 3.2).  Each popped box is cut by the leaf that holds its lowest
 * corner; the remainder is at most three boxes. */
static int overlaps(const o_model* m, const double* Lo, const double* Hi, subbox* out, int max) {
  const o_tree* t = &m->t;
  int N = 1 << m->D;
  double st[3 * O_MAXK + 8][6];
  int ns = 0, n = 0;
  for (int d = 0; d < 3; ++d) {
    st[0][d] = Lo[d];
    st[0][3 + d] = Hi[d];
  }
  ns = 1;
  while (ns > 0) {
    --ns;
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = st[ns][d];
      b[d] = st[ns][3 + d];
    }
    int q[3];
    for (int d = 0; d < 3; ++d) {
      q[d] = (int)floor(a[d]);
      if (q[d] > N - 1) q[d] = N - 1;
      if (q[d] < 0) q[d] = 0;
    }
    int K = o_locate(t, q[0], q[1], q[2]);
    int s = 1 << (m->D - t->lev[K]);
    double kh[3], e[3];
    for (int d = 0; d < 3; ++d) {
      kh[d] = (double)(t->a[3 * K + d] + s);
      e[d] = b[d] < kh[d] ? b[d] : kh[d];
    }
    if (n >= max) return -1;
    out[n].K = K;
    for (int d = 0; d < 3; ++d) {
      out[n].a[d] = a[d];
      out[n].e[d] = e[d];
    }
    ++n;
    if (ns + 3 > 3 * O_MAXK + 8) return -1;
    if (b[0] > kh[0]) {
      double* r = st[ns++];
      r[0] = kh[0]; r[1] = a[1]; r[2] = a[2];
      r[3] = b[0];  r[4] = b[1]; r[5] = b[2];
    }
    if (b[1] > kh[1]) {
      double* r = st[ns++];
      r[0] = a[0]; r[1] = kh[1]; r[2] = a[2];
      r[3] = e[0]; r[4] = b[1];  r[5] = b[2];
    }
    if (b[2] > kh[2]) {
      double* r = st[ns++];
      r[0] = a[0]; r[1] = a[1]; r[2] = kh[2];
      r[3] = e[0]; r[4] = e[1]; r[5] = b[2];
    }
  }
  return n;
}

/* Same cutting as overlaps(), stopping at the first leaf K of K_p with
 * l_K < lim (grid units).  A box that overlaps more leaves than the work list
 * holds necessarily meets leaves far smaller than itself and is split too. */
static int needs_split(const o_model* m, const double* Lo, const double* Hi, double lim) {
  const o_tree* t = &m->t;
  int N = 1 << m->D;
  enum { CAP = 4096 };
  static double st[CAP][6];
  int ns = 1;
  for (int d = 0; d < 3; ++d) {
    st[0][d] = Lo[d];
    st[0][3 + d] = Hi[d];
  }
  while (ns > 0) {
    --ns;
    double a[3], b[3], kh[3], e[3];
    int q[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = st[ns][d];
      b[d] = st[ns][3 + d];
      q[d] = (int)floor(a[d]);
      if (q[d] > N - 1) q[d] = N - 1;
      if (q[d] < 0) q[d] = 0;
    }
    int K = o_locate(t, q[0], q[1], q[2]);
    int s = 1 << (m->D - t->lev[K]);
    if (0.5 * (double)s < lim) return 1;
    for (int d = 0; d < 3; ++d) {
      kh[d] = (double)(t->a[3 * K + d] + s);
      e[d] = b[d] < kh[d] ? b[d] : kh[d];
    }
    if (ns + 3 > CAP) return 1;
    if (b[0] > kh[0]) {
      double* r = st[ns++];
      r[0] = kh[0]; r[1] = a[1]; r[2] = a[2];
      r[3] = b[0];  r[4] = b[1]; r[5] = b[2];
    }
    if (b[1] > kh[1]) {
      double* r = st[ns++];
      r[0] = a[0]; r[1] = kh[1]; r[2] = a[2];
      r[3] = e[0]; r[4] = b[1];  r[5] = b[2];
    }
    if (b[2] > kh[2]) {
      double* r = st[ns++];
      r[0] = a[0]; r[1] = a[1]; r[2] = kh[2];
      r[3] = e[0]; r[4] = e[1]; r[5] = b[2];
    }
  }
  return 0;
}

/* Sec. 5: split GIMP p into 8 if some overlapped leaf has l_K < beta l_p.
 * Reading: l_p is the largest reference half-length l0 (the domain as first
 * generated, halved at each split).  Children copy all state; V0 and m are
 * divided by 8.  Child 0 replaces the parent, children 1..7 are appended in
 * parent order.  Repeated until no point qualifies. */
int o_split_points(o_model* m) {
  for (int round = 0; round < 32; ++round) {
    int np = m->np;
    int* flag = (int*)calloc((size_t)np, sizeof(int));
    int cnt = 0;
    for (int p = 0; p < np; ++p) {
      double Lo[3], Hi[3];
      point_box(m, p, Lo, Hi);
      for (int d = 0; d < 3; ++d)
        if (!(Hi[d] > Lo[d])) {
          free(flag);
          return O_ERR_DOMAIN;
        }
      double l0 = m->l0[3 * p];
      if (m->l0[3 * p + 1] > l0) l0 = m->l0[3 * p + 1];
      if (m->l0[3 * p + 2] > l0) l0 = m->l0[3 * p + 2];
      flag[p] = needs_split(m, Lo, Hi, m->p.beta * l0 * m->scale);
      cnt += flag[p];
    }
    if (cnt == 0) {
      free(flag);
      return O_OK;
    }
    int nn = np + 7 * cnt;
    if (nn > m->cap) {
      int cap = nn;
      m->x = (double*)realloc(m->x, sizeof(double) * 3 * (size_t)cap);
      m->lp = (double*)realloc(m->lp, sizeof(double) * 3 * (size_t)cap);
      m->l0 = (double*)realloc(m->l0, sizeof(double) * 3 * (size_t)cap);
      m->F = (double*)realloc(m->F, sizeof(double) * 9 * (size_t)cap);
      m->be = (double*)realloc(m->be, sizeof(double) * 6 * (size_t)cap);
      m->V0 = (double*)realloc(m->V0, sizeof(double) * (size_t)cap);
      m->mass = (double*)realloc(m->mass, sizeof(double) * (size_t)cap);
      m->E = (double*)realloc(m->E, sizeof(double) * (size_t)cap);
      m->ys = (double*)realloc(m->ys, sizeof(double) * (size_t)cap);
      m->v = (double*)realloc(m->v, sizeof(double) * 3 * (size_t)cap);
      m->cap = cap;
    }
    int next = np;
    for (int p = 0; p < np; ++p) {
      if (!flag[p]) continue;
      double xc[3], lc[3], l0c[3];
      for (int d = 0; d < 3; ++d) {
        xc[d] = m->x[3 * p + d];
        lc[d] = m->lp[3 * p + d];
        l0c[d] = m->l0[3 * p + d];
      }
      for (int c = 0; c < 8; ++c) {
        int q = c == 0 ? p : next++;
        for (int d = 0; d < 3; ++d) {
          double sgn = ((c >> d) & 1) ? 0.5 : -0.5;
          m->x[3 * q + d] = xc[d] + sgn * lc[d];
          m->lp[3 * q + d] = 0.5 * lc[d];
          m->l0[3 * q + d] = 0.5 * l0c[d];
        }
        if (q != p) {
          for (int i = 0; i < 9; ++i) m->F[9 * q + i] = m->F[9 * p + i];
          for (int i = 0; i < 6; ++i) m->be[6 * q + i] = m->be[6 * p + i];
          m->V0[q] = m->V0[p] / 8.0;
          m->mass[q] = m->mass[p] / 8.0;
          m->E[q] = m->E[p];
          m->ys[q] = m->ys[p];
          for (int d = 0; d < 3; ++d) m->v[3 * q + d] = m->v[3 * p + d];
        }
      }
      /* child 0 keeps the parent slot */
      m->V0[p] /= 8.0;
      m->mass[p] /= 8.0;
    }
    m->np = nn;
    free(flag);
  }
  return O_ERR_SUPPORT;
}

/* Eq. (hanging node basis) for every active node of leaf K at local
 * coordinates xi in [0,1]^3: phi~_iK = sum over corners c of phi_cK times the
 * constraint weight of c on i.  Gradients are per finest-grid unit. */
int o_leaf_basis(const o_model* m, int K, const double* xi, int* nent, int* idx, double* phi,
                 double* dphi) {
  int s = 1 << (m->D - m->t.lev[K]);
  int n = 0;
  for (int c = 0; c < 8; ++c) {
    double f[3], g[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = ((c >> d) & 1) ? xi[d] : 1.0 - xi[d];
      g[d] = (((c >> d) & 1) ? 1.0 : -1.0) / (double)s;
    }
    double ph = f[0] * f[1] * f[2];
    double dp[3] = {g[0] * f[1] * f[2], f[0] * g[1] * f[2], f[0] * f[1] * g[2]};
    int node = m->nd.corner[8 * K + c];
    for (int k = m->nd.cptr[node]; k < m->nd.cptr[node + 1]; ++k) {
      int j = m->nd.cidx[k];
      double w = m->nd.cw[k];
      int slot = -1;
      for (int i = 0; i < n; ++i)
        if (idx[i] == j) slot = i;
      if (slot < 0) {
        if (n >= O_MAXS) return O_ERR_SUPPORT;
        slot = n++;
        idx[slot] = j;
        phi[slot] = 0.0;
        dphi[3 * slot] = dphi[3 * slot + 1] = dphi[3 * slot + 2] = 0.0;
      }
      phi[slot] += w * ph;
      for (int d = 0; d < 3; ++d) dphi[3 * slot + d] += w * dp[d];
    }
  }
  *nent = n;
  return O_OK;
}

/* Eq. (GIMP numerical): S_vp = (1/V_p) sum_K phi~_vK(x_Kp) V_Kp, with x_Kp the
 * centre and V_Kp the volume of the box-leaf intersection.  The gradient is
 * the derivative of the same integral with respect to x_p (reading):
 * grad S_vp = (1/V_p) sum_K grad phi~_vK(x_Kp) V_Kp; both are exact for
 * trilinear functions on axis-aligned boxes. */
int o_build_basis(o_model* m) {
  const o_tree* t = &m->t;
  int np = m->np;
  free(m->nsup);
  free(m->sidx);
  free(m->S);
  free(m->dS);
  free(m->populated);
  free(m->betaK);
  m->nsup = (int*)calloc((size_t)np, sizeof(int));
  m->sidx = (int*)malloc(sizeof(int) * O_MAXS * (size_t)np);
  m->S = (double*)calloc(O_MAXS * (size_t)np, sizeof(double));
  m->dS = (double*)calloc(3 * O_MAXS * (size_t)np, sizeof(double));
  m->populated = (int*)calloc((size_t)t->n, sizeof(int));
  m->betaK = (double*)calloc((size_t)t->n, sizeof(double));
  subbox sb[O_MAXK];
  int idx[O_MAXS], nent;
  double ph[O_MAXS], dph[3 * O_MAXS];
  for (int p = 0; p < np; ++p) {
    double Lo[3], Hi[3];
    double Vp = point_box(m, p, Lo, Hi);
    for (int d = 0; d < 3; ++d)
      if (!(Hi[d] > Lo[d])) return O_ERR_DOMAIN;
    int nk = overlaps(m, Lo, Hi, sb, O_MAXK);
    if (nk < 0) return O_ERR_SUPPORT;
    int* si = m->sidx + O_MAXS * (size_t)p;
    double* S = m->S + O_MAXS * (size_t)p;
    double* dS = m->dS + 3 * O_MAXS * (size_t)p;
    int ns = 0;
    for (int k = 0; k < nk; ++k) {
      int K = sb[k].K;
      int s = 1 << (m->D - t->lev[K]);
      double vol = 1.0, xi[3];
      for (int d = 0; d < 3; ++d) {
        vol *= sb[k].e[d] - sb[k].a[d];
        double cen = 0.5 * (sb[k].a[d] + sb[k].e[d]);
        xi[d] = (cen - (double)t->a[3 * K + d]) / (double)s;
      }
      m->populated[K] = 1;
      if (m->E[p] > m->betaK[K]) m->betaK[K] = m->E[p];
      int st = o_leaf_basis(m, K, xi, &nent, idx, ph, dph);
      if (st) return st;
      double w = vol / Vp;
      for (int i = 0; i < nent; ++i) {
        int slot = -1;
        for (int j = 0; j < ns; ++j)
          if (si[j] == idx[i]) slot = j;
        if (slot < 0) {
          if (ns >= O_MAXS) return O_ERR_SUPPORT;
          slot = ns++;
          si[slot] = idx[i];
          S[slot] = 0.0;
          dS[3 * slot] = dS[3 * slot + 1] = dS[3 * slot + 2] = 0.0;
        }
        S[slot] += ph[i] * w;
        for (int d = 0; d < 3; ++d) dS[3 * slot + d] += dph[3 * i + d] * w;
      }
    }
    /* physical gradients; sort the support by node id */
    for (int j = 0; j < 3 * ns; ++j) dS[j] *= m->scale;
    for (int i = 1; i < ns; ++i)
      for (int j = i; j > 0 && si[j - 1] > si[j]; --j) {
        int ti = si[j]; si[j] = si[j - 1]; si[j - 1] = ti;
        double ts = S[j]; S[j] = S[j - 1]; S[j - 1] = ts;
        for (int d = 0; d < 3; ++d) {
          double td = dS[3 * j + d];
          dS[3 * j + d] = dS[3 * (j - 1) + d];
          dS[3 * (j - 1) + d] = td;
        }
      }
    m->nsup[p] = ns;
  }
  /* active nodes: those in some support; dofs numbered in node (Morton) order */
  o_nodes* nd = &m->nd;
  for (int n = 0; n < nd->n; ++n) nd->dof[n] = -1;
  for (int p = 0; p < np; ++p)
    for (int k = 0; k < m->nsup[p]; ++k) nd->dof[m->sidx[O_MAXS * (size_t)p + k]] = 0;
  int nd_ = 0;
  for (int n = 0; n < nd->n; ++n)
    if (nd->dof[n] == 0) nd->dof[n] = nd_++;
  nd->ndof = nd_;
  for (int p = 0; p < np; ++p)
    for (int k = 0; k < m->nsup[p]; ++k) {
      int* s = m->sidx + O_MAXS * (size_t)p + k;
      *s = nd->dof[*s];
    }
  /* Dirichlet mask: components fixed on the roller / fixed planes (Sec. 2.4) */
  free(m->bcmask);
  m->bcmask = (int*)calloc((size_t)(nd_ > 0 ? nd_ : 1), sizeof(int));
  for (int n = 0; n < nd->n; ++n) {
    int dof = nd->dof[n];
    if (dof < 0) continue;
    int mask = 0;
    for (int b = 0; b < m->p.nbc; ++b) {
      int plane = (int)floor(m->p.bc_pos[b] * m->scale + 0.5);
      if (nd->c[3 * n + m->p.bc_axis[b]] == plane) mask |= m->p.bc_mask[b];
    }
    m->bcmask[dof] = mask;
  }
  return O_OK;
}

/* ---------------- pattern and ghost (Sec. 4) ---------------- */

static int cmp_u64(const void* A, const void* B) {
  uint64_t a = *(const uint64_t*)A, b = *(const uint64_t*)B;
  return (a > b) - (a < b);
}

typedef struct {
  int K, N;        /* K the smaller (or equal) leaf whose face is F */
  int axis, sign;  /* outward normal of K: sign * e_axis          */
} gface;

/* leaf of the region just across face (axis, sign) of K, at the offset
 * (o1, o2) along the two tangential axes */
static int across(const o_model* m, int K, int axis, int sign, int o1, int o2) {
  const o_tree* t = &m->t;
  int N = 1 << m->D, s = 1 << (m->D - t->lev[K]);
  int q[3];
  for (int d = 0; d < 3; ++d) q[d] = t->a[3 * K + d];
  q[axis] = sign > 0 ? q[axis] + s : q[axis] - 1;
  if (q[axis] < 0 || q[axis] >= N) return -1;
  int t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
  q[t1] += o1;
  q[t2] += o2;
  return o_locate(t, q[0], q[1], q[2]);
}

int o_find_slot(const o_model* m, int i, int j) {
  int lo = m->row_ptr[i], hi = m->row_ptr[i + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (m->col[mid] == j) return mid;
    if (m->col[mid] < j)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

int o_build_pattern_and_ghost(o_model* m) {
  const o_tree* t = &m->t;
  int nl = t->n, ndof = m->nd.ndof;
  /* boundary elements T^B: populated leaves sharing a face with an unpopulated one */
  int* isB = (int*)calloc((size_t)nl, sizeof(int));
  for (int K = 0; K < nl; ++K) {
    if (!m->populated[K]) continue;
    int s = 1 << (m->D - t->lev[K]);
    for (int f = 0; f < 6 && !isB[K]; ++f) {
      int axis = f / 2, sign = (f & 1) ? 1 : -1;
      int nb = across(m, K, axis, sign, 0, 0);
      if (nb < 0) continue;
      if (t->lev[nb] <= t->lev[K]) {
        if (!m->populated[nb]) isB[K] = 1;
      } else {
        for (int o = 0; o < 4; ++o) {
          int nb2 = across(m, K, axis, sign, (o & 1) * (s / 2), ((o >> 1) & 1) * (s / 2));
          if (!m->populated[nb2]) isB[K] = 1;
        }
      }
    }
  }
  /* ghost faces F_B: both leaves populated, at least one in T^B.  Each face is
   * listed once, from its smaller leaf (equal leaves: from the lower one). */
  int cap = 16, nf = 0;
  gface* fl = (gface*)malloc(sizeof(gface) * (size_t)cap);
  if (m->p.ghost_on) {
    for (int K = 0; K < nl; ++K) {
      if (!m->populated[K]) continue;
      for (int f = 0; f < 6; ++f) {
        int axis = f / 2, sign = (f & 1) ? 1 : -1;
        int nb = across(m, K, axis, sign, 0, 0);
        if (nb < 0) continue;
        if (t->lev[nb] > t->lev[K]) continue;
        if (t->lev[nb] == t->lev[K] && sign < 0) continue;
        if (!m->populated[nb]) continue;
        if (!(isB[K] || isB[nb])) continue;
        if (nf == cap) {
          cap *= 2;
          fl = (gface*)realloc(fl, sizeof(gface) * (size_t)cap);
        }
        fl[nf].K = K;
        fl[nf].N = nb;
        fl[nf].axis = axis;
        fl[nf].sign = sign;
        ++nf;
      }
    }
  }
  free(isB);
  m->nghost = nf;
  /* pattern: pairs from every point support, plus ghost couplings */
  size_t npair = 0;
  for (int p = 0; p < m->np; ++p) npair += (size_t)m->nsup[p] * (size_t)m->nsup[p];
  size_t gpair_cap = (size_t)nf * 2 * O_MAXS * 2 * O_MAXS;
  uint64_t* pr = (uint64_t*)malloc(sizeof(uint64_t) * (npair + gpair_cap + 1));
  size_t c = 0;
  for (int p = 0; p < m->np; ++p) {
    const int* si = m->sidx + O_MAXS * (size_t)p;
    for (int a = 0; a < m->nsup[p]; ++a)
      for (int b = 0; b < m->nsup[p]; ++b)
        pr[c++] = (uint64_t)si[a] * (uint64_t)ndof + (uint64_t)si[b];
  }
  int idxK[O_MAXS], idxN[O_MAXS], nK, nN;
  double phK[O_MAXS], phN[O_MAXS], dK[3 * O_MAXS], dN[3 * O_MAXS];
  double half[3] = {0.5, 0.5, 0.5};
  for (int f = 0; f < nf; ++f) {
    o_leaf_basis(m, fl[f].K, half, &nK, idxK, phK, dK);
    o_leaf_basis(m, fl[f].N, half, &nN, idxN, phN, dN);
    int u[2 * O_MAXS], nu = 0;
    for (int i = 0; i < nK; ++i) u[nu++] = m->nd.dof[idxK[i]];
    for (int i = 0; i < nN; ++i) u[nu++] = m->nd.dof[idxN[i]];
    for (int a = 0; a < nu; ++a)
      for (int b = 0; b < nu; ++b) pr[c++] = (uint64_t)u[a] * (uint64_t)ndof + (uint64_t)u[b];
  }
  qsort(pr, c, sizeof(uint64_t), cmp_u64);
  size_t nu = 0;
  for (size_t i = 0; i < c; ++i)
    if (i == 0 || pr[i] != pr[i - 1]) pr[nu++] = pr[i];
  free(m->row_ptr);
  free(m->col);
  m->nnzb = (int)nu;
  m->row_ptr = (int*)calloc((size_t)ndof + 1, sizeof(int));
  m->col = (int*)malloc(sizeof(int) * (nu > 0 ? nu : 1));
  for (size_t i = 0; i < nu; ++i) {
    int r = (int)(pr[i] / (uint64_t)ndof);
    m->col[i] = (int)(pr[i] % (uint64_t)ndof);
    m->row_ptr[r + 1]++;
  }
  for (int r = 0; r < ndof; ++r) m->row_ptr[r + 1] += m->row_ptr[r];
  free(pr);
  /* Eq. (ghost): j_F = (h_F beta_F / kappa) ([d_n u], [d_n v])_F, integrated by
   * 2x2 Gauss points on the smaller face, mapped into the larger leaf.  Reading:
   * component-wise jumps, so the block is the scalar coefficient times I_3. */
  free(m->kg);
  m->kg = (double*)calloc((size_t)(nu > 0 ? nu : 1), sizeof(double));
  const double gq = 0.5 / sqrt(3.0);
  for (int f = 0; f < nf; ++f) {
    int K = fl[f].K, Nb = fl[f].N, axis = fl[f].axis, sign = fl[f].sign;
    int sK = 1 << (m->D - t->lev[K]), sN = 1 << (m->D - t->lev[Nb]);
    double hF = (double)(sK > sN ? sK : sN) * m->unit;
    double bF = m->betaK[K] > m->betaK[Nb] ? m->betaK[K] : m->betaK[Nb];
    double area = ((double)sK * m->unit) * ((double)sK * m->unit);
    double coef = hF * bF / m->p.kappa * area / 4.0;
    int t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
    for (int g = 0; g < 4; ++g) {
      double X[3];
      X[axis] = (double)t->a[3 * K + axis] + (sign > 0 ? (double)sK : 0.0);
      X[t1] = (double)t->a[3 * K + t1] + (double)sK * ((g & 1) ? 0.5 + gq : 0.5 - gq);
      X[t2] = (double)t->a[3 * K + t2] + (double)sK * ((g & 2) ? 0.5 + gq : 0.5 - gq);
      double xiK[3], xiN[3];
      for (int d = 0; d < 3; ++d) {
        xiK[d] = (X[d] - (double)t->a[3 * K + d]) / (double)sK;
        xiN[d] = (X[d] - (double)t->a[3 * Nb + d]) / (double)sN;
      }
      o_leaf_basis(m, K, xiK, &nK, idxK, phK, dK);
      o_leaf_basis(m, Nb, xiN, &nN, idxN, phN, dN);
      /* jump of the normal derivative, per dof */
      int ids[2 * O_MAXS], n = 0;
      double J[2 * O_MAXS];
      for (int i = 0; i < nK; ++i) {
        ids[n] = m->nd.dof[idxK[i]];
        J[n] = sign * dK[3 * i + axis] * m->scale;
        ++n;
      }
      for (int i = 0; i < nN; ++i) {
        int dof = m->nd.dof[idxN[i]], slot = -1;
        for (int j = 0; j < n; ++j)
          if (ids[j] == dof) slot = j;
        if (slot < 0) {
          slot = n++;
          ids[slot] = dof;
          J[slot] = 0.0;
        }
        J[slot] -= sign * dN[3 * i + axis] * m->scale;
      }
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          int sl = o_find_slot(m, ids[a], ids[b]);
          m->kg[sl] += coef * J[a] * J[b];
        }
    }
  }
  free(m->gface);
  m->gface = (int*)malloc(sizeof(int) * 4 * (size_t)(nf > 0 ? nf : 1));
  for (int f = 0; f < nf; ++f) {
    m->gface[4 * f] = fl[f].K;
    m->gface[4 * f + 1] = fl[f].N;
    m->gface[4 * f + 2] = fl[f].axis;
    m->gface[4 * f + 3] = fl[f].sign;
  }
  free(fl);
  return O_OK;
}
