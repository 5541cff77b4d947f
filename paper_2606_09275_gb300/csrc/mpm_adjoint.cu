// Discrete adjoint of a sequence of quasi-static load steps (Sec. 2.4 Newton
// load steps with the re-adaptation of Sec. 5): gradients of a linear
// functional of the final reaction force with respect to the per-point Young's
// modulus and yield stress.  Discrete events (octree, GIMP splits, supports,
// plastic/elastic branch, contact set, ghost faces and their beta) are frozen
// at their forward values.  Per step, in reverse:
//   1. restore the checkpoint, rebuild the mesh (recording the splits) and
//      re-solve Newton for the converged increment u;
//   2. adjoint right-hand side from the point update (x, F, b_e, l) and, for
//      the last step, from the reaction;
//   3. K mu = rhs with the (symmetric) consistent tangent;
//   4. backward kernels of -mu^T R through the constitutive update, the basis,
//      the contact and the ghost coefficients;
//   5. fold the adjoints of split children into their parents.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mpm_internal.cuh"
#include "mpm_law.cuh"

namespace mpm {
namespace {

// ---------------------------------------------------------------- small 3x3 helpers

__device__ inline void mm3(const double* a, const double* b, double* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}
__device__ inline void mtm3(const double* a, const double* b, double* c) {  // a^T b
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[i] * b[j] + a[3 + i] * b[3 + j] + a[6 + i] * b[6 + j];
}
__device__ inline void mmt3(const double* a, const double* b, double* c) {  // a b^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      c[3 * i + j] = a[3 * i] * b[3 * j] + a[3 * i + 1] * b[3 * j + 1] + a[3 * i + 2] * b[3 * j + 2];
}
__device__ inline double det33(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}
__device__ inline void inv33(const double* a, double* o) {
  double id = 1.0 / det33(a);
  o[0] = (a[4] * a[8] - a[5] * a[7]) * id;
  o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  o[3] = (a[5] * a[6] - a[3] * a[8]) * id;
  o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  o[6] = (a[3] * a[7] - a[4] * a[6]) * id;
  o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}
// symmetric matrix from the 6-component storage (xx yy zz xy yz xz)
__device__ inline void sym6_to9(const double* s, double* m) {
  m[0] = s[0]; m[4] = s[1]; m[8] = s[2];
  m[1] = m[3] = s[3]; m[5] = m[7] = s[4]; m[2] = m[6] = s[5];
}
// adjoint of the 6-component storage: off-diagonal entries count twice
__device__ inline void adj9_to6(const double* m, double* s) {
  s[0] = m[0]; s[1] = m[4]; s[2] = m[8];
  s[3] = m[1] + m[3]; s[4] = m[5] + m[7]; s[5] = m[2] + m[6];
}
// B = Q B' Q^T and B' = Q^T B Q
__device__ inline void rot_out(const double* Q, const double* Bp, double* B) {
  double t[9];
  mm3(Q, Bp, t);
  mmt3(t, Q, B);
}
__device__ inline void rot_in(const double* Q, const double* B, double* Bp) {
  double t[9];
  mtm3(Q, B, t);
  mm3(t, Q, Bp);
}

// ---------------------------------------------------------------- law state

struct LawState {
  double lam[3], Q[9], eps[3], ta[3], dd[9], gr, bw[3];
  double mu, lm, kb, nh[3];
  int plastic;
};

// the forward law at (b_e,n, dF) with every intermediate kept
__device__ bool law_state(const Law& L, double E, double ys, const double* be6, const double* dF,
                          LawState& S) {
  double b[9], t[9], bt[9];
  sym6_to9(be6, b);
  mm3(dF, b, t);
  mmt3(t, dF, bt);
  bt[1] = bt[3] = 0.5 * (bt[1] + bt[3]);
  bt[2] = bt[6] = 0.5 * (bt[2] + bt[6]);
  bt[5] = bt[7] = 0.5 * (bt[5] + bt[7]);
  jacobi3(bt, S.lam, S.Q);
  if (!(S.lam[0] > 0 && S.lam[1] > 0 && S.lam[2] > 0)) return false;
  for (int a = 0; a < 3; ++a) S.eps[a] = 0.5 * log(S.lam[a]);
  principal_return(L, E, ys, S.eps, S.ta, S.dd, &S.gr);
  S.mu = E / (2.0 * (1.0 + L.nu));
  S.lm = E * L.nu / ((1.0 + L.nu) * (1.0 - 2.0 * L.nu));
  S.kb = S.lm + 2.0 * S.mu / 3.0;
  double tr = S.eps[0] + S.eps[1] + S.eps[2], dn = 0.0;
  for (int a = 0; a < 3; ++a) {
    S.nh[a] = S.eps[a] - tr / 3.0;
    dn += S.nh[a] * S.nh[a];
  }
  dn = sqrt(dn);
  for (int a = 0; a < 3; ++a) S.nh[a] = dn > 0 ? S.nh[a] / dn : 0.0;
  S.plastic = (L.model == 1 && 1.224744871391589 * 2.0 * S.mu * dn > ys) ? 1 : 0;
  double tt = S.ta[0] + S.ta[1] + S.ta[2];
  for (int a = 0; a < 3; ++a)
    S.bw[a] = exp(2.0 * (S.ta[a] - S.lm * tt / (3.0 * S.lm + 2.0 * S.mu)) / (2.0 * S.mu));
  return true;
}

// adjoint of tau(b_tr; E, ys): given the symmetric seed tb, add to bbar (3x3)
// the b_tr adjoint and to (gE, gys) the parameter adjoints
__device__ void tau_adjoint(const LawState& S, double E, const double* tb, double* bbar, double* gE,
                            double* gys) {
  double Yp[9], Bp[9];
  rot_in(S.Q, tb, Yp);
  for (int b = 0; b < 3; ++b) {
    double v = 0.0;
    for (int a = 0; a < 3; ++a) v += Yp[4 * a] * S.dd[3 * a + b];
    Bp[4 * b] = v / (2.0 * S.lam[b]);
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b) Bp[3 * a + b] = 0.5 * S.gr * ln_divdiff(S.lam[a], S.lam[b]) * Yp[3 * a + b];
  double B[9];
  rot_out(S.Q, Bp, B);
  for (int i = 0; i < 9; ++i) bbar[i] += B[i];
  double tr = S.eps[0] + S.eps[1] + S.eps[2];
  for (int a = 0; a < 3; ++a) {
    if (S.plastic) {
      *gE += Yp[4 * a] * S.kb * tr / E;
      *gys += Yp[4 * a] * 0.816496580927726 * S.nh[a];
    } else {
      *gE += Yp[4 * a] * S.ta[a] / E;
    }
  }
}

// adjoint of b_e,new(b_tr; E, ys)
__device__ void be_adjoint(const LawState& S, double E, double ys, const double* Bb, double* bbar,
                           double* gE, double* gys) {
  double Yp[9], Bp[9];
  rot_in(S.Q, Bb, Yp);
  // d bw_a / d lam_b = bw_a (Dinv d)_ab / lam_b,  Dinv_ac = (delta_ac - lm/(3lm+2mu))/(2mu)
  double c0 = S.lm / (3.0 * S.lm + 2.0 * S.mu);
  for (int b = 0; b < 3; ++b) {
    double v = 0.0;
    for (int a = 0; a < 3; ++a) {
      double sumd = S.dd[b] + S.dd[3 + b] + S.dd[6 + b];  // sum_c d_cb
      double dinvd = (S.dd[3 * a + b] - c0 * sumd) / (2.0 * S.mu);
      v += Yp[4 * a] * S.bw[a] * dinvd / S.lam[b];
    }
    Bp[4 * b] = v;
  }
  double f = S.gr / (2.0 * S.mu);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      if (a == b) continue;
      double rho;
      if (!S.plastic) {
        rho = 1.0;
      } else {
        double D = S.eps[a] - S.eps[b];
        double eeb = 0.5 * log(S.bw[b]);
        double pre = exp(2.0 * (eeb - S.eps[b]));
        rho = fabs(D) < 1e-8 ? pre * f * (1.0 + (f - 1.0) * D) : pre * expm1(2.0 * f * D) / expm1(2.0 * D);
      }
      Bp[3 * a + b] = rho * Yp[3 * a + b];
    }
  double B[9];
  rot_out(S.Q, Bp, B);
  for (int i = 0; i < 9; ++i) bbar[i] += B[i];
  if (S.plastic) {
    for (int a = 0; a < 3; ++a) {
      double sa = ys * 0.816496580927726 * S.nh[a];
      *gE += Yp[4 * a] * 2.0 * S.bw[a] * (-sa / (2.0 * S.mu * E));
      *gys += Yp[4 * a] * 2.0 * S.bw[a] * (0.816496580927726 * S.nh[a] / (2.0 * S.mu));
    }
  }
}

// ---------------------------------------------------------------- adjoint state

struct Adj {
  double *x, *lp, *F, *be, *E, *ys;  // canonical order
};

// 1a. point update backward: x' = x + sum S u, F' = dF F, b_e' = b_e,new,
// l' = l0 diag(sqrt(F'^T F')).  Seeds from a (state after the step); writes
// the explicit adjoints of the state before the step into mid, the basis
// adjoints into Sb/Gb, and adds the nodal seed to ub.
__global__ void k_adj_update(int P, Law L, const int* __restrict__ perm, const int* __restrict__ nsup,
                             const int* __restrict__ sidx, const double* __restrict__ S,
                             const double* __restrict__ dS, const double* __restrict__ u,
                             const double* __restrict__ pE, const double* __restrict__ pys,
                             const double* __restrict__ pbe, const double* __restrict__ pF,
                             const double* __restrict__ pl0, Adj a, Adj mid, double* Sb, double* Gb,
                             double* ub, int* err) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  size_t p = perm[w];
  int n = nsup[w];
  double dF[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  for (int k = 0; k < n; ++k) {
    size_t o = (size_t)w * MAXS + k;
    int j = sidx[o];
    for (int i = 0; i < 3; ++i)
      for (int jj = 0; jj < 3; ++jj) dF[3 * i + jj] += u[3 * (size_t)j + i] * dS[3 * o + jj];
  }
  LawState LS;
  double E = pE[w], ys = pys[w];
  if (!law_state(L, E, ys, pbe + 6 * (size_t)w, dF, LS)) {
    atomicOr(err, EB_NAN);
    return;
  }
  const double* Fo = pF + 9 * (size_t)w;
  double Fn[9];
  mm3(dF, Fo, Fn);
  // stretch: lbar' -> Fbar'
  double Fb[9];
  for (int i = 0; i < 9; ++i) Fb[i] = a.F[9 * p + i];
  {
    double C[9], mu_[3], N[9];
    mtm3(Fn, Fn, C);
    jacobi3(C, mu_, N);
    double Ub[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int d = 0; d < 3; ++d) Ub[4 * d] = pl0[3 * (size_t)w + d] * a.lp[3 * p + d];
    double Up[9], Cp[9], Cb[9];
    rot_in(N, Ub, Up);
    double sq[3] = {sqrt(mu_[0]), sqrt(mu_[1]), sqrt(mu_[2])};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Cp[3 * i + j] = i == j ? Up[4 * i] / (2.0 * sq[i]) : Up[3 * i + j] / (sq[i] + sq[j]);
    rot_out(N, Cp, Cb);
    double t[9];
    mm3(Fn, Cb, t);
    for (int i = 0; i < 9; ++i) Fb[i] += t[i] + t[i];  // C = F^T F, Cbar symmetric
  }
  // F' = dF F_n
  double dFb[9], Fob[9];
  mmt3(Fb, Fo, dFb);   // Fbar' F_n^T
  mtm3(dF, Fb, Fob);   // dF^T Fbar'
  // b_e' = b_e,new(b_tr)
  double Bb[9], bbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gE = 0.0, gys = 0.0;
  {
    double s6[6];
    for (int i = 0; i < 6; ++i) s6[i] = a.be[6 * p + i];
    // adjoint seed of the 6-storage -> symmetric matrix adjoint
    Bb[0] = s6[0]; Bb[4] = s6[1]; Bb[8] = s6[2];
    Bb[1] = Bb[3] = 0.5 * s6[3]; Bb[5] = Bb[7] = 0.5 * s6[4]; Bb[2] = Bb[6] = 0.5 * s6[5];
  }
  be_adjoint(LS, E, ys, Bb, bbar, &gE, &gys);
  // b_tr = dF b_n dF^T
  double bn[9], t1[9], t2[9];
  sym6_to9(pbe + 6 * (size_t)w, bn);
  double bs[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) bs[3 * i + j] = 0.5 * (bbar[3 * i + j] + bbar[3 * j + i]);
  mm3(bs, dF, t1);
  mm3(t1, bn, t2);
  for (int i = 0; i < 9; ++i) dFb[i] += 2.0 * t2[i];
  double bnb[9];
  mtm3(dF, bs, t1);
  mm3(t1, dF, bnb);
  double bn6[6];
  adj9_to6(bnb, bn6);
  // x' = x + sum S u; dF = I + sum u (x) G
  double xb[3] = {a.x[3 * p], a.x[3 * p + 1], a.x[3 * p + 2]};
  for (int k = 0; k < n; ++k) {
    size_t o = (size_t)w * MAXS + k;
    int j = sidx[o];
    const double* uj = u + 3 * (size_t)j;
    Sb[o] = xb[0] * uj[0] + xb[1] * uj[1] + xb[2] * uj[2];
    const double* g = dS + 3 * o;
    for (int c = 0; c < 3; ++c) Gb[3 * o + c] = dFb[c] * uj[0] + dFb[3 + c] * uj[1] + dFb[6 + c] * uj[2];
    for (int i = 0; i < 3; ++i)
      atomicAdd(ub + 3 * (size_t)j + i, S[o] * xb[i] + dFb[3 * i] * g[0] + dFb[3 * i + 1] * g[1] + dFb[3 * i + 2] * g[2]);
  }
  for (int d = 0; d < 3; ++d) {
    mid.x[3 * p + d] = xb[d];
    mid.lp[3 * p + d] = 0.0;
  }
  for (int i = 0; i < 9; ++i) mid.F[9 * p + i] = Fob[i];
  for (int i = 0; i < 6; ++i) mid.be[6 * p + i] = bn6[i];
  a.E[p] += gE;
  a.ys[p] += gys;
}

// ---------------------------------------------------------------- contact corner basis

// background basis (dof, value, physical gradient) at corner c of sorted point w,
// in the leaf on the inside of the domain; clipped axes give zero gradient
__device__ int corner_basis(int w, int c, const Geo& g, const double* px, const double* plp,
                            const uint64_t* lkey, const int* llev, int nl, const int* corner,
                            const int* cptr, const int* cidx, const double* cw, const int* node_dof,
                            int* ids, double* ph, double* gph, double* y0) {
  double Lo[3], Hi[3];
  bool clip_lo[3], clip_hi[3];
  for (int d = 0; d < 3; ++d) {
    double lo = snap_grid((px[3 * (size_t)w + d] - plp[3 * (size_t)w + d]) * g.scale);
    double hi = snap_grid((px[3 * (size_t)w + d] + plp[3 * (size_t)w + d]) * g.scale);
    clip_lo[d] = lo < 0.0;
    clip_hi[d] = hi > (double)g.N;
    Lo[d] = clip_lo[d] ? 0.0 : lo;
    Hi[d] = clip_hi[d] ? (double)g.N : hi;
  }
  int q[3];
  double X[3];
  bool fixed[3];
  for (int d = 0; d < 3; ++d) {
    int side = (c >> d) & 1;
    X[d] = side ? Hi[d] : Lo[d];
    fixed[d] = side ? clip_hi[d] : clip_lo[d];
    int v = side ? (int)ceil(X[d]) - 1 : (int)floor(X[d]);
    q[d] = v < 0 ? 0 : (v > g.N - 1 ? g.N - 1 : v);
    y0[d] = px[3 * (size_t)w + d] + (side ? 1.0 : -1.0) * plp[3 * (size_t)w + d];
  }
  int K = locate(lkey, nl, q[0], q[1], q[2]);
  int s = 1 << (g.D - llev[K]);
  int a[3];
  demorton(lkey[K], a);
  double xi[3];
  for (int d = 0; d < 3; ++d) xi[d] = (X[d] - (double)a[d]) / (double)s;
  int n = 0;
  for (int cc = 0; cc < 8; ++cc) {
    double f[3], sg[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = ((cc >> d) & 1) ? xi[d] : 1.0 - xi[d];
      sg[d] = ((cc >> d) & 1) ? 1.0 : -1.0;
    }
    double phv = f[0] * f[1] * f[2];
    double gv[3] = {sg[0] * f[1] * f[2], f[0] * sg[1] * f[2], f[0] * f[1] * sg[2]};
    for (int d = 0; d < 3; ++d) gv[d] = fixed[d] ? 0.0 : gv[d] * g.scale / (double)s;
    int node = corner[8 * (size_t)K + cc];
    for (int t = cptr[node]; t < cptr[node + 1]; ++t) {
      int j = node_dof[cidx[t]];
      if (j < 0) continue;
      int slot = -1;
      for (int e = 0; e < n; ++e)
        if (ids[e] == j) slot = e;
      if (slot < 0) {
        if (n >= MAXCB) continue;
        slot = n++;
        ids[slot] = j;
        ph[slot] = 0.0;
        gph[3 * slot] = gph[3 * slot + 1] = gph[3 * slot + 2] = 0.0;
      }
      ph[slot] += cw[t] * phv;
      for (int d = 0; d < 3; ++d) gph[3 * slot + d] += cw[t] * gv[d];
    }
  }
  return n;
}

struct MeshView {
  Geo g;
  const double *px, *plp;
  const uint64_t* lkey;
  const int* llev;
  int nl;
  const int *corner, *cptr, *cidx;
  const double* cw;
  const int* node_dof;
};

// contact backward, one thread per candidate corner.  mode 0: -mu^T R_c terms
// (x, l and E adjoints); mode 1: the reaction functional J = w . reaction
// (nodal seed into ub and x, l, E adjoints).
__global__ void k_adj_contact(int nc8, int mode, const int* __restrict__ cand, MeshView mv,
                              const int* __restrict__ perm, const double* __restrict__ pE,
                              const double* __restrict__ pV0, Body body, double pf,
                              const double* __restrict__ u, const double* __restrict__ mu, double w0,
                              double w1, double w2, double* ub, Adj mid, Adj a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc8) return;
  int w = cand[i >> 3], c = i & 7;
  int ids[MAXCB];
  double ph[MAXCB], gph[3 * MAXCB], y[3];
  int n = corner_basis(w, c, mv.g, mv.px, mv.plp, mv.lkey, mv.llev, mv.nl, mv.corner, mv.cptr, mv.cidx,
                       mv.cw, mv.node_dof, ids, ph, gph, y);
  for (int e = 0; e < n; ++e)
    for (int d = 0; d < 3; ++d) y[d] += ph[e] * u[3 * (size_t)ids[e] + d];
  double phi, nv[3], H[9];
  if (!body_sdf(body, mv.g.L, y, &phi, nv, H) || !(phi < 0.0)) return;
  double E = pE[w];
  double eps = pf * E * pow(pV0[w], 2.0 / 3.0);
  double f[3] = {-eps * phi * nv[0], -eps * phi * nv[1], -eps * phi * nv[2]};
  size_t p = perm[w];
  double xc[3], gE;
  if (mode == 0) {
    double muc[3] = {0, 0, 0};
    for (int e = 0; e < n; ++e)
      for (int d = 0; d < 3; ++d) muc[d] += ph[e] * mu[3 * (size_t)ids[e] + d];
    double mn = muc[0] * nv[0] + muc[1] * nv[1] + muc[2] * nv[2];
    double gy[3];
    for (int d = 0; d < 3; ++d)
      gy[d] = -eps * (nv[d] * mn + phi * (H[3 * d] * muc[0] + H[3 * d + 1] * muc[1] + H[3 * d + 2] * muc[2]));
    for (int d = 0; d < 3; ++d) xc[d] = gy[d];
    for (int e = 0; e < n; ++e) {
      const double* mj = mu + 3 * (size_t)ids[e];
      const double* uj = u + 3 * (size_t)ids[e];
      double mf = mj[0] * f[0] + mj[1] * f[1] + mj[2] * f[2];
      double ug = uj[0] * gy[0] + uj[1] * gy[1] + uj[2] * gy[2];
      for (int d = 0; d < 3; ++d) xc[d] += gph[3 * e + d] * (mf + ug);
    }
    gE = (muc[0] * f[0] + muc[1] * f[1] + muc[2] * f[2]) / E;
  } else {
    double wn = w0 * nv[0] + w1 * nv[1] + w2 * nv[2];
    double wv[3] = {w0, w1, w2};
    double jy[3];
    for (int d = 0; d < 3; ++d)
      jy[d] = eps * (nv[d] * wn + phi * (H[3 * d] * wv[0] + H[3 * d + 1] * wv[1] + H[3 * d + 2] * wv[2]));
    for (int d = 0; d < 3; ++d) xc[d] = jy[d];
    for (int e = 0; e < n; ++e) {
      const double* uj = u + 3 * (size_t)ids[e];
      double ug = uj[0] * jy[0] + uj[1] * jy[1] + uj[2] * jy[2];
      for (int d = 0; d < 3; ++d) {
        xc[d] += gph[3 * e + d] * ug;
        atomicAdd(ub + 3 * (size_t)ids[e] + d, ph[e] * jy[d]);
      }
    }
    gE = -(w0 * f[0] + w1 * f[1] + w2 * f[2]) / E;
  }
  for (int d = 0; d < 3; ++d) {
    double sg = ((c >> d) & 1) ? 1.0 : -1.0;
    atomicAdd(mid.x + 3 * p + d, xc[d]);
    atomicAdd(mid.lp + 3 * p + d, sg * xc[d]);
  }
  atomicAdd(a.E + p, gE);
}

// ---------------------------------------------------------------- residual backward

// -mu^T (f_int - load f_ext) at fixed u: basis adjoints, b_e,n and parameters
__global__ void k_adj_residual(int P, Law L, double load, double g0, double g1, double g2,
                               const int* __restrict__ perm, const int* __restrict__ nsup,
                               const int* __restrict__ sidx, const double* __restrict__ dS,
                               const double* __restrict__ u, const double* __restrict__ mu,
                               const double* __restrict__ pE, const double* __restrict__ pys,
                               const double* __restrict__ pbe, const double* __restrict__ pV0,
                               const double* __restrict__ pmass, Adj mid, Adj a, double* Sb, double* Gb,
                               int* err) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  size_t p = perm[w];
  int n = nsup[w];
  double dF[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < n; ++k) {
    size_t o = (size_t)w * MAXS + k;
    int j = sidx[o];
    for (int i = 0; i < 3; ++i)
      for (int jj = 0; jj < 3; ++jj) {
        dF[3 * i + jj] += u[3 * (size_t)j + i] * dS[3 * o + jj];
        M[3 * i + jj] += mu[3 * (size_t)j + i] * dS[3 * o + jj];
      }
  }
  LawState LS;
  double E = pE[w], ys = pys[w];
  if (!law_state(L, E, ys, pbe + 6 * (size_t)w, dF, LS)) {
    atomicOr(err, EB_NAN);
    return;
  }
  double tau[9], tp[9] = {LS.ta[0], 0, 0, 0, LS.ta[1], 0, 0, 0, LS.ta[2]};
  rot_out(LS.Q, tp, tau);
  double V0 = pV0[w];
  double Fi[9], FiT[9];
  inv33(dF, Fi);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) FiT[3 * i + j] = Fi[3 * j + i];
  // Phi = V0 tau : (M dF^{-1})
  double MFi[9], Mb[9], dFb[9], tb[9], t1[9], t2[9];
  mm3(M, Fi, MFi);
  mm3(tau, FiT, Mb);
  for (int i = 0; i < 9; ++i) Mb[i] *= V0;                      // dPhi/dM
  mtm3(MFi, tau, t1);                                           // (M Fi)^T tau
  mm3(t1, FiT, t2);
  for (int i = 0; i < 9; ++i) dFb[i] = -V0 * t2[i];             // via dF^{-1}
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) tb[3 * i + j] = 0.5 * V0 * (MFi[3 * i + j] + MFi[3 * j + i]);
  double bbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gE = 0.0, gys = 0.0;
  tau_adjoint(LS, E, tb, bbar, &gE, &gys);
  double bn[9], bs[9];
  sym6_to9(pbe + 6 * (size_t)w, bn);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) bs[3 * i + j] = 0.5 * (bbar[3 * i + j] + bbar[3 * j + i]);
  mm3(bs, dF, t1);
  mm3(t1, bn, t2);
  for (int i = 0; i < 9; ++i) dFb[i] += 2.0 * t2[i];
  double bnb[9], bn6[6];
  mtm3(dF, bs, t1);
  mm3(t1, dF, bnb);
  adj9_to6(bnb, bn6);
  // subtract dPhi/ds: G, S, b_e,n and the parameters
  double m = pmass[w];
  for (int k = 0; k < n; ++k) {
    size_t o = (size_t)w * MAXS + k;
    int j = sidx[o];
    const double* mj = mu + 3 * (size_t)j;
    const double* uj = u + 3 * (size_t)j;
    for (int c = 0; c < 3; ++c)
      Gb[3 * o + c] -= Mb[c] * mj[0] + Mb[3 + c] * mj[1] + Mb[6 + c] * mj[2] +
                       dFb[c] * uj[0] + dFb[3 + c] * uj[1] + dFb[6 + c] * uj[2];
    Sb[o] += load * m * (mj[0] * g0 + mj[1] * g1 + mj[2] * g2);
  }
  for (int i = 0; i < 6; ++i) mid.be[6 * p + i] -= bn6[i];
  a.E[p] -= gE;
  a.ys[p] -= gys;
}

// ---------------------------------------------------------------- ghost backward

// -mu^T K_G u: K_G is proportional to beta_F, the modulus of the argmax point
__global__ void k_adj_ghost(int nf, Geo g, double kappa, const int* __restrict__ face,
                            const uint64_t* __restrict__ lkey, const int* __restrict__ llev,
                            const double* __restrict__ betaK, const int* __restrict__ argK,
                            const int* __restrict__ gdof, const int* __restrict__ gn,
                            const int* __restrict__ corner, const int* __restrict__ cptr,
                            const int* __restrict__ cidx, const double* __restrict__ cw,
                            const int* __restrict__ node_dof, const double* __restrict__ u,
                            const double* __restrict__ mu, double* aE) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int K = face[4 * f], Nb = face[4 * f + 1], axis = face[4 * f + 2], sign = face[4 * f + 3];
  int sK = 1 << (g.D - llev[K]), sN = 1 << (g.D - llev[Nb]);
  int aK[3], aN[3];
  demorton(lkey[K], aK);
  demorton(lkey[Nb], aN);
  double hF = (double)(sK > sN ? sK : sN) * g.unit;
  int Kb = betaK[K] >= betaK[Nb] ? K : Nb;
  double bF = betaK[Kb];
  int pstar = argK[Kb];
  if (pstar < 0 || pstar == 0x7fffffff || !(bF > 0)) return;
  double area = ((double)sK * g.unit) * ((double)sK * g.unit);
  double coef = hF * bF / kappa * area / 4.0;
  const double gq = 0.5 / sqrt(3.0);
  int t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
  int n = gn[f];
  const int* ids = gdof + (size_t)f * MAXG;
  double phi_face = 0.0;
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
    double Jm[3] = {0, 0, 0}, Ju[3] = {0, 0, 0};
    for (int e = 0; e < n; ++e) {
      int j = ids[e];
      double jv = 0.0;
      for (int side = 0; side < 2; ++side) {
        int L = side ? Nb : K, s = side ? sN : sK;
        const double* xi = side ? xiN : xiK;
        for (int c = 0; c < 8; ++c) {
          double fv[3];
          for (int d = 0; d < 3; ++d) fv[d] = ((c >> d) & 1) ? xi[d] : 1.0 - xi[d];
          fv[axis] = (((c >> axis) & 1) ? 1.0 : -1.0) / (double)s;
          double dp = fv[0] * fv[1] * fv[2];
          int node = corner[8 * (size_t)L + c];
          for (int t = cptr[node]; t < cptr[node + 1]; ++t)
            if (node_dof[cidx[t]] == j) jv += (side ? -1.0 : 1.0) * cw[t] * dp;
        }
      }
      jv *= (double)sign * g.scale;
      for (int d = 0; d < 3; ++d) {
        Jm[d] += jv * mu[3 * (size_t)j + d];
        Ju[d] += jv * u[3 * (size_t)j + d];
      }
    }
    phi_face += coef * (Jm[0] * Ju[0] + Jm[1] * Ju[1] + Jm[2] * Ju[2]);
  }
  atomicAdd(aE + pstar, -phi_face / bF);
}

// ---------------------------------------------------------------- basis backward

constexpr int AW = 4;

struct ASub {
  double a[3], e[3];
  int K, s;
  unsigned char lo_dep[3], hi_dep[3];
};

// S_vp, grad S_vp as functions of the domain box [x - l, x + l] with the
// leaf-intersection structure frozen; one warp per point.  Also records, per
// leaf, the lowest caller index among the points with the leaf's beta.
__global__ void __launch_bounds__(32 * AW)
    k_adj_basis(int P, Geo g, const int* __restrict__ perm, const double* __restrict__ px,
                const double* __restrict__ plp, const double* __restrict__ pE,
                const double* __restrict__ betaK, const uint64_t* __restrict__ lkey,
                const int* __restrict__ llev, int nl, const int* __restrict__ corner,
                const int* __restrict__ cptr, const int* __restrict__ cidx,
                const double* __restrict__ cw, const int* __restrict__ node_dof,
                const int* __restrict__ nsup, const int* __restrict__ sidx,
                const double* __restrict__ Sb, const double* __restrict__ Gb, Adj mid, int* argK,
                int* err) {
  __shared__ ASub sb[AW][MAXK];
  __shared__ double wb[AW][MAXK], xb[AW][MAXK][3];
  __shared__ int nsub_s[AW];
  __shared__ double vp_s[AW], lo_s[AW][3], hi_s[AW][3];
  __shared__ unsigned char clo_s[AW][3], chi_s[AW][3];
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int w = blockIdx.x * AW + wi;
  if (w >= P) return;
  if (lane == 0) {
    double lo[3], hi[3], Lo[3], Hi[3], Vp = 1.0;
    for (int d = 0; d < 3; ++d) {
      lo[d] = snap_grid((px[3 * (size_t)w + d] - plp[3 * (size_t)w + d]) * g.scale);
      hi[d] = snap_grid((px[3 * (size_t)w + d] + plp[3 * (size_t)w + d]) * g.scale);
      Vp *= hi[d] - lo[d];
      clo_s[wi][d] = lo[d] < 0.0;
      chi_s[wi][d] = hi[d] > (double)g.N;
      Lo[d] = clo_s[wi][d] ? 0.0 : lo[d];
      Hi[d] = chi_s[wi][d] ? (double)g.N : hi[d];
      lo_s[wi][d] = lo[d];
      hi_s[wi][d] = hi[d];
    }
    vp_s[wi] = Vp;
    double st[3 * MAXK + 8][6];
    int ns = 1, nsub = 0;
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
        q[d] = q[d] > g.N - 1 ? g.N - 1 : (q[d] < 0 ? 0 : q[d]);
      }
      int K = locate(lkey, nl, q[0], q[1], q[2]);
      int s = 1 << (g.D - llev[K]);
      int ka[3];
      demorton(lkey[K], ka);
      for (int d = 0; d < 3; ++d) {
        kh[d] = (double)(ka[d] + s);
        e[d] = b[d] < kh[d] ? b[d] : kh[d];
      }
      if (nsub >= MAXK || ns + 3 > 3 * MAXK + 8) {
        atomicOr(err, EB_SUPPORT);
        nsub = -1;
        break;
      }
      ASub& o = sb[wi][nsub];
      o.K = K;
      o.s = s;
      for (int d = 0; d < 3; ++d) {
        o.a[d] = a[d];
        o.e[d] = e[d];
        o.lo_dep[d] = (a[d] == Lo[d]) && !clo_s[wi][d];
        o.hi_dep[d] = (e[d] == Hi[d]) && !chi_s[wi][d];
        xb[wi][nsub][d] = 0.0;
      }
      wb[wi][nsub] = 0.0;
      ++nsub;
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
    nsub_s[wi] = nsub;
  }
  __syncwarp();
  int nsub = nsub_s[wi];
  if (nsub < 0) return;
  size_t p = perm[w];
  if (lane < nsub) {
    int K = sb[wi][lane].K;
    if (pE[w] == betaK[K]) atomicMin(argK + K, (int)p);
  }
  // entries (sub, corner, constraint): adjoints of w and xi per sub-box
  int ns_sup = nsup[w];
  const int* sup = sidx + (size_t)w * MAXS;
  for (int q = lane; q < 8 * nsub; q += 32) {
    const ASub& o = sb[wi][q >> 3];
    int c = q & 7;
    double vol = 1.0, xi[3];
    for (int d = 0; d < 3; ++d) vol *= o.e[d] - o.a[d];
    int ka[3];
    demorton(lkey[o.K], ka);
    for (int d = 0; d < 3; ++d) xi[d] = (0.5 * (o.a[d] + o.e[d]) - (double)ka[d]) / (double)o.s;
    double wv = vol / vp_s[wi];
    double f[3], sg[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = ((c >> d) & 1) ? xi[d] : 1.0 - xi[d];
      sg[d] = ((c >> d) & 1) ? 1.0 : -1.0;
    }
    double phv = f[0] * f[1] * f[2];
    double gr[3] = {sg[0] * f[1] * f[2], f[0] * sg[1] * f[2], f[0] * f[1] * sg[2]};
    double H01 = sg[0] * sg[1] * f[2], H02 = sg[0] * f[1] * sg[2], H12 = f[0] * sg[1] * sg[2];
    double sc = g.scale / (double)o.s;
    int node = corner[8 * (size_t)o.K + c];
    double wacc = 0.0, xacc[3] = {0, 0, 0};
    for (int t = cptr[node]; t < cptr[node + 1]; ++t) {
      int j = node_dof[cidx[t]];
      int lo = 0, hi = ns_sup - 1, k = -1;
      while (lo <= hi) {
        int mid_ = (lo + hi) >> 1;
        if (sup[mid_] == j) {
          k = mid_;
          break;
        }
        if (sup[mid_] < j)
          lo = mid_ + 1;
        else
          hi = mid_ - 1;
      }
      if (k < 0) continue;
      size_t o2 = (size_t)w * MAXS + k;
      double sbv = Sb[o2], gb0 = Gb[3 * o2], gb1 = Gb[3 * o2 + 1], gb2 = Gb[3 * o2 + 2];
      double cwt = cw[t];
      wacc += cwt * (sbv * phv + sc * (gb0 * gr[0] + gb1 * gr[1] + gb2 * gr[2]));
      xacc[0] += cwt * wv * (sbv * gr[0] + sc * (H01 * gb1 + H02 * gb2));
      xacc[1] += cwt * wv * (sbv * gr[1] + sc * (H01 * gb0 + H12 * gb2));
      xacc[2] += cwt * wv * (sbv * gr[2] + sc * (H02 * gb0 + H12 * gb1));
    }
    atomicAdd(&wb[wi][q >> 3], wacc);
    for (int d = 0; d < 3; ++d) atomicAdd(&xb[wi][q >> 3][d], xacc[d]);
  }
  __syncwarp();
  // geometry chain: sub-box bounds -> box bounds -> (x, l)
  double lob[3] = {0, 0, 0}, hib[3] = {0, 0, 0};
  if (lane < nsub) {
    const ASub& o = sb[wi][lane];
    double ext[3], vol = 1.0;
    for (int d = 0; d < 3; ++d) {
      ext[d] = o.e[d] - o.a[d];
      vol *= ext[d];
    }
    double volb = wb[wi][lane] / vp_s[wi];
    double vpb = -wb[wi][lane] * vol / (vp_s[wi] * vp_s[wi]);
    for (int d = 0; d < 3; ++d) {
      double cb = xb[wi][lane][d] / (double)o.s;
      double other = ext[(d + 1) % 3] * ext[(d + 2) % 3];
      double ab = 0.5 * cb - volb * other, eb = 0.5 * cb + volb * other;
      if (o.lo_dep[d]) lob[d] += ab;
      if (o.hi_dep[d]) hib[d] += eb;
      // V_p = prod (hi - lo), unclipped
      double vo = (hi_s[wi][(d + 1) % 3] - lo_s[wi][(d + 1) % 3]) * (hi_s[wi][(d + 2) % 3] - lo_s[wi][(d + 2) % 3]);
      hib[d] += vpb * vo;
      lob[d] -= vpb * vo;
    }
  }
  for (int d = 0; d < 3; ++d) {
    lob[d] = warp_sum(lob[d]);
    hib[d] = warp_sum(hib[d]);
  }
  if (lane == 0)
    for (int d = 0; d < 3; ++d) {
      atomicAdd(mid.x + 3 * p + d, g.scale * (lob[d] + hib[d]));
      atomicAdd(mid.lp + 3 * p + d, g.scale * (hib[d] - lob[d]));
    }
}

// ---------------------------------------------------------------- split fold

// children of each split parent (child 0 in the parent's slot, children 1..7
// at P + 7 rank + c - 1): sum their adjoints into the parent
__global__ void k_adj_split(int P, const int* __restrict__ flag, const int* __restrict__ rank, Adj a) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P || !flag[p]) return;
  double x[3] = {0, 0, 0}, l[3] = {0, 0, 0}, F[9] = {0}, be[6] = {0}, E = 0.0, ys = 0.0;
  for (int c = 0; c < 8; ++c) {
    size_t q = c == 0 ? (size_t)p : (size_t)P + 7 * (size_t)rank[p] + (c - 1);
    for (int d = 0; d < 3; ++d) {
      double sg = ((c >> d) & 1) ? 0.5 : -0.5;
      x[d] += a.x[3 * q + d];
      l[d] += sg * a.x[3 * q + d] + 0.5 * a.lp[3 * q + d];
    }
    for (int i = 0; i < 9; ++i) F[i] += a.F[9 * q + i];
    for (int i = 0; i < 6; ++i) be[i] += a.be[6 * q + i];
    E += a.E[q];
    ys += a.ys[q];
  }
  for (int d = 0; d < 3; ++d) {
    a.x[3 * (size_t)p + d] = x[d];
    a.lp[3 * (size_t)p + d] = l[d];
  }
  for (int i = 0; i < 9; ++i) a.F[9 * (size_t)p + i] = F[i];
  for (int i = 0; i < 6; ++i) a.be[6 * (size_t)p + i] = be[i];
  a.E[p] = E;
  a.ys[p] = ys;
}

__global__ void k_mask_vec(int nd, const int* __restrict__ mask, double* v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  for (int c = 0; c < 3; ++c)
    if ((mask[i] >> c) & 1) v[3 * (size_t)i + c] = 0.0;
}

__global__ void k_fill_int(int n, int* a, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

}  // namespace
}  // namespace mpm

using namespace mpm;

namespace mpm {
namespace {

// device memory of one adjoint call, released on every exit path
struct AdjointScratch {
  mpm_ctx* c;
  Buf work[9], adj[6], mid[4], sg[2], vec[4], argk;
  mpm_mesh* m = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  explicit AdjointScratch(mpm_ctx* ctx) : c(ctx) {}
  ~AdjointScratch() {
    for (Buf* set : {work, adj, mid})
      for (int i = 0; i < (set == work ? 9 : (set == adj ? 6 : 4)); ++i) free_buf(c, set[i]);
    for (auto& b : sg) free_buf(c, b);
    for (auto& b : vec) free_buf(c, b);
    free_buf(c, argk);
    if (m) {
      mesh_release(m);
      delete m;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  float lap() {
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    return t;
  }
};

}  // namespace
}  // namespace mpm

extern "C" int mpm_adjoint(mpm_ctx* c, const mpm_domain* dom, const mpm_rigid* body,
                           const mpm_adapt* ad, const mpm_material* mat, const mpm_checkpoint* ck,
                           int nsteps, const mpm_step_params* prm, const double* dJ_dreaction,
                           double* dJ_dE, double* dJ_dys, mpm_adjoint_stats* stats) {
  if (!c || !dom || !ad || !mat || !ck || nsteps <= 0 || !prm || !dJ_dreaction || !dJ_dE || !dJ_dys)
    return MPM_ERR_ARG;
  if (mat->model != 0 && mat->model != 1) {
    set_error(c, "adjoint: supports the Hencky elastic and von Mises models (symmetric tangent)");
    return MPM_ERR_ARG;
  }
  if (mat->mu > 0.0 && mat->contact_on) {
    set_error(c, "adjoint: frictional contact (mu > 0) has a non-symmetric tangent; not supported");
    return MPM_ERR_ARG;
  }
  if (body && (body->kind == 3 || body->kind == 4 || body->free)) {
    set_error(c, "adjoint: the prescribed analytic bodies (kinds 1, 2) only");
    return MPM_ERR_ARG;
  }
  if (prm->dt != 0.0) {
    set_error(c, "adjoint: quasi-static load steps only (dt = 0)");
    return MPM_ERR_ARG;
  }
  if (!(prm->tol > 0) || prm->maxit < 0 || prm->maxit > 63) {
    set_error(c, "adjoint: need tol > 0 and 0 <= maxit <= 63");
    return MPM_ERR_ARG;
  }
  mpm_adjoint_stats stt{};
  int status = MPM_OK;
  try {
    AdjointScratch X(c);
    cudaStream_t st = c->stream;
    MPM_CUDA(cudaEventCreate(&X.e0));
    MPM_CUDA(cudaEventCreate(&X.e1));
    int cap = 0;
    for (int n = 0; n < nsteps; ++n) {
      const mpm_points& q = ck[n].pts;
      if (q.count <= 0 || q.capacity < q.count || !q.x || !q.lp || !q.l0 || !q.F || !q.be || !q.V0 ||
          !q.mass || !q.E || !q.ys)
        throw CudaError(MPM_ERR_ARG, "adjoint: checkpoint " + std::to_string(n) + " is not a valid point set");
      cap = std::max(cap, q.capacity);
    }
    int P0 = ck[0].pts.count;
    // working points (the checkpoint is copied, then split in place)
    mpm_points W{};
    W.capacity = cap;
    double** wp[9] = {&W.x, &W.lp, &W.l0, &W.F, &W.be, &W.V0, &W.mass, &W.E, &W.ys};
    const int wd[9] = {3, 3, 3, 9, 6, 1, 1, 1, 1};
    for (int i = 0; i < 9; ++i) *wp[i] = grow<double>(c, X.work[i], (size_t)wd[i] * cap);
    // adjoint of the point state (caller order), and of the state before the
    // point update (E and ys are carried unchanged, so they share one array)
    const int aw[6] = {3, 3, 9, 6, 1, 1};
    double* ap[6];
    for (int i = 0; i < 6; ++i) {
      ap[i] = grow<double>(c, X.adj[i], (size_t)aw[i] * cap);
      MPM_CUDA(cudaMemsetAsync(ap[i], 0, sizeof(double) * aw[i] * cap, st));
    }
    Adj A{ap[0], ap[1], ap[2], ap[3], ap[4], ap[5]};
    Adj Mid{grow<double>(c, X.mid[0], 3 * (size_t)cap), grow<double>(c, X.mid[1], 3 * (size_t)cap),
            grow<double>(c, X.mid[2], 9 * (size_t)cap), grow<double>(c, X.mid[3], 6 * (size_t)cap), A.E,
            A.ys};
    X.m = new mpm_mesh();
    X.m->ctx = c;
    X.m->record_splits = true;
    mpm_mesh* m = X.m;
    Law L = make_law(*mat);
    mpm_rigid nob{};
    for (int n = nsteps - 1; n >= 0; --n) {
      const mpm_checkpoint& k = ck[n];
      // 1. restore, rebuild (same events), re-solve
      MPM_CUDA(cudaEventRecord(X.e0, st));
      W.count = k.pts.count;
      const double* src[9] = {k.pts.x, k.pts.lp, k.pts.l0, k.pts.F, k.pts.be, k.pts.V0, k.pts.mass, k.pts.E, k.pts.ys};
      for (int i = 0; i < 9; ++i)
        MPM_CUDA(cudaMemcpyAsync(*wp[i], src[i], sizeof(double) * wd[i] * W.count,
                                 cudaMemcpyDeviceToDevice, st));
      mpm_rigid bd = body ? *body : nob;
      bd.z = k.body_z;
      build_mesh(c, m, *dom, bd, *ad, *mat, &W, 0);
      int e = check_device_error(c, "adjoint: mesh build");
      if (e) throw CudaError(e, c->err);
      if (n + 1 < nsteps && m->np != ck[n + 1].pts.count)
        throw CudaError(MPM_ERR_ARG, "adjoint: step " + std::to_string(n) + " rebuilt " + std::to_string(m->np) +
                                         " points, the next checkpoint holds " + std::to_string(ck[n + 1].pts.count));
      const double* u = nullptr;
      if (k.du) {
        // the increment the forward stored: no second Newton solve
        if (k.du_len != 3LL * m->ndof)
          throw CudaError(MPM_ERR_ARG, "adjoint: checkpoint " + std::to_string(n) + " stores " +
                                           std::to_string(k.du_len) + " increments, the rebuilt step has " +
                                           std::to_string(3LL * m->ndof));
        u = k.du;
      } else {
        mpm_step_params sp = *prm;
        sp.load = k.load;
        sp.du_out = nullptr;
        mpm_step_stats ss{};
        double* un = nullptr;
        newton(c, m, mat, bd, &sp, ss, &un);
        u = un;
      }
      stt.ms_forward += X.lap();
      MPM_CUDA(cudaEventRecord(X.e0, st));
      // consistent FP64 tangent at the converged increment
      int P = m->np, nd = m->ndof, n3 = 3 * nd;
      double* R = grow<double>(c, X.vec[0], n3);
      double* ub = grow<double>(c, X.vec[1], n3);
      double* mu = grow<double>(c, X.vec[2], n3);
      double* K = grow<double>(c, X.vec[3], 9 * (size_t)m->nslot);
      AsmOut o{};
      assemble(c, m, *mat, bd, u, k.load, MPM_FP64, R, K, &o, true);
      if (n == nsteps - 1)
        for (int d = 0; d < 3; ++d) stt.reaction[d] = o.reaction[d];
      double* Sb = grow<double>(c, X.sg[0], (size_t)P * MAXS);
      double* Gb = grow<double>(c, X.sg[1], (size_t)P * MAXS * 3);
      MPM_CUDA(cudaMemsetAsync(ub, 0, sizeof(double) * n3, st));
      MPM_CUDA(cudaMemsetAsync(Sb, 0, sizeof(double) * (size_t)P * MAXS, st));
      MPM_CUDA(cudaMemsetAsync(Gb, 0, sizeof(double) * (size_t)P * MAXS * 3, st));
      // 2. seeds: the point update, and the reaction at the last step
      MPM_LAUNCH(k_adj_update<<<grid_for(P, 128), 128, 0, st>>>(
          P, L, ptr<int>(m->perm), ptr<int>(m->nsup), ptr<int>(m->sidx), ptr<double>(m->S),
          ptr<double>(m->dS), u, ptr<double>(m->pE), ptr<double>(m->pys), ptr<double>(m->pbe),
          ptr<double>(m->pF), ptr<double>(m->pl0), A, Mid, Sb, Gb, ub, c->d_err));
      MeshView mv{m->g, ptr<double>(m->px), ptr<double>(m->plp), ptr<uint64_t>(m->leaf_key),
                  ptr<int>(m->leaf_lev), m->nleaf, ptr<int>(m->corner), ptr<int>(m->cptr),
                  ptr<int>(m->cidx), ptr<double>(m->cw), ptr<int>(m->node_dof)};
      bool contact = m->ncand && mat->contact_on && bd.kind != 0;
      if (n == nsteps - 1 && contact)
        MPM_LAUNCH(k_adj_contact<<<grid_for(8LL * m->ncand, 128), 128, 0, st>>>(
            8 * m->ncand, 1, ptr<int>(m->cand), mv, ptr<int>(m->perm), ptr<double>(m->pE),
            ptr<double>(m->pV0), body_view(m, bd), mat->pf, u, nullptr, dJ_dreaction[0], dJ_dreaction[1],
            dJ_dreaction[2], ub, Mid, A));
      MPM_LAUNCH(k_mask_vec<<<grid_for(nd, 256), 256, 0, st>>>(nd, ptr<int>(m->dof_mask), ub));
      // 3. K mu = seed (K symmetric)
      // FP64 PCG, multigrid-preconditioned when the forward used method 3
      mpm_solve_params lp{prm->lin.method == 3 ? 3 : 1, MPM_FP64, prm->lin.tol, prm->lin.maxit, 0.0,
                          prm->lin.mg_reuse};
      mpm_solve_stats ls{};
      solve(c, m, *mat, K, ub, mu, lp, &ls);
      stt.lin_its += ls.iterations;
      e = check_device_error(c, "adjoint: linear solve");
      if (e) throw CudaError(e, c->err);
      if (ls.status) throw CudaError(ls.status, "adjoint: linear solve did not converge");
      MPM_LAUNCH(k_mask_vec<<<grid_for(nd, 256), 256, 0, st>>>(nd, ptr<int>(m->dof_mask), mu));
      // 4. backward of -mu^T R(u; state, E, ys)
      MPM_LAUNCH(k_adj_residual<<<grid_for(P, 128), 128, 0, st>>>(
          P, L, k.load, mat->g[0], mat->g[1], mat->g[2], ptr<int>(m->perm), ptr<int>(m->nsup),
          ptr<int>(m->sidx), ptr<double>(m->dS), u, mu, ptr<double>(m->pE), ptr<double>(m->pys),
          ptr<double>(m->pbe), ptr<double>(m->pV0), ptr<double>(m->pmass), Mid, A, Sb, Gb, c->d_err));
      if (contact)
        MPM_LAUNCH(k_adj_contact<<<grid_for(8LL * m->ncand, 128), 128, 0, st>>>(
            8 * m->ncand, 0, ptr<int>(m->cand), mv, ptr<int>(m->perm), ptr<double>(m->pE),
            ptr<double>(m->pV0), body_view(m, bd), mat->pf, u, mu, 0.0, 0.0, 0.0, nullptr, Mid, A));
      int* argK = grow<int>(c, X.argk, m->nleaf);
      MPM_LAUNCH(k_fill_int<<<grid_for(m->nleaf, 256), 256, 0, st>>>(m->nleaf, argK, 0x7fffffff));
      MPM_LAUNCH(k_adj_basis<<<grid_for(P, AW), 32 * AW, 0, st>>>(
          P, m->g, ptr<int>(m->perm), ptr<double>(m->px), ptr<double>(m->plp), ptr<double>(m->pE),
          ptr<double>(m->betaK), ptr<uint64_t>(m->leaf_key), ptr<int>(m->leaf_lev), m->nleaf,
          ptr<int>(m->corner), ptr<int>(m->cptr), ptr<int>(m->cidx), ptr<double>(m->cw),
          ptr<int>(m->node_dof), ptr<int>(m->nsup), ptr<int>(m->sidx), Sb, Gb, Mid, argK, c->d_err));
      if (m->nghost && mat->ghost_on)
        MPM_LAUNCH(k_adj_ghost<<<grid_for(m->nghost, 64), 64, 0, st>>>(
            m->nghost, m->g, mat->kappa, ptr<int>(m->gface), ptr<uint64_t>(m->leaf_key),
            ptr<int>(m->leaf_lev), ptr<double>(m->betaK), argK, ptr<int>(m->gdof), ptr<int>(m->gn),
            ptr<int>(m->corner), ptr<int>(m->cptr), ptr<int>(m->cidx), ptr<double>(m->cw),
            ptr<int>(m->node_dof), u, mu, A.E));
      // 5. adjoint of the state at the start of the step: fold split children
      MPM_CUDA(cudaMemcpyAsync(A.x, Mid.x, sizeof(double) * 3 * P, cudaMemcpyDeviceToDevice, st));
      MPM_CUDA(cudaMemcpyAsync(A.lp, Mid.lp, sizeof(double) * 3 * P, cudaMemcpyDeviceToDevice, st));
      MPM_CUDA(cudaMemcpyAsync(A.F, Mid.F, sizeof(double) * 9 * P, cudaMemcpyDeviceToDevice, st));
      MPM_CUDA(cudaMemcpyAsync(A.be, Mid.be, sizeof(double) * 6 * P, cudaMemcpyDeviceToDevice, st));
      for (int r = (int)m->split_log.size() - 1; r >= 0; --r) {
        const SplitRound& sr = m->split_log[r];
        MPM_LAUNCH(k_adj_split<<<grid_for(sr.P, 128), 128, 0, st>>>(sr.P, ptr<int>(sr.flag),
                                                                    ptr<int>(sr.rank), A));
      }
      e = check_device_error(c, "adjoint: backward kernels");
      if (e) throw CudaError(e, c->err);
      stt.ms_backward += X.lap();
    }
    MPM_CUDA(cudaMemcpyAsync(dJ_dE, A.E, sizeof(double) * P0, cudaMemcpyDeviceToDevice, st));
    MPM_CUDA(cudaMemcpyAsync(dJ_dys, A.ys, sizeof(double) * P0, cudaMemcpyDeviceToDevice, st));
    MPM_CUDA(cudaStreamSynchronize(st));
  } catch (const CudaError& e) {
    set_error(c, e.what());
    status = e.code;
  } catch (const std::exception& e) {
    set_error(c, e.what());
    status = MPM_ERR_ARG;
  }
  stt.status = status;
  if (stats) *stats = stt;
  return status;
}
