// Per-Newton-iteration assembly of Eq. (MPMweak) (static part): point
// kinematics, the Hencky / return-map constitutive update with its consistent
// spatial tangent (Sec. 2.2), the internal force, the tangent gathered row by
// row into the 3x3 block matrix, the ghost term (Sec. 4), the penalty contact
// (Sec. 2.3) and the strong Dirichlet rows (Sec. 2.4).
#include <algorithm>

#include "mpm_internal.cuh"
#include "mpm_law.cuh"

namespace mpm {
namespace {

// ------------------------------------------------------------------ kinematics

// dF = I + sum_v du_v (x) grad S_vp; eight lanes per point, four points per warp
__global__ void k_kinematics(int P, const int* __restrict__ nsup, const int* __restrict__ sidx,
                             const double* __restrict__ dS, const double* __restrict__ du,
                             double* dF) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int w = (int)(t >> 3), sub = (int)(t & 7);
  double a[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) a[i] = 0.0;
  if (w < P) {
    int n = nsup[w];
    for (int k = sub; k < n; k += 8) {
      size_t o = (size_t)w * MAXS + k;
      int j = sidx[o];
      double u0 = du[3 * (size_t)j], u1 = du[3 * (size_t)j + 1], u2 = du[3 * (size_t)j + 2];
      double g0 = dS[3 * o], g1 = dS[3 * o + 1], g2 = dS[3 * o + 2];
      a[0] += u0 * g0; a[1] += u0 * g1; a[2] += u0 * g2;
      a[3] += u1 * g0; a[4] += u1 * g1; a[5] += u1 * g2;
      a[6] += u2 * g0; a[7] += u2 * g1; a[8] += u2 * g2;
    }
  }
  // reduce-scatter of a[0..7] over the 8 lanes of the point (lane sub ends
  // with the sum of a[sub]: 7 FP64 additions instead of 24; the FP64 pipe
  // bounds this kernel), a[8] by a butterfly
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    bool up = sub & 4;
    double send = up ? a[i] : a[i + 4];
    double keep = up ? a[i + 4] : a[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    bool up = sub & 2;
    double send = up ? a[i] : a[i + 2];
    double keep = up ? a[i + 2] : a[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  {
    bool up = sub & 1;
    double send = up ? a[0] : a[1];
    double keep = up ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
  a[8] += __shfl_xor_sync(0xffffffffu, a[8], 4);
  a[8] += __shfl_xor_sync(0xffffffffu, a[8], 2);
  a[8] += __shfl_xor_sync(0xffffffffu, a[8], 1);
  if (w < P) {
    dF[9 * (size_t)w + sub] = a[0] + ((sub % 4 == 0) ? 1.0 : 0.0);
    if (sub == 0) dF[9 * (size_t)w + 8] = a[8] + 1.0;
  }
}

// ------------------------------------------------------------------ constitutive

// Full per-point update.  in: dF, b_e,n (6); out: tau (6: xx yy zz xy yz xz),
// b_e (6), A' (81, layout [(i*9 + k*3 + m)*3 + j] = A_ijkm - tau_im delta_jk)
// The consistent spatial tangent from the spectral state: theta_ab =
// (tau_a - tau_b)/(lam_a - lam_b) = g/2 * divided difference of ln (in FP64),
// then the eigenbasis rotation of the 81 entries in the precision the tangent
// is stored in (FP32 for the mixed path, where it runs on the FP32 pipe).
// Layout [(i*9 + k*3 + m)*3 + j] = A_ijkm - tau_im delta_jk.
template <class TA>
__device__ void tangent_rotate(const double* Q, const double* lam, const double* dd, double gr,
                               const double* tau6, TA* Aout) {
  // theta_ab = (tau_a - tau_b)/(lam_a - lam_b) = g/2 * divided difference of ln
  // (in FP64), then the eigenbasis rotation of the 81 entries in the
  // precision the tangent is stored in: FP32 for the mixed path, where it
  // runs on the FP32 pipe
  typedef TA R;
  double th01 = 0.5 * gr * ln_divdiff(lam[0], lam[1]);
  double th02 = 0.5 * gr * ln_divdiff(lam[0], lam[2]);
  double th12 = 0.5 * gr * ln_divdiff(lam[1], lam[2]);
  R th[9] = {(R)0, (R)th01, (R)th02, (R)th01, (R)0, (R)th12, (R)th02, (R)th12, (R)0};
  R q[9], d[9], lr[3];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    q[i] = (R)Q[i];
    d[i] = (R)dd[i];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) lr[a] = (R)lam[a];
  R taum[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      int s = (i == j) ? i : (i + j == 1 ? 3 : (i + j == 3 ? 4 : 5));
      taum[3 * i + j] = (R)tau6[s];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m) {
          R s = (R)0;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            R qia = q[3 * i + a];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              s += d[3 * a + c] * qia * q[3 * j + a] * q[3 * k + c] * q[3 * m + c];
              if (a != c)
                s += th[3 * a + c] * qia * q[3 * j + c] *
                     (lr[c] * q[3 * k + a] * q[3 * m + c] + lr[a] * q[3 * k + c] * q[3 * m + a]);
            }
          }
          if (j == k) s -= taum[3 * i + m];
          Aout[(i * 9 + k * 3 + m) * 3 + j] = s;
        }
}

template <bool TANGENT, class TA>
__device__ bool point_update_law(const Law& L, double E, double ys, const double* be, const double* dF,
                                 double* tau6, double* be_new, TA* Aout, double* save = nullptr) {
  double b[9] = {be[0], be[3], be[5], be[3], be[1], be[4], be[5], be[4], be[2]};
  double t[9], bt[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      t[3 * i + j] = dF[3 * i] * b[j] + dF[3 * i + 1] * b[3 + j] + dF[3 * i + 2] * b[6 + j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      bt[3 * i + j] = t[3 * i] * dF[3 * j] + t[3 * i + 1] * dF[3 * j + 1] + t[3 * i + 2] * dF[3 * j + 2];
  // symmetrise before the rotations
  bt[1] = bt[3] = 0.5 * (bt[1] + bt[3]);
  bt[2] = bt[6] = 0.5 * (bt[2] + bt[6]);
  bt[5] = bt[7] = 0.5 * (bt[5] + bt[7]);
  double lam[3], Q[9];
  jacobi3(bt, lam, Q);
  if (!(lam[0] > 0.0 && lam[1] > 0.0 && lam[2] > 0.0) || !isfinite(lam[0] + lam[1] + lam[2]))
    return false;
  double eps[3] = {0.5 * log(lam[0]), 0.5 * log(lam[1]), 0.5 * log(lam[2])};
  double ta[3], dd[9], gr;
  principal_return(L, E, ys, eps, ta, dd, &gr);
  double mu = E / (2.0 * (1.0 + L.nu));
  double lm = E * L.nu / ((1.0 + L.nu) * (1.0 - 2.0 * L.nu));
  double tt = ta[0] + ta[1] + ta[2];
  double bw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) bw[a] = exp(2.0 * (ta[a] - lm * tt / (3.0 * lm + 2.0 * mu)) / (2.0 * mu));
  // tau = Q diag(ta) Q^T, b_e = Q diag(bw) Q^T
  const int ii[6] = {0, 1, 2, 0, 1, 0}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    int i = ii[s], j = jj[s];
    tau6[s] = Q[3 * i] * ta[0] * Q[3 * j] + Q[3 * i + 1] * ta[1] * Q[3 * j + 1] + Q[3 * i + 2] * ta[2] * Q[3 * j + 2];
    be_new[s] = Q[3 * i] * bw[0] * Q[3 * j] + Q[3 * i + 1] * bw[1] * Q[3 * j + 1] + Q[3 * i + 2] * bw[2] * Q[3 * j + 2];
  }
  if (TANGENT) tangent_rotate<TA>(Q, lam, dd, gr, tau6, Aout);
  if (save) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      save[i] = Q[i];
      save[12 + i] = dd[i];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) save[9 + a] = lam[a];
    save[21] = gr;
  }
  return true;
}

__device__ inline double det3(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}

// also M = V0 tau dF^-T (row-major, 12 per point, the last 3 unused), so that
// the internal force of support k is M grad S_k (k_residual_rows)
template <bool TANGENT, class TA>
__global__ void k_constitutive(int P, Law L, const double* __restrict__ E, const double* __restrict__ ys,
                               const double* __restrict__ be, const double* __restrict__ dF,
                               const double* __restrict__ V0, double* tau, double* dFinv,
                               double* Mf, TA* Aalg, double* lawst, int* err) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  double f[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = dF[9 * (size_t)w + i];
  double det = det3(f);
  double t6[6], bn[6];
  bool ok = det > 0.0 && isfinite(det) &&
            point_update_law<TANGENT, TA>(L, E[w], ys[w], be + 6 * (size_t)w, f, t6, bn,
                                          Aalg + 81 * (size_t)w,
                                          lawst ? lawst + 22 * (size_t)w : nullptr);
  if (!ok) {
    atomicOr(err, EB_NAN);
#pragma unroll
    for (int s = 0; s < 6; ++s) t6[s] = 0.0;
    det = 1.0;
  }
#pragma unroll
  for (int s = 0; s < 6; ++s) tau[6 * (size_t)w + s] = t6[s];
  double id = 1.0 / det;
  double* o = dFinv + 9 * (size_t)w;
  o[0] = (f[4] * f[8] - f[5] * f[7]) * id;
  o[1] = (f[2] * f[7] - f[1] * f[8]) * id;
  o[2] = (f[1] * f[5] - f[2] * f[4]) * id;
  o[3] = (f[5] * f[6] - f[3] * f[8]) * id;
  o[4] = (f[0] * f[8] - f[2] * f[6]) * id;
  o[5] = (f[2] * f[3] - f[0] * f[5]) * id;
  o[6] = (f[3] * f[7] - f[4] * f[6]) * id;
  o[7] = (f[1] * f[6] - f[0] * f[7]) * id;
  o[8] = (f[0] * f[4] - f[1] * f[3]) * id;
  // M_il = V0 sum_j tau_ij (dF^-1)_lj
  double fi[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) fi[e] = o[e];
  double tm[9] = {t6[0], t6[3], t6[5], t6[3], t6[1], t6[4], t6[5], t6[4], t6[2]};
  double v0 = V0[w];
  double* M = Mf + 12 * (size_t)w;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      M[3 * i + l] = v0 * (tm[3 * i] * fi[3 * l] + tm[3 * i + 1] * fi[3 * l + 1] + tm[3 * i + 2] * fi[3 * l + 2]);
}

// the tangent of the state the last residual evaluation left (same increment):
// no second eigen-decomposition or return map
template <class TA>
__global__ void k_tangent_state(int P, const double* __restrict__ lawst, const double* __restrict__ tau,
                                TA* Aalg) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  const double* st = lawst + 22 * (size_t)w;
  double Q[9], lam[3], dd[9], t6[6];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    Q[i] = st[i];
    dd[i] = st[12 + i];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) lam[a] = st[9 + a];
#pragma unroll
  for (int i = 0; i < 6; ++i) t6[i] = tau[6 * (size_t)w + i];
  tangent_rotate<TA>(Q, lam, dd, st[21], t6, Aalg + 81 * (size_t)w);
}

// grad_x S = grad S . dF^{-1} for the tangent gather (in its precision), without
// the internal force; also V0 in that precision, so that the gather converts
// nothing.  A conversion from FP64 occupies the FP64 pipe (2 lanes per clock
// per SM on this part) as long as an FMA, for a whole warp instruction: dF^-1
// is converted one entry per lane and shared by shuffles, and the FP32 path
// reads grad S from its FP32 copy (TS = float), made once per mesh build.
template <class TG, class TS>
__global__ void k_gx(int P, const int* __restrict__ nsup, const TS* __restrict__ dS,
                     const double* __restrict__ dFinv, const double* __restrict__ V0, TG* gx,
                     TG* V0t) {
  int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= P) return;
  TG mine = lane < 9 ? (TG)dFinv[9 * (size_t)w + lane] : lane == 9 ? (TG)V0[w] : (TG)0;
  TG fi[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fi[i] = __shfl_sync(0xffffffffu, mine, i);
  if (lane == 9) V0t[w] = mine;
  int n = nsup[w];
  for (int k = lane; k < n; k += 32) {
    size_t o = (size_t)w * MAXS + k;
    TG a0 = (TG)dS[3 * o], a1 = (TG)dS[3 * o + 1], a2 = (TG)dS[3 * o + 2];
    gx[3 * o] = a0 * fi[0] + a1 * fi[3] + a2 * fi[6];
    gx[3 * o + 1] = a0 * fi[1] + a1 * fi[4] + a2 * fi[7];
    gx[3 * o + 2] = a0 * fi[2] + a1 * fi[5] + a2 * fi[8];
  }
}

// the FP32 copy of the basis gradients (the used slots of every point)
__global__ void k_dS_to_float(int P, const int* __restrict__ nsup, const double* __restrict__ dS,
                              float* dS32) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int w = (int)(t / (3 * MAXS)), e = (int)(t - (long long)w * 3 * MAXS);
  if (w >= P || e >= 3 * nsup[w]) return;
  dS32[t] = (float)dS[t];
}

// ------------------------------------------------------------------ internal force and residual

// R = f_int - load f_ext + K_G du, one warp per row r, where f_int,r is the sum
// over the point sources (p, k) of the row (the pattern's sorted source keys)
// of M_p grad S_pk, M_p = V0 tau dF^-T from k_constitutive.  A fixed-order
// gather: every lane sums a fixed set of sources in key order and the lanes
// are combined by a fixed shuffle tree, so f_int and R are the same bit for
// bit on every run (no floating-point atomics).
__global__ void k_residual_rows(int nd, int P, double load, const long long* __restrict__ sptr,
                                const uint64_t* __restrict__ skeys, const double* __restrict__ M,
                                const double* __restrict__ dS, const int* __restrict__ rp,
                                const int* __restrict__ col, const double* __restrict__ kg,
                                const double* __restrict__ du, const double* __restrict__ fext,
                                double* fint, double* R) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nd) return;
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  long long q1 = sptr[r + 1];
  for (long long q = sptr[r] + lane; q < q1; q += 32) {
    uint32_t sid = (uint32_t)skeys[q];
    int w = (int)(sid >> 6), k = (int)(sid & 63);
    if (w >= P) continue;  // ghost-face source
    const double2* m = reinterpret_cast<const double2*>(M + 12 * (size_t)w);
    double2 m01 = m[0], m23 = m[1], m45 = m[2], m67 = m[3], m8x = m[4];
    const double* a = dS + 3 * ((size_t)w * MAXS + k);
    double a0 = a[0], a1 = a[1], a2 = a[2];
    f0 += m01.x * a0 + m01.y * a1 + m23.x * a2;
    f1 += m23.y * a0 + m45.x * a1 + m45.y * a2;
    f2 += m67.x * a0 + m67.y * a1 + m8x.x * a2;
  }
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int s = rp[r] + lane; s < rp[r + 1]; s += 32) {
    double k = kg[s];
    if (k != 0.0) {
      int c = col[s];
      g0 += k * du[3 * (size_t)c];
      g1 += k * du[3 * (size_t)c + 1];
      g2 += k * du[3 * (size_t)c + 2];
    }
  }
  f0 = warp_sum(f0);
  f1 = warp_sum(f1);
  f2 = warp_sum(f2);
  g0 = warp_sum(g0);
  g1 = warp_sum(g1);
  g2 = warp_sum(g2);
  if (lane < 3) {
    double f = lane == 0 ? f0 : (lane == 1 ? f1 : f2);
    double g = lane == 0 ? g0 : (lane == 1 ? g1 : g2);
    size_t i = 3 * (size_t)r + lane;
    fint[i] = f;
    R[i] = f - load * fext[i] + g;
  }
}

// ------------------------------------------------------------------ tangent (row gather)

constexpr int TW = 4;  // warps per block of the tangent gather (at most)

// open-addressing table of a row's columns (dof -> position in the row), in
// shared memory: a power of two at least twice the longest row
__host__ __device__ inline int tangent_hash_size(int mr) {
  int h = 64;
  while (h < 2 * mr) h <<= 1;
  return h;
}

// a block's 9 accumulators, padded to a 16-byte multiple so that one column
// is read and written with vector accesses: 12 floats or 10 doubles
template <class T>
__host__ __device__ constexpr int tangent_acc_stride() {
  return sizeof(T) == 4 ? 12 : 10;
}

// shared memory of one warp: the row's accumulators, the 32 terms of the
// current source, then the row's column table
template <class T>
__host__ __device__ inline size_t tangent_warp_bytes(int mr) {
  return (size_t)mr * tangent_acc_stride<T>() * sizeof(T) + 32 * sizeof(T) +
         (size_t)tangent_hash_size(mr) * 2 * sizeof(int);
}

__device__ inline unsigned tangent_hash(int c, int hmask) {
  return ((unsigned)c * 2654435761u >> 7) & (unsigned)hmask;
}

// the 27 terms (grad_x S_k)^T A'_p of a source from shared memory (16-byte
// aligned, 32 entries) in vector loads
__device__ inline void tangent_terms(const float* Tt, float* t) {
  const float4* v = reinterpret_cast<const float4*>(Tt);
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    float4 a = v[i];
    t[4 * i] = a.x;
    if (4 * i + 1 < 27) t[4 * i + 1] = a.y;
    if (4 * i + 2 < 27) t[4 * i + 2] = a.z;
    if (4 * i + 3 < 27) t[4 * i + 3] = a.w;
  }
}
__device__ inline void tangent_terms(const double* Tt, double* t) {
  const double2* v = reinterpret_cast<const double2*>(Tt);
#pragma unroll
  for (int i = 0; i < 14; ++i) {
    double2 a = v[i];
    t[2 * i] = a.x;
    if (2 * i + 1 < 27) t[2 * i + 1] = a.y;
  }
}

// acc[0..8] += the block t (x) g of one (source, column) pair, with vector
// shared-memory accesses
__device__ inline void tangent_add(float* a, const float* t, float g0, float g1, float g2) {
  float4* v = reinterpret_cast<float4*>(a);
  float4 x = v[0], y = v[1];
  float z = a[8];
  x.x += t[0] * g0 + t[1] * g1 + t[2] * g2;
  x.y += t[3] * g0 + t[4] * g1 + t[5] * g2;
  x.z += t[6] * g0 + t[7] * g1 + t[8] * g2;
  x.w += t[9] * g0 + t[10] * g1 + t[11] * g2;
  y.x += t[12] * g0 + t[13] * g1 + t[14] * g2;
  y.y += t[15] * g0 + t[16] * g1 + t[17] * g2;
  y.z += t[18] * g0 + t[19] * g1 + t[20] * g2;
  y.w += t[21] * g0 + t[22] * g1 + t[23] * g2;
  z += t[24] * g0 + t[25] * g1 + t[26] * g2;
  v[0] = x;
  v[1] = y;
  a[8] = z;
}
__device__ inline void tangent_add(double* a, const double* t, double g0, double g1, double g2) {
  double2* v = reinterpret_cast<double2*>(a);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double2 x = v[i];
    x.x += t[6 * i] * g0 + t[6 * i + 1] * g1 + t[6 * i + 2] * g2;
    x.y += t[6 * i + 3] * g0 + t[6 * i + 4] * g1 + t[6 * i + 5] * g2;
    v[i] = x;
  }
  a[8] += t[24] * g0 + t[25] * g1 + t[26] * g2;
}

// the loads of one source (point w, local index k) of a row, issued together:
// lane l holds the l-th column of the point's support and its grad_x S, lanes
// < 27 the three A'_p values of one of the 27 terms
template <class T>
struct TangentSrc {
  int w, n, c;
  T v0, gk0, gk1, gk2, a0, a1, a2, g0, g1, g2;
};

template <class T>
__device__ inline void tangent_fetch(TangentSrc<T>& s, uint32_t sid, int P, int lane,
                                     const int* __restrict__ nsup, const int* __restrict__ sidx,
                                     const T* __restrict__ gx, const T* __restrict__ Aalg,
                                     const T* __restrict__ V0) {
  int w = (int)(sid >> 6), k = (int)(sid & 63);
  s.w = w < P ? w : -1;  // w >= P: a ghost-face source, no point tangent
  if (s.w < 0) return;
  size_t ok = ((size_t)w * MAXS + k) * 3;
  s.gk0 = gx[ok];
  s.gk1 = gx[ok + 1];
  s.gk2 = gx[ok + 2];
  s.v0 = V0[w];
  s.n = nsup[w];
  if (lane < 27) {
    const T* A = Aalg + 81 * (size_t)w + 3 * lane;
    s.a0 = A[0];
    s.a1 = A[1];
    s.a2 = A[2];
  }
  // lane < 32 <= MAXS: inside the point's slot range whatever its support size
  size_t o = (size_t)w * MAXS + lane;
  s.c = sidx[o];
  s.g0 = gx[3 * o];
  s.g1 = gx[3 * o + 1];
  s.g2 = gx[3 * o + 2];
}

// one (source, column) pair: its column's place in the row, then the block
template <class T, bool UPPER>
__device__ inline void tangent_pair(T* acc, const int* hkey, const int* hval, int hmask, int r, int c,
                                    const T* t, T g0, T g1, T g2) {
  constexpr int AS = tangent_acc_stride<T>();
  if (UPPER && c < r) return;
  unsigned h = tangent_hash(c, hmask);
  int key;
  while ((key = hkey[h]) != c && key != -1) h = (h + 1) & hmask;
  if (key != c) return;
  tangent_add(acc + AS * hval[h], t, g0, g1, g2);
}

// One warp owns block row r: for every point p with r in its support (local
// index k), K_{r,w} += V0_p (grad_x S_k)^T A'_p (grad_x S_w) for all w in the
// support of p.  The row accumulates in shared memory (mr = longest row, a
// multiple of 4), in source order, free of atomics and deterministic; the
// position of a column in the row comes from a per-row hash table.  Ghost coefficients and the
// Dirichlet identity rows/columns are applied when the row is written out,
// coalesced, in the sliced layout.
// UPPER (a symmetric tangent: Hencky, von Mises, frictionless contact): only
// the blocks of columns c >= r are formed and written, about half the work;
// k_tangent_mirror then copies each into its transposed place.
template <class T, bool UPPER>
__global__ void __launch_bounds__(32 * TW)
    k_tangent_rows(int nd, int P, int minlen, int mr, int last, const int* __restrict__ rp,
                   const int* __restrict__ col,
                   Sliced S, const long long* __restrict__ sptr, const uint64_t* __restrict__ skeys,
                   const int* __restrict__ nsup, const int* __restrict__ sidx,
                   const T* __restrict__ gx, const T* __restrict__ Aalg,
                   const T* __restrict__ V0, const double* __restrict__ kg,
                   const int* __restrict__ mask, T* K, int* err) {
  constexpr int AS = tangent_acc_stride<T>();
  extern __shared__ __align__(16) unsigned char smraw[];
  int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* acc = (T*)(smraw + wi * tangent_warp_bytes<T>(mr));
  T* Tt = acc + AS * (size_t)mr;
  int* hkey = (int*)(Tt + 32);
  int hs = tangent_hash_size(mr), hmask = hs - 1;
  int* hval = hkey + hs;
  int r = blockIdx.x * (blockDim.x >> 5) + wi;
  if (r >= nd) return;
  int s0 = rp[r], nb = rp[r + 1] - s0;
  if (nb <= minlen) return;  // done by the pass for shorter rows
  if (nb > mr) {
    // left to the pass for longer rows; an error only in the last pass
    if (lane == 0 && last) atomicOr(err, EB_ROW);
    return;
  }
  for (int i = lane; i < hs; i += 32) hkey[i] = -1;
  for (int i = lane; i < AS * nb; i += 32) acc[i] = (T)0;
  __syncwarp();
  for (int i = lane; i < nb; i += 32) {
    int c = col[s0 + i];
    unsigned h = tangent_hash(c, hmask);
    while (atomicCAS(hkey + h, -1, c) != -1) h = (h + 1) & hmask;
    hval[h] = i;
  }
  __syncwarp();
  // the row's source keys 32 at a time (one coalesced load, then broadcast)
  const unsigned FULL = 0xffffffffu;
  long long q0 = sptr[r], q1 = sptr[r + 1];
  for (long long qb = q0; qb < q1; qb += 32) {
    int cnt = (int)min(32LL, q1 - qb);
    uint32_t kb = lane < cnt ? (uint32_t)skeys[qb + lane] : 0u;
    for (int u = 0; u < cnt; ++u) {
      TangentSrc<T> s;
      tangent_fetch(s, __shfl_sync(FULL, kb, u), P, lane, nsup, sidx, gx, Aalg, V0);
      if (s.w < 0) continue;  // the same for every lane
      if (lane < 27) Tt[lane] = s.v0 * (s.gk0 * s.a0 + s.gk1 * s.a1 + s.gk2 * s.a2);
      __syncwarp();
      T t[27];
      tangent_terms(Tt, t);
      if (lane < s.n) tangent_pair<T, UPPER>(acc, hkey, hval, hmask, r, s.c, t, s.g0, s.g1, s.g2);
      // supports of more than 32 nodes (deep hanging chains)
      for (int l = lane + 32; l < s.n; l += 32) {
        size_t o = (size_t)s.w * MAXS + l;
        tangent_pair<T, UPPER>(acc, hkey, hval, hmask, r, sidx[o], t, gx[3 * o], gx[3 * o + 1], gx[3 * o + 2]);
      }
      __syncwarp();
    }
  }
  // ghost, then the Dirichlet identity, then the row (and its padding slots,
  // zero) into the sliced storage
  int mr_ = mask[r];
  int sr = S.pos[r], sl = sr >> 5, W = S.w[sl];
  long long b0 = S.base[sl];
  for (int i = lane; i < W; i += 32) {
    long long slot = sliced_slot(b0, sr, i);
    if (i >= nb) {
#pragma unroll
      for (int e = 0; e < 9; ++e) K[sliced_entry(b0, W, slot, e)] = (T)0;
      continue;
    }
    // the ghost coefficient is zero away from the cut cells: convert only
    // where some lane of the warp has one
    double kd = kg[s0 + i];
    T kv = __any_sync(__activemask(), kd != 0.0) ? (T)kd : (T)0;
    int c = col[s0 + i];
    if (UPPER && c < r) continue;  // written by k_tangent_mirror
    int mc = mask[c];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        int e = 3 * a + b;
        T v = acc[AS * i + e];
        if (a == b) v += kv;
        if (((mr_ >> a) & 1) || ((mc >> b) & 1)) v = (c == r && a == b) ? (T)1 : (T)0;
        K[sliced_entry(b0, W, slot, e)] = v;
      }
  }
}

// the lower blocks of a symmetric tangent: block (r, c), c < r, is the
// transpose of block (c, r), found by binary search in row c (one warp per row)
template <class T>
__global__ void k_tangent_mirror(int nd, const int* __restrict__ rp, const int* __restrict__ col,
                                 Sliced S, T* K) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int r = (int)(t >> 5), lane = (int)(t & 31);
  if (r >= nd) return;
  int s0 = rp[r], nb = rp[r + 1] - s0;
  int sr = S.pos[r], sl = sr >> 5, W = S.w[sl];
  long long b0 = S.base[sl];
  for (int i = lane; i < nb; i += 32) {
    int c = col[s0 + i];
    if (c >= r) break;  // columns sorted: the rest is the upper part
    int lo = rp[c], hi = rp[c + 1] - 1, j = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1, v = col[mid];
      if (v == r) {
        j = mid;
        break;
      }
      if (v < r)
        lo = mid + 1;
      else
        hi = mid - 1;
    }
    if (j < 0) continue;  // (the pattern is symmetric: never)
    int src = S.pos[c], slc = src >> 5, Wc = S.w[slc];
    long long bc = S.base[slc], sc = sliced_slot(bc, src, j - rp[c]);
    T v[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) v[e] = K[sliced_entry(bc, Wc, sc, e)];
    long long slot = sliced_slot(b0, sr, i);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) K[sliced_entry(b0, W, slot, 3 * a + b)] = v[3 * b + a];
  }
}

// rows beyond ndof in the last slice (stored in place): zero padding slots
template <class T>
__global__ void k_zero_pad_rows(int nd, int npad, Sliced S, T* K) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int r = nd + (int)(t >> 5), lane = (int)(t & 31);
  if (r >= npad) return;
  int sl = r >> 5, W = S.w[sl];
  long long b0 = S.base[sl];
  for (int i = lane; i < W; i += 32) {
    long long slot = sliced_slot(b0, r, i);
    for (int e = 0; e < 9; ++e) K[sliced_entry(b0, W, slot, e)] = (T)0;
  }
}

// sliced values -> plain [nnzb][3][3] blocks (FP64)
template <class T>
__global__ void k_blocks_export(int nd, const int* __restrict__ rp, Sliced S, const T* __restrict__ K,
                                double* out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int r = (int)(t >> 5), lane = (int)(t & 31);
  if (r >= nd) return;
  int sr = S.pos[r], sl = sr >> 5, W = S.w[sl];
  long long b0 = S.base[sl];
  for (int i = lane; i < rp[r + 1] - rp[r]; i += 32) {
    long long slot = sliced_slot(b0, sr, i);
    for (int e = 0; e < 9; ++e) out[9 * (size_t)(rp[r] + i) + e] = (double)K[sliced_entry(b0, W, slot, e)];
  }
}

// ------------------------------------------------------------------ contact (Sec. 2.3)

__device__ inline int find_slot(const int* __restrict__ rp, const int* __restrict__ col, int r, int c) {
  int lo = rp[r], hi = rp[r + 1] - 1;
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

// [a]x, the matrix of b -> a x b (row-major)
__device__ inline void cross_mat(const double* a, double* C) {
  C[0] = 0.0;
  C[1] = -a[2];
  C[2] = a[1];
  C[3] = a[2];
  C[4] = 0.0;
  C[5] = -a[0];
  C[6] = -a[1];
  C[7] = a[0];
  C[8] = 0.0;
}

__device__ inline void mul33(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// one thread per candidate domain corner: the gap against the body at the moved
// corner; in contact the force on the material f (normal f_N n with
// f_N = -eps_N phi, plus Coulomb friction) and k_c = -d f / d y are stored for
// the row gather below (zeros and on = 0 otherwise), and with `reac` the
// force on the body, -sum f, is summed in a fixed order (every thread of the
// grid takes part).  The body sits at its given pose moved by bi.shift; the
// friction measures the node's slip against the body's own displacement at
// the node, qt + qr x d (d = y - X, X the body's reference point); with
// `ct` the derivative of f in the body's rotation ([d]x through the slip) and
// d are stored per corner for the body's equations.
__global__ void k_contact_corner(int nc8, const int* __restrict__ cand, const int* __restrict__ cb_n,
                                 const int* __restrict__ cb_idx, const double* __restrict__ cb_phi,
                                 const double* __restrict__ cb_y0, const double* __restrict__ pE,
                                 const double* __restrict__ pV0, Body body, double L, double pf,
                                 double pt, double mu, BodyInc bi,
                                 const double* __restrict__ du, double* cf, double* ck, int* con,
                                 double* ct, double* cdv, double* reac, GridRed gr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double f[3] = {0.0, 0.0, 0.0};
  if (i < nc8) {
    int w = cand[i >> 3], n = cb_n[i];
    const int* ids = cb_idx + (size_t)i * MAXCB;
    const double* ph = cb_phi + (size_t)i * MAXCB;
    double y[3] = {cb_y0[3 * (size_t)i], cb_y0[3 * (size_t)i + 1], cb_y0[3 * (size_t)i + 2]};
    for (int e = 0; e < n; ++e)
      for (int d = 0; d < 3; ++d) y[d] += ph[e] * du[3 * (size_t)ids[e] + d];
    double phi, nv[3], H[9], yb[3], dv[3];
    for (int d = 0; d < 3; ++d) yb[d] = y[d] - bi.shift[d];
    bool on = body_sdf(body, L, yb, &phi, nv, H) && phi < 0.0;
    dv[0] = y[0] - (body.b.cx + bi.shift[0]);
    dv[1] = y[1] - (body.b.cy + bi.shift[1]);
    dv[2] = y[2] - (body.b.z + bi.shift[2]);
    double Fy[9], Ft[9];
    for (int e = 0; e < 9; ++e) Fy[e] = Ft[e] = 0.0;
    if (on) {
      double A0 = pow(pV0[w], 2.0 / 3.0);
      double epsN = pf * pE[w] * A0, fN = -epsN * phi;
      for (int d = 0; d < 3; ++d) f[d] = fN * nv[d];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Fy[3 * a + b] = -epsN * (nv[a] * nv[b] + phi * H[3 * a + b]);
      if (mu > 0.0) {
        // Coulomb friction: the slip g = (y - y0) - (qt + qr x d) on the
        // tangent plane; trial force t = -eps_T (I - n n^T) g, stick while
        // |t| <= mu f_N, else slip with mu f_N t / |t|; Jd, Jg its
        // derivatives in d (through n, H, f_N) and in g
        double epsT = pt * pE[w] * A0;
        double g[3], t[3], Hg[3], Td[9], Tg[9], Jd[9], Jg[9];
        for (int d = 0; d < 3; ++d) {
          double rot = bi.qr[(d + 1) % 3] * dv[(d + 2) % 3] - bi.qr[(d + 2) % 3] * dv[(d + 1) % 3];
          g[d] = (y[d] - cb_y0[3 * (size_t)i + d]) - (bi.qt[d] + rot);
        }
        double ng = nv[0] * g[0] + nv[1] * g[1] + nv[2] * g[2];
        for (int a = 0; a < 3; ++a) Hg[a] = H[3 * a] * g[0] + H[3 * a + 1] * g[1] + H[3 * a + 2] * g[2];
        for (int d = 0; d < 3; ++d) t[d] = -epsT * (g[d] - nv[d] * ng);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            Td[3 * a + b] = epsT * (ng * H[3 * a + b] + nv[a] * Hg[b]);
            Tg[3 * a + b] = -epsT * ((a == b ? 1.0 : 0.0) - nv[a] * nv[b]);
          }
        double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (tn <= mu * fN) {
          for (int d = 0; d < 3; ++d) f[d] += t[d];
          for (int e = 0; e < 9; ++e) {
            Jd[e] = Td[e];
            Jg[e] = Tg[e];
          }
        } else {
          double u[3] = {t[0] / tn, t[1] / tn, t[2] / tn};
          for (int d = 0; d < 3; ++d) f[d] += mu * fN * u[d];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double sd = 0.0, sg = 0.0;
              for (int c = 0; c < 3; ++c) {
                double P = (a == c ? 1.0 : 0.0) - u[a] * u[c];
                sd += P * Td[3 * c + b];
                sg += P * Tg[3 * c + b];
              }
              Jd[3 * a + b] = mu * u[a] * (-epsN * nv[b]) + mu * fN * sd / tn;
              Jg[3 * a + b] = mu * fN * sg / tn;
            }
        }
        // d f / d y = N + Jd + Jg (I - [qr]x); d f / d qr = Jg [d]x
        double Qr[9], IQ[9], T[9], Dx[9];
        cross_mat(bi.qr, Qr);
        for (int e = 0; e < 9; ++e) IQ[e] = (e % 4 == 0 ? 1.0 : 0.0) - Qr[e];
        mul33(Jg, IQ, T);
        for (int e = 0; e < 9; ++e) Fy[e] += Jd[e] + T[e];
        cross_mat(dv, Dx);
        mul33(Jg, Dx, Ft);
      }
    }
    for (int d = 0; d < 3; ++d) cf[3 * (size_t)i + d] = f[d];
    for (int e = 0; e < 9; ++e) ck[9 * (size_t)i + e] = -Fy[e];
    con[i] = on ? 1 : 0;
    if (ct) {
      for (int e = 0; e < 9; ++e) ct[9 * (size_t)i + e] = Ft[e];
      for (int d = 0; d < 3; ++d) cdv[3 * (size_t)i + d] = dv[d];
    }
  }
  if (reac) {
    double v[3] = {-f[0], -f[1], -f[2]};
    double* o[3] = {reac, reac + 1, reac + 2};
    grid_sum<3>(v, o, gr);
  }
}

// The rigid body's sums over the contact corners, in a fixed order (one
// block; each thread takes the corners i = t, t + blockDim, ..., then the
// block's fixed tree): out[0..5] the residual terms f and d x f, out[6..41]
// their derivative in the body's increment q (row-major 6 x 6):
// [d f / d qt, d f / d qr; [f]x + [d]x d f / d qt, [d]x d f / d qr] with
// d f / d qt = -d f / d y
__global__ void k_body_sums(int nc8, const double* __restrict__ cf, const double* __restrict__ ck,
                            const double* __restrict__ ct, const double* __restrict__ cdv,
                            const int* __restrict__ con, double* out) {
  __shared__ double sh[32];
  double acc[42];
  for (int e = 0; e < 42; ++e) acc[e] = 0.0;
  for (int i = threadIdx.x; i < nc8; i += blockDim.x) {
    if (!con[i]) continue;
    const double* f = cf + 3 * (size_t)i;
    const double* d = cdv + 3 * (size_t)i;
    const double* Ft = ct + 9 * (size_t)i;
    double FX[9], Dx[9], Fx[9], DF[9], DT[9];
    for (int e = 0; e < 9; ++e) FX[e] = ck[9 * (size_t)i + e];  // -d f / d y
    cross_mat(d, Dx);
    cross_mat(f, Fx);
    mul33(Dx, FX, DF);
    mul33(Dx, Ft, DT);
    for (int a = 0; a < 3; ++a) {
      acc[a] += f[a];
      acc[3 + a] += d[(a + 1) % 3] * f[(a + 2) % 3] - d[(a + 2) % 3] * f[(a + 1) % 3];
      for (int b = 0; b < 3; ++b) {
        acc[6 + 6 * a + b] += FX[3 * a + b];
        acc[6 + 6 * a + 3 + b] += Ft[3 * a + b];
        acc[6 + 6 * (3 + a) + b] += Fx[3 * a + b] + DF[3 * a + b];
        acc[6 + 6 * (3 + a) + 3 + b] += DT[3 * a + b];
      }
    }
  }
  for (int e = 0; e < 42; ++e) {
    double v = block_sum(acc[e], sh);
    if (threadIdx.x == 0) out[e] = v;
  }
}

// the body's coupling columns and rows at the rows of the contact list (one
// warp per row, a lane per output value, the row's corner entries in list
// order): Kgb[j][3r + a] = d R_{r,a} / d q_j = sum phi (d f / d y)[a][j] for
// the translation (j < 3) and -sum phi (d f / d qr)[a][j - 3] for the
// rotation; Kbg[j][3r + b] = d Rb_j / d du_{r,b} = sum phi (d f / d y)[j][b]
// (j < 3) and sum phi ([d]x d f / d y - [f]x)[j - 3][b]
__global__ void k_body_rows(int nrow, const int* __restrict__ crow, const int* __restrict__ cptr,
                            const int* __restrict__ cent, const double* __restrict__ cb_phi,
                            const double* __restrict__ cf, const double* __restrict__ ck,
                            const double* __restrict__ ct, const double* __restrict__ cdv,
                            const int* __restrict__ con, long long n3, double* Kgb, double* Kbg) {
  int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= nrow) return;
  int r = crow[t], e0 = cptr[t], e1 = cptr[t + 1];
  for (int o = lane; o < 36; o += 32) {
    // o < 18: Kgb, component a = o / 6 of row r, body column j = o % 6;
    // o >= 18: Kbg, body row j = (o - 18) / 3, component b = (o - 18) % 3
    bool gb = o < 18;
    int a = gb ? o / 6 : (o - 18) % 3, j = gb ? o % 6 : (o - 18) / 3;
    double s = 0.0;
    for (int e = e0; e < e1; ++e) {
      int pk = cent[e], i = pk >> 5;
      if (!con[i]) continue;
      double ph = cb_phi[(size_t)i * MAXCB + (pk & 31)];
      const double* Fm = ck + 9 * (size_t)i;  // -d f / d y
      double v;
      if (gb) {
        v = j < 3 ? -Fm[3 * a + j] : -ct[9 * (size_t)i + 3 * a + (j - 3)];
      } else if (j < 3) {
        v = -Fm[3 * j + a];
      } else {
        const double* d = cdv + 3 * (size_t)i;
        const double* f = cf + 3 * (size_t)i;
        int jr = j - 3, j1 = (jr + 1) % 3, j2 = (jr + 2) % 3;
        // ([d]x (d f / d y))[jr][a] - ([f]x)[jr][a]
        double dF = -(d[j1] * Fm[3 * j2 + a] - d[j2] * Fm[3 * j1 + a]);
        double fx = (a == j2 ? f[j1] : 0.0) - (a == j1 ? f[j2] : 0.0);
        v = dF - fx;
      }
      s += ph * v;
    }
    if (gb)
      Kgb[(size_t)j * n3 + 3 * (size_t)r + a] = s;
    else
      Kbg[(size_t)j * n3 + 3 * (size_t)r + a] = s;
  }
}

// Newmark inertia of each point (time steps): m_p a_p with
// a_p = (2 / dt^2) (sum_v S_vp du_v - dt v_p)
__global__ void k_point_inertia(int P, const int* __restrict__ nsup, const int* __restrict__ sidx,
                                const double* __restrict__ S, const double* __restrict__ du,
                                const double* __restrict__ v, const double* __restrict__ mass,
                                double dt, double* ma) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  double u[3] = {0.0, 0.0, 0.0};
  int n = nsup[w];
  for (int k = 0; k < n; ++k) {
    size_t o = (size_t)w * MAXS + k;
    int j = sidx[o];
    for (int d = 0; d < 3; ++d) u[d] += S[o] * du[3 * (size_t)j + d];
  }
  double c2 = 2.0 / (dt * dt);
  for (int d = 0; d < 3; ++d) ma[3 * (size_t)w + d] = mass[w] * (c2 * (u[d] - dt * v[3 * (size_t)w + d]));
}

// the inertia term of Eq. (MPMweak), sum_p S_vp m_p a_p, gathered per row over
// the row's point sources (warp per row): added to R and stored in finert
__global__ void k_inertia_rows(int nd, int P, const long long* __restrict__ sptr,
                               const uint64_t* __restrict__ skeys, const double* __restrict__ S,
                               const double* __restrict__ ma, double* R, double* finert) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nd) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long q = sptr[r] + lane; q < sptr[r + 1]; q += 32) {
    uint32_t sid = (uint32_t)skeys[q];
    int w = (int)(sid >> 6), k = (int)(sid & 63);
    if (w >= P) continue;  // ghost-face source
    double sv = S[(size_t)w * MAXS + k];
    a0 += sv * ma[3 * (size_t)w];
    a1 += sv * ma[3 * (size_t)w + 1];
    a2 += sv * ma[3 * (size_t)w + 2];
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if (lane < 3) {
    double a = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
    R[3 * (size_t)r + lane] += a;
    finert[3 * (size_t)r + lane] = a;
  }
}

// the consistent mass of a time step, (2 / dt^2) m_p S_vp S_wp I, added to the
// tangent's diagonal entries: one warp per row r, the row's point sources in
// key order, the lanes over the source point's support (distinct columns),
// the Dirichlet components skipped
template <class T>
__global__ void k_mass_rows(int nd, int P, const long long* __restrict__ sptr,
                            const uint64_t* __restrict__ skeys, const int* __restrict__ nsup,
                            const int* __restrict__ sidx, const double* __restrict__ S,
                            const double* __restrict__ mass, double c2, const int* __restrict__ rp,
                            const int* __restrict__ col, Sliced SL, const int* __restrict__ mask, T* K) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= nd) return;
  int s0r = rp[r], ma = mask[r];
  int srr = SL.pos[r], slc = srr >> 5, W = SL.w[slc];
  long long b0 = SL.base[slc];
  for (long long q = sptr[r]; q < sptr[r + 1]; ++q) {
    uint32_t sid = (uint32_t)skeys[q];
    int w = (int)(sid >> 6), k = (int)(sid & 63);
    if (w >= P) continue;
    double sk = c2 * mass[w] * S[(size_t)w * MAXS + k];
    int n = nsup[w];
    for (int l = lane; l < n; l += 32) {
      size_t o = (size_t)w * MAXS + l;
      int cb = sidx[o];
      int sl = find_slot(rp, col, r, cb);
      if (sl < 0) continue;
      long long slot = sliced_slot(b0, srr, sl - s0r);
      int mb = mask[cb];
      double v = sk * S[o];
      for (int a = 0; a < 3; ++a) {
        if (((ma >> a) & 1) || ((mb >> a) & 1)) continue;
        T* kv = K + sliced_entry(b0, W, slot, 4 * a);
        *kv += (T)v;
      }
    }
    __syncwarp();
  }
}

// One warp per row r of the contact list (the rows that the background basis
// of some candidate corner touches; entries (corner, basis entry) in sorted
// order).  RES: R_r -= sum of phi_e f and f_c,r += the same sum, lanes strided
// over the entries and combined by the fixed shuffle tree.  TANGENT: K_{r,b}
// += phi_e phi_b k_c over the basis entries b of each corner, one corner entry
// at a time in list order (the lanes of one entry write distinct columns), the
// Dirichlet components skipped.  No atomics: the same sums on every run.
template <class T, bool RES, bool TANGENT>
__global__ void k_contact_rows(int nrow, const int* __restrict__ crow, const int* __restrict__ cptr,
                               const int* __restrict__ cent, const int* __restrict__ cb_n,
                               const int* __restrict__ cb_idx, const double* __restrict__ cb_phi,
                               const double* __restrict__ cf, const double* __restrict__ ck,
                               const int* __restrict__ con, double* R, double* fc,
                               const int* __restrict__ rp, const int* __restrict__ col, Sliced S,
                               const int* __restrict__ mask, T* K) {
  int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= nrow) return;
  int r = crow[t], e0 = cptr[t], e1 = cptr[t + 1];
  if (RES) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) {
      int pk = cent[e], i = pk >> 5;
      double ph = cb_phi[(size_t)i * MAXCB + (pk & 31)];
      s0 += ph * cf[3 * (size_t)i];
      s1 += ph * cf[3 * (size_t)i + 1];
      s2 += ph * cf[3 * (size_t)i + 2];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane < 3) {
      double v = lane == 0 ? s0 : (lane == 1 ? s1 : s2);
      R[3 * (size_t)r + lane] -= v;
      fc[3 * (size_t)r + lane] += v;
    }
  }
  if (!TANGENT) return;
  int s0r = rp[r], ma = mask[r];
  int srr = S.pos[r], slc = srr >> 5, W = S.w[slc];
  long long b0 = S.base[slc];
  for (int e = e0; e < e1; ++e) {
    int pk = cent[e], i = pk >> 5;
    if (!con[i]) continue;
    const double* kc = ck + 9 * (size_t)i;
    double pa = cb_phi[(size_t)i * MAXCB + (pk & 31)];
    int n = cb_n[i];
    for (int eb = lane; eb < n; eb += 32) {
      int cb = cb_idx[(size_t)i * MAXCB + eb];
      int sl = find_slot(rp, col, r, cb);
      if (sl < 0) continue;
      long long slot = sliced_slot(b0, srr, sl - s0r);
      int mb = mask[cb];
      double pp = pa * cb_phi[(size_t)i * MAXCB + eb];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          if (((ma >> a) & 1) || ((mb >> b) & 1)) continue;
          T* kv = K + sliced_entry(b0, W, slot, 3 * a + b);
          *kv += (T)(pp * kc[3 * a + b]);
        }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ norms

// slots: 0 ||R_free||^2, 1 ||f_int||^2, 2 ||load f_ext + f_c||^2, 3
// ||f_inert||^2 (time steps) (fixed-order grid sums: the norms, and so
// Newton's convergence test and line search, are the same on every run)
__global__ void k_norms(int n3, const double* __restrict__ R, const double* __restrict__ fint,
                        const double* __restrict__ fext, const double* __restrict__ fc, double load,
                        const double* __restrict__ finert, const int* __restrict__ mask, double* out,
                        GridRed gr) {
  double a = 0.0, b = 0.0, c = 0.0, e2 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    if (!((mask[i / 3] >> (i % 3)) & 1)) a += R[i] * R[i];
    if (fint) b += fint[i] * fint[i];
    if (fext) {
      double e = load * fext[i] + (fc ? fc[i] : 0.0);
      c += e * e;
    }
    if (finert) e2 += finert[i] * finert[i];
  }
  double v[4] = {a, b, c, e2};
  double* o[4] = {out, out + 1, out + 2, out + 3};
  grid_sum<4>(v, o, gr);
}

}  // namespace


double norm_free(mpm_ctx* c, const mpm_mesh* m, const double* R) {
  double* slot = c->d_red + 16;
  MPM_CUDA(cudaMemsetAsync(slot, 0, 4 * sizeof(double), c->stream));
  MPM_LAUNCH(k_norms<<<4 * 152, 256, 0, c->stream>>>(3 * m->ndof, R, nullptr, nullptr, nullptr, 0.0,
                                          nullptr, ptr<int>(m->dof_mask), slot, grid_red(c, 4, 4 * 152)));
  MPM_CUDA(cudaMemcpyAsync(c->h_red + 16, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  return sqrt(c->h_red[16]);
}

namespace {

// the penalty contact of one assembly: per-corner forces and stiffness (and
// the reaction when `reac` is given), then the row gather; with a free body
// (dyn->body) also the body's sums (bsum, device [42]: k_body_sums) and, with
// the tangent, the coupling blocks
template <class T, bool RES, bool TANGENT>
void contact_terms(mpm_ctx* c, mpm_mesh* m, const mpm_material& mat, const mpm_rigid& body,
                   const double* du, double* R, double* fc, double* reac, T* K, const Dyn* dyn,
                   double* bsum) {
  cudaStream_t st = c->stream;
  int n8 = 8 * m->ncand;
  double* cf = grow<double>(c, m->cc_f, 3 * (size_t)n8);
  double* ck = grow<double>(c, m->cc_k, 9 * (size_t)n8);
  int* con = grow<int>(c, m->cc_on, n8);
  bool couple = dyn && dyn->body;
  double* ct = couple ? grow<double>(c, m->cc_t, 9 * (size_t)n8) : nullptr;
  double* cdv = couple ? grow<double>(c, m->cc_d, 3 * (size_t)n8) : nullptr;
  BodyInc bi{};
  for (int d = 0; d < 3; ++d) {
    bi.qt[d] = dyn ? dyn->q[d] : body.step_d[d];
    bi.qr[d] = dyn ? dyn->q[3 + d] : 0.0;
    bi.shift[d] = body.free ? bi.qt[d] : 0.0;
  }
  MPM_LAUNCH_P(MPM_PROF_CONTACT, k_contact_corner<<<grid_for(n8, 128), 128, 0, st>>>(
      n8, ptr<int>(m->cand), ptr<int>(m->cb_n), ptr<int>(m->cb_idx), ptr<double>(m->cb_phi),
      ptr<double>(m->cb_y0), ptr<double>(m->pE), ptr<double>(m->pV0), body_view(m, body), m->g.L,
      mat.pf, mat.pt, mat.mu, bi, du, cf, ck, con, ct, cdv, reac,
      grid_red(c, 3, grid_for(n8, 128))));
  if (couple && bsum)
    MPM_LAUNCH_P(MPM_PROF_CONTACT, k_body_sums<<<1, 256, 0, st>>>(n8, cf, ck, ct, cdv, con, bsum));
  if (!m->nct) return;
  Sliced S = sliced_view(m);
  MPM_LAUNCH_P(MPM_PROF_CONTACT, k_contact_rows<T, RES, TANGENT><<<grid_for(m->nct, 4), 128, 0, st>>>(
      m->nct, ptr<int>(m->ct_row), ptr<int>(m->ct_ptr), ptr<int>(m->ct_ent), ptr<int>(m->cb_n),
      ptr<int>(m->cb_idx), ptr<double>(m->cb_phi), cf, ck, con, R, fc, ptr<int>(m->row_ptr),
      ptr<int>(m->col), S, ptr<int>(m->dof_mask), K));
  if (TANGENT && couple && dyn->Kgb && dyn->Kbg)
    MPM_LAUNCH_P(MPM_PROF_CONTACT, k_body_rows<<<grid_for(m->nct, 4), 128, 0, st>>>(
        m->nct, ptr<int>(m->ct_row), ptr<int>(m->ct_ptr), ptr<int>(m->ct_ent),
        ptr<double>(m->cb_phi), cf, ck, ct, cdv, con, 3LL * m->ndof, dyn->Kgb, dyn->Kbg));
}

}  // namespace

namespace {

// one pass of the tangent gather (rows of lo < length <= hi blocks)
template <class T>
void tangent_launch(mpm_ctx* c, mpm_mesh* m, bool upper, int lo, int hi, int last, const void* gx,
                    const void* Aalg, const void* V0t, void* K) {
  cudaStream_t st = c->stream;
  int nd = m->ndof, P = m->np;
  size_t wb = tangent_warp_bytes<T>(hi);
  int tw = (int)std::min<size_t>(TW, (size_t)(220 * 1024) / wb);
  if (tw < 1) throw CudaError(MPM_ERR_SUPPORT, "stiffness row too long for the tangent gather");
  size_t smem = wb * tw;
  Sliced S = sliced_view(m);
  auto kern = upper ? k_tangent_rows<T, true> : k_tangent_rows<T, false>;
  MPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MPM_LAUNCH_P(MPM_PROF_TANGENT, kern<<<grid_for(nd, tw), 32 * tw, smem, st>>>(
      nd, P, lo, hi, last, ptr<int>(m->row_ptr), ptr<int>(m->col), S, ptr<long long>(m->src_ptr),
      ptr<uint64_t>(m->src_key), ptr<int>(m->nsup), ptr<int>(m->sidx), (const T*)gx, (const T*)Aalg,
      (const T*)V0t, ptr<double>(m->kg), ptr<int>(m->dof_mask), (T*)K, c->d_err));
}

}  // namespace

namespace {

// the free body's equations on the host from the contact sums (bsum, device
// [42]): Rb = m (2 / dt^2) (qt - dt v) - m load g + sum f,
// J (2 / dt^2) (qr - dt w) + sum d x f, and (with the tangent) Kbb = the
// sums' derivative plus the inertia's m (2 / dt^2) I, J (2 / dt^2) I
void body_out(mpm_ctx* c, const mpm_material& mat, const mpm_rigid& body, double load, const Dyn* dyn,
              const double* bsum, AsmOut* out, bool tangent) {
  double h[42];
  MPM_CUDA(cudaMemcpyAsync(h, bsum, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  double dt = dyn->dt, c2 = dt > 0.0 ? 2.0 / (dt * dt) : 0.0;
  for (int d = 0; d < 3; ++d) {
    out->Rb[d] = h[d];
    out->Rb[3 + d] = h[3 + d];
    if (dt > 0.0) {
      out->Rb[d] += body.mass * (c2 * (dyn->q[d] - dt * body.v[d]) - load * mat.g[d]);
      out->Rb[3 + d] += body.inertia * c2 * (dyn->q[3 + d] - dt * body.w[d]);
    }
  }
  if (!tangent) return;
  for (int e = 0; e < 36; ++e) out->Kbb[e] = h[6 + e];
  if (dt > 0.0)
    for (int d = 0; d < 3; ++d) {
      out->Kbb[7 * d] += body.mass * c2;
      out->Kbb[7 * (3 + d)] += body.inertia * c2;
    }
}

}  // namespace

void assemble(mpm_ctx* c, const mpm_mesh* mc, const mpm_material& mat, const mpm_rigid& body,
              const double* du, double load, int precision, double* R, void* K, AsmOut* out,
              bool want_norms, bool reuse, const Dyn* dyn) {
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  cudaStream_t st = c->stream;
  int P = m->np, nd = m->ndof;
  Law L = make_law(mat);
  double* dF = grow<double>(c, m->dF, 9 * (size_t)P);
  double* dFinv = grow<double>(c, m->dFinv, 9 * (size_t)P);
  double* tau = grow<double>(c, m->tau, 6 * (size_t)P);
  double* lawst = grow<double>(c, m->lawst, 22 * (size_t)P);
  double* Mf = grow<double>(c, m->Mf, 12 * (size_t)P);
  const int* nsup = ptr<int>(m->nsup);
  const int* sidx = ptr<int>(m->sidx);
  const double* dS = ptr<double>(m->dS);
  const double* V0 = ptr<double>(m->pV0);
  const int* rp = ptr<int>(m->row_ptr);
  const int* col = ptr<int>(m->col);
  Sliced S = sliced_view(m);
  bool mixed = precision == MPM_MIXED;
  size_t asz = mixed ? sizeof(float) : sizeof(double);
  void* Aalg = K ? grow_bytes(c, m->Aalg, 81 * (size_t)P * asz) : nullptr;
  void* gx = K ? grow_bytes(c, m->gx, 3 * (size_t)P * MAXS * asz) : nullptr;
  void* V0t = K ? grow_bytes(c, m->V0t, (size_t)P * asz) : nullptr;
  const float* dS32 = nullptr;
  if (K && mixed) {
    float* d32 = grow<float>(c, m->dS32, 3 * (size_t)P * MAXS);
    if (m->dS32_gen != m->gen) {
      MPM_LAUNCH_P(MPM_PROF_FORCE, k_dS_to_float<<<grid_for(3LL * MAXS * P, 256), 256, 0, st>>>(P, nsup, dS, d32));
      m->dS32_gen = m->gen;
    }
    dS32 = d32;
  }
  double* fint = grow<double>(c, c->v[0], 3 * (size_t)nd);
  double* fc = grow<double>(c, c->v[1], 3 * (size_t)nd);
  bool contact = m->ncand && mat.contact_on && body.kind != 0;
  bool inertia = dyn && dyn->dt > 0.0;
  if (inertia && !m->has_v) throw CudaError(MPM_ERR_ARG, "a time step needs point velocities");
  double* finert = inertia ? grow<double>(c, c->v[2], 3 * (size_t)nd) : nullptr;
  bool couple = dyn && dyn->body;
  double* bsum = couple ? grow<double>(c, m->cc_b, 42) : nullptr;
  if (couple) MPM_CUDA(cudaMemsetAsync(bsum, 0, 42 * sizeof(double), st));
  if (couple && K && dyn->Kgb && dyn->Kbg) {
    MPM_CUDA(cudaMemsetAsync(dyn->Kgb, 0, sizeof(double) * 18 * (size_t)nd, st));
    MPM_CUDA(cudaMemsetAsync(dyn->Kbg, 0, sizeof(double) * 18 * (size_t)nd, st));
  }
  // grid-sum partials for every reduction below, sized once; a clean ticket
  grid_red(c, 4, std::max(4096, grid_for(8LL * m->ncand, 128)));
  MPM_CUDA(cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), st));
  if (K && reuse) {
    // Newton's tangent at the increment of the last residual evaluation: its
    // dF, dF^-1, tau and spectral state are still in place, R is complete
    if (mixed) {
      MPM_LAUNCH_P(MPM_PROF_CONSTITUTIVE, k_tangent_state<float><<<grid_for(P, 128), 128, 0, st>>>(P, lawst, tau, (float*)Aalg));
      MPM_LAUNCH_P(MPM_PROF_FORCE, k_gx<float, float><<<grid_for(P, 8), 256, 0, st>>>(P, nsup, dS32, dFinv, V0, (float*)gx, (float*)V0t));
    } else {
      MPM_LAUNCH_P(MPM_PROF_CONSTITUTIVE, k_tangent_state<double><<<grid_for(P, 128), 128, 0, st>>>(P, lawst, tau, (double*)Aalg));
      MPM_LAUNCH_P(MPM_PROF_FORCE, k_gx<double, double><<<grid_for(P, 8), 256, 0, st>>>(P, nsup, dS, dFinv, V0, (double*)gx, (double*)V0t));
    }
  } else {
    MPM_LAUNCH_P(MPM_PROF_KINEMATICS, k_kinematics<<<grid_for(8LL * P, 256), 256, 0, st>>>(P, nsup, sidx, dS, du, dF));
    if (!K)
      MPM_LAUNCH_P(MPM_PROF_CONSTITUTIVE, k_constitutive<false, double><<<grid_for(P, 128), 128, 0, st>>>(
          P, L, ptr<double>(m->pE), ptr<double>(m->pys), ptr<double>(m->pbe), dF, V0, tau, dFinv, Mf,
          nullptr, lawst, c->d_err));
    else if (mixed)
      MPM_LAUNCH_P(MPM_PROF_CONSTITUTIVE, k_constitutive<true, float><<<grid_for(P, 128), 128, 0, st>>>(
          P, L, ptr<double>(m->pE), ptr<double>(m->pys), ptr<double>(m->pbe), dF, V0, tau, dFinv, Mf,
          (float*)Aalg, nullptr, c->d_err));
    else
      MPM_LAUNCH_P(MPM_PROF_CONSTITUTIVE, k_constitutive<true, double><<<grid_for(P, 128), 128, 0, st>>>(
          P, L, ptr<double>(m->pE), ptr<double>(m->pys), ptr<double>(m->pbe), dF, V0, tau, dFinv, Mf,
          (double*)Aalg, nullptr, c->d_err));
    MPM_CUDA(cudaMemsetAsync(fc, 0, sizeof(double) * 3 * nd, st));
    MPM_LAUNCH_P(MPM_PROF_RESIDUAL, k_residual_rows<<<grid_for(nd, 8), 256, 0, st>>>(
        nd, P, load, ptr<long long>(m->src_ptr), ptr<uint64_t>(m->src_key), Mf, dS, rp, col,
        ptr<double>(m->kg), du, ptr<double>(m->fext), fint, R));
    if (inertia) {
      double* ma = grow<double>(c, m->pma, 3 * (size_t)P);
      MPM_LAUNCH_P(MPM_PROF_RESIDUAL, k_point_inertia<<<grid_for(P, 128), 128, 0, st>>>(
          P, nsup, sidx, ptr<double>(m->S), du, ptr<double>(m->pv), ptr<double>(m->pmass), dyn->dt, ma));
      MPM_LAUNCH_P(MPM_PROF_RESIDUAL, k_inertia_rows<<<grid_for(nd, 8), 256, 0, st>>>(
          nd, P, ptr<long long>(m->src_ptr), ptr<uint64_t>(m->src_key), ptr<double>(m->S), ma, R, finert));
    }
    if (K) {
      if (mixed)
        MPM_LAUNCH_P(MPM_PROF_FORCE, k_gx<float, float><<<grid_for(P, 8), 256, 0, st>>>(P, nsup, dS32, dFinv, V0, (float*)gx, (float*)V0t));
      else
        MPM_LAUNCH_P(MPM_PROF_FORCE, k_gx<double, double><<<grid_for(P, 8), 256, 0, st>>>(P, nsup, dS, dFinv, V0, (double*)gx, (double*)V0t));
    }
  }
  if (K) {
    // two passes: rows up to 128 blocks (the 5^3 interior stencil and below)
    // with a small shared-memory footprint per warp, for occupancy, then the
    // longer rows near hanging nodes; a symmetric tangent forms only its upper
    // blocks and mirrors them
    // a symmetric FP64 tangent forms only its upper blocks and mirrors them:
    // its pairs are bound by the FP64 FMA rate, which the halving pays for
    // (about 5 ms of 108 per load step at the indentation workload); the FP32
    // gather is bound by its per-source loads and table lookups instead, and
    // the mirror pass would cost more than the halved pairs save
    bool upper = !mixed && (mat.model == 0 || mat.model == 1) && !(mat.mu > 0.0 && contact);
    int mr = (m->maxrow + 3) & ~3;
    const int SHORT = 128;
    int passes[2][2] = {{-1, std::min(mr, SHORT)}, {SHORT, mr}};
    int np_ = mr > SHORT ? 2 : 1;
    for (int ps = 0; ps < np_; ++ps) {
      int lo = passes[ps][0], hi = passes[ps][1], last = ps == np_ - 1;
      if (mixed)
        tangent_launch<float>(c, m, upper, lo, hi, last, gx, Aalg, V0t, K);
      else
        tangent_launch<double>(c, m, upper, lo, hi, last, gx, Aalg, V0t, K);
    }
    if (upper) {
      if (mixed)
        MPM_LAUNCH_P(MPM_PROF_TANGENT, k_tangent_mirror<float><<<grid_for(32LL * nd, 256), 256, 0, st>>>(nd, rp, col, S, (float*)K));
      else
        MPM_LAUNCH_P(MPM_PROF_TANGENT, k_tangent_mirror<double><<<grid_for(32LL * nd, 256), 256, 0, st>>>(nd, rp, col, S, (double*)K));
    }
    if (inertia) {
      double c2 = 2.0 / (dyn->dt * dyn->dt);
      if (mixed)
        MPM_LAUNCH_P(MPM_PROF_TANGENT, k_mass_rows<float><<<grid_for(nd, 4), 128, 0, st>>>(
            nd, P, ptr<long long>(m->src_ptr), ptr<uint64_t>(m->src_key), nsup, sidx, ptr<double>(m->S),
            ptr<double>(m->pmass), c2, rp, col, S, ptr<int>(m->dof_mask), (float*)K));
      else
        MPM_LAUNCH_P(MPM_PROF_TANGENT, k_mass_rows<double><<<grid_for(nd, 4), 128, 0, st>>>(
            nd, P, ptr<long long>(m->src_ptr), ptr<uint64_t>(m->src_key), nsup, sidx, ptr<double>(m->S),
            ptr<double>(m->pmass), c2, rp, col, S, ptr<int>(m->dof_mask), (double*)K));
    }
    int npad = 32 * m->nslice;
    if (npad > nd) {
      if (mixed)
        MPM_LAUNCH(k_zero_pad_rows<float><<<grid_for(32LL * (npad - nd), 256), 256, 0, st>>>(nd, npad, S, (float*)K));
      else
        MPM_LAUNCH(k_zero_pad_rows<double><<<grid_for(32LL * (npad - nd), 256), 256, 0, st>>>(nd, npad, S, (double*)K));
    }
  }
  double* reac = c->d_red + 20;
  if (K && reuse) {
    // contact stiffness only: its forces are already in R
    if (contact) {
      if (mixed)
        contact_terms<float, false, true>(c, m, mat, body, du, R, fc, nullptr, (float*)K, dyn, bsum);
      else
        contact_terms<double, false, true>(c, m, mat, body, du, R, fc, nullptr, (double*)K, dyn, bsum);
    }
    if (couple) body_out(c, mat, body, load, dyn, bsum, out, true);
    return;
  }
  MPM_CUDA(cudaMemsetAsync(reac, 0, 3 * sizeof(double), st));
  if (contact) {
    if (!K)
      contact_terms<double, true, false>(c, m, mat, body, du, R, fc, reac, (double*)nullptr, dyn, bsum);
    else if (mixed)
      contact_terms<float, true, true>(c, m, mat, body, du, R, fc, reac, (float*)K, dyn, bsum);
    else
      contact_terms<double, true, true>(c, m, mat, body, du, R, fc, reac, (double*)K, dyn, bsum);
  }
  if (want_norms) {
    double* slot = c->d_red + 16;
    MPM_CUDA(cudaMemsetAsync(slot, 0, 4 * sizeof(double), st));
    MPM_LAUNCH(k_norms<<<4 * 152, 256, 0, st>>>(3 * nd, R, fint, ptr<double>(m->fext), fc, load, finert,
                                     ptr<int>(m->dof_mask), slot, grid_red(c, 4, 4 * 152)));
    MPM_CUDA(cudaMemcpyAsync(c->h_red + 16, slot, 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    out->fint_norm = sqrt(c->h_red[17]);
    out->fextc_norm = sqrt(c->h_red[18]);
    out->finert_norm = sqrt(c->h_red[19]);
    for (int d = 0; d < 3; ++d) out->reaction[d] = c->h_red[20 + d];
  }
  if (couple) body_out(c, mat, body, load, dyn, bsum, out, K != nullptr);
}

void blocks_export(mpm_ctx* c, const mpm_mesh* m, const void* K, int precision, double* out) {
  Sliced S = sliced_view(m);
  int nd = m->ndof;
  if (precision == MPM_MIXED)
    MPM_LAUNCH(k_blocks_export<float><<<grid_for(32LL * nd, 256), 256, 0, c->stream>>>(nd, ptr<int>(m->row_ptr), S, (const float*)K, out));
  else
    MPM_LAUNCH(k_blocks_export<double><<<grid_for(32LL * nd, 256), 256, 0, c->stream>>>(nd, ptr<int>(m->row_ptr), S, (const double*)K, out));
}

// ------------------------------------------------------------------ point update helpers (used by mpm_step.cu)

namespace {

// end-of-step update, one thread per (sorted) point: x += sum S du, F <- dF F,
// b_e from the converged return, l = l0 diag(U), U = sqrt(F^T F)
__global__ void k_point_update(int P, Law L, const int* __restrict__ perm,
                               const int* __restrict__ nsup, const int* __restrict__ sidx,
                               const double* __restrict__ S, const double* __restrict__ dS,
                               const double* __restrict__ du, const double* __restrict__ pE,
                               const double* __restrict__ pys, const double* __restrict__ pbe,
                               const double* __restrict__ pF, const double* __restrict__ px,
                               const double* __restrict__ pl0, const double* __restrict__ pv,
                               double dt, mpm_points pts, int* err) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= P) return;
  double dF[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, dx[3] = {0, 0, 0};
  int n = nsup[w];
  for (int k = 0; k < n; ++k) {
    size_t o = (size_t)w * MAXS + k;
    int j = sidx[o];
    double u[3] = {du[3 * (size_t)j], du[3 * (size_t)j + 1], du[3 * (size_t)j + 2]};
    for (int i = 0; i < 3; ++i) {
      dx[i] += S[o] * u[i];
      for (int jj = 0; jj < 3; ++jj) dF[3 * i + jj] += u[i] * dS[3 * o + jj];
    }
  }
  double t6[6], bn[6];
  if (!point_update_law<false, double>(L, pE[w], pys[w], pbe + 6 * (size_t)w, dF, t6, bn, nullptr)) {
    atomicOr(err, EB_NAN);
    return;
  }
  const double* Fo = pF + 9 * (size_t)w;
  double Fn[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Fn[3 * i + j] = dF[3 * i] * Fo[j] + dF[3 * i + 1] * Fo[3 + j] + dF[3 * i + 2] * Fo[6 + j];
  double C[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = Fn[i] * Fn[j] + Fn[3 + i] * Fn[3 + j] + Fn[6 + i] * Fn[6 + j];
  double lam[3], Q[9];
  jacobi3(C, lam, Q);
  size_t p = perm[w];
  for (int d = 0; d < 3; ++d) {
    double u = 0.0;
    for (int a = 0; a < 3; ++a) u += sqrt(lam[a]) * Q[3 * d + a] * Q[3 * d + a];
    pts.x[3 * p + d] = px[3 * (size_t)w + d] + dx[d];
    pts.lp[3 * p + d] = pl0[3 * (size_t)w + d] * u;
    // a time step's velocity: v + dt a, a = (2 / dt^2) (du_p - dt v)
    if (dt > 0.0) {
      double v = pv[3 * (size_t)w + d];
      pts.v[3 * p + d] = v + dt * ((2.0 / (dt * dt)) * (dx[d] - dt * v));
    }
  }
  for (int i = 0; i < 9; ++i) pts.F[9 * p + i] = Fn[i];
  for (int s = 0; s < 6; ++s) pts.be[6 * p + s] = bn[s];
}

}  // namespace

void point_update(mpm_ctx* c, const mpm_mesh* mc, const mpm_material& mat, const double* du,
                  mpm_points* pts, double dt) {
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  int P = m->np;
  if (dt > 0.0 && !(m->has_v && pts->v)) throw CudaError(MPM_ERR_ARG, "a time step needs point velocities");
  MPM_LAUNCH(k_point_update<<<grid_for(P, 128), 128, 0, c->stream>>>(
      P, make_law(mat), ptr<int>(m->perm), ptr<int>(m->nsup), ptr<int>(m->sidx), ptr<double>(m->S),
      ptr<double>(m->dS), du, ptr<double>(m->pE), ptr<double>(m->pys), ptr<double>(m->pbe),
      ptr<double>(m->pF), ptr<double>(m->px), ptr<double>(m->pl0), dt > 0.0 ? ptr<double>(m->pv) : nullptr,
      dt, *pts, c->d_err));
}

}  // namespace mpm
