// Krylov solves of the linearised system K dx = -R (Sec. 2.4) with a 3x3
// block-Jacobi preconditioner (Sec. 1 names Krylov solvers with Jacobi-type
// preconditioning as the scalable alternative to the direct solver):
//  * PCG for symmetric tangents, two fused kernels per iteration, scalars kept
//    on the device in rotating slots, convergence decided on the device;
//  * BiCGStab (right preconditioned) for the non-symmetric Drucker-Prager
//    tangent;
//  * MPM_MIXED: FP32 matrix and FP32 inner solves inside FP64 iterative
//    refinement, the refinement residual accumulated in FP64.
#include <algorithm>
#include <atomic>
#include <vector>
#include <cmath>
#include <string>

#include "mpm_internal.cuh"
#include "mpm_sliced.cuh"

namespace mpm {
namespace {

constexpr int SW = 8;  // warps (slices of 32 rows) per block of the row kernels


// block-Jacobi: inverse of each 3x3 diagonal block, rows padded to 4 (12 per dof)
template <class T, class V>
__global__ void k_block_jacobi(int nd, const int* __restrict__ rp, const int* __restrict__ col,
                               Sliced S, const T* __restrict__ K, V* Dinv, int* err) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nd) return;
  int s0 = rp[r], nb = rp[r + 1] - s0, k = -1;
  int lo = 0, hi = nb - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int c = col[s0 + mid];
    if (c == r) {
      k = mid;
      break;
    }
    if (c < r)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  int sr = S.pos[r], sl = sr >> 5;
  long long b0 = S.base[sl], slot = k >= 0 ? sliced_slot(b0, sr, k) : 0;
  double a[9];
  for (int e = 0; e < 9; ++e)
    a[e] = k >= 0 ? (double)K[sliced_entry(b0, S.w[sl], slot, e)] : (double)(e % 4 == 0);
  double c0 = a[4] * a[8] - a[5] * a[7], c1 = a[5] * a[6] - a[3] * a[8], c2 = a[3] * a[7] - a[4] * a[6];
  double det = a[0] * c0 + a[1] * c1 + a[2] * c2;
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    atomicOr(err, EB_KRYLOV);
    det = 1.0;
  }
  double id = 1.0 / det;
  V* o = Dinv + 12 * (size_t)r;
  o[0] = (V)(c0 * id);
  o[1] = (V)((a[2] * a[7] - a[1] * a[8]) * id);
  o[2] = (V)((a[1] * a[5] - a[2] * a[4]) * id);
  o[3] = (V)0;
  o[4] = (V)(c1 * id);
  o[5] = (V)((a[0] * a[8] - a[2] * a[6]) * id);
  o[6] = (V)((a[2] * a[3] - a[0] * a[5]) * id);
  o[7] = (V)0;
  o[8] = (V)(c2 * id);
  o[9] = (V)((a[1] * a[6] - a[0] * a[7]) * id);
  o[10] = (V)((a[0] * a[4] - a[1] * a[3]) * id);
  o[11] = (V)0;
}


// ---------------------------------------------------------------- PCG
// vectors r, z, p, q are padded to 4 components over 32*nslice rows; x keeps
// the 3-component layout of the caller.

// setup: r = b (free components), x = 0, z = M r, p = z, rz_0, ||b||^2
template <class V>
__global__ void k_pcg_init(int nd, int npad, const double* __restrict__ b, const int* __restrict__ mask,
                           const V* __restrict__ Dinv, V* x, V* r, V* z, V* p, Scal* sc,
                           GridRed gr) {
  double rz = 0.0, bb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    V rv[4] = {(V)0, (V)0, (V)0, (V)0}, zv[4] = {(V)0, (V)0, (V)0, (V)0};
    if (i < nd) {
      int mk = mask[i];
      for (int c = 0; c < 3; ++c) {
        rv[c] = ((mk >> c) & 1) ? (V)0 : (V)b[3 * (size_t)i + c];
        x[3 * (size_t)i + c] = (V)0;
        bb += (double)rv[c] * (double)rv[c];
      }
      apply_dinv(Dinv, i, rv, zv);
      for (int c = 0; c < 3; ++c) rz += (double)rv[c] * (double)zv[c];
    }
    st4(r + 4 * (size_t)i, rv);
    st4(z + 4 * (size_t)i, zv);
    st4(p + 4 * (size_t)i, zv);
  }
  grid_sum2(rz, bb, &sc->rz[0], &sc->bb, gr);
}

// q = K p, pq_0 (one thread per row)
template <class T, class V>
__global__ void k_pcg_q0(int nd, int npad, Sliced S, const T* __restrict__ K, const V* __restrict__ p,
                         V* q, Scal* sc, GridRed gr) {
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  double part = 0.0;
  if (sr < npad) {
    int r = S.row[sr];
    V y[3];
    sliced_row<T, V, V, 4>(sr, S, K, p, y);
    V yv[4] = {y[0], y[1], y[2], (V)0};
    if (r >= nd) yv[0] = yv[1] = yv[2] = (V)0;
    st4(q + 4 * (size_t)r, yv);
    V pv[4];
    ld4(p + 4 * (size_t)r, pv);
    part = (double)yv[0] * pv[0] + (double)yv[1] * pv[1] + (double)yv[2] * pv[2];
  }
  grid_sum1(part, &sc->pq[0], gr);
}

// A_k: alpha = rz_k/pq_k; x += alpha p; r -= alpha q; z = M r; rz_{k+1}, rr_{k+1}
template <class V, bool PRE = true>
__global__ void k_pcg_a(int nd, int k, const V* __restrict__ Dinv, V* x, V* r, V* z,
                        const V* __restrict__ p, const V* __restrict__ q, Scal* sc, GridRed gr) {
  // early returns are taken by every block alike (scalars of earlier launches)
  if (sc->done) return;
  int i0 = k % 3, i1 = (k + 1) % 3;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->pq[i1] = 0.0;
  double pq = sc->pq[i0];
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->breakdown = 1;
      sc->done = 1;
      sc->iters = k;
    }
    return;
  }
  V alpha = (V)(sc->rz[i0] / pq);
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
    V pv[4], qv[4], rv[4], zv[4];
    ld4(p + 4 * (size_t)i, pv);
    ld4(q + 4 * (size_t)i, qv);
    ld4(r + 4 * (size_t)i, rv);
    for (int c = 0; c < 3; ++c) {
      x[3 * (size_t)i + c] += alpha * pv[c];
      rv[c] -= alpha * qv[c];
      rr += (double)rv[c] * (double)rv[c];
    }
    st4(r + 4 * (size_t)i, rv);
    if (PRE) {
      apply_dinv(Dinv, i, rv, zv);
      st4(z + 4 * (size_t)i, zv);
      for (int c = 0; c < 3; ++c) rz += (double)rv[c] * (double)zv[c];
    }
  }
  grid_sum2(rz, rr, PRE ? &sc->rz[i1] : nullptr, &sc->rr[i1], gr);
}

// multigrid-preconditioned start: r = b (free components), x = 0, ||b||^2
template <class V>
__global__ void k_pcg_init_mg(int nd, int npad, const double* __restrict__ b, const int* __restrict__ mask,
                              V* x, V* r, Scal* sc, GridRed gr) {
  double bb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    V rv[4] = {(V)0, (V)0, (V)0, (V)0};
    if (i < nd) {
      int mk = mask[i];
      for (int c = 0; c < 3; ++c) {
        rv[c] = ((mk >> c) & 1) ? (V)0 : (V)b[3 * (size_t)i + c];
        x[3 * (size_t)i + c] = (V)0;
        bb += (double)rv[c] * (double)rv[c];
      }
    }
    st4(r + 4 * (size_t)i, rv);
  }
  grid_sum1(bb, &sc->bb, gr);
}

template <class V>
__global__ void k_copy4(int npad, const V* __restrict__ a, V* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) {
    V v[4];
    ld4(a + 4 * (size_t)i, v);
    st4(b + 4 * (size_t)i, v);
  }
}

// B_k: converged? else beta = rz_{k+1}/rz_k; w = K z; p = z + beta p;
// q = w + beta q; pq_{k+1}  (one thread per row)
template <class T, class V>
__global__ void k_pcg_b(int nd, int npad, int k, Sliced S, const T* __restrict__ K,
                        const V* __restrict__ z, V* p, V* q, Scal* sc, GridRed gr) {
  if (sc->done) return;
  int i0 = k % 3, i1 = (k + 1) % 3, i2 = (k + 2) % 3;
  double rr = sc->rr[i1];
  if (rr <= sc->thr || !isfinite(rr)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->done = 1;
      sc->iters = k + 1;
      if (!isfinite(rr)) sc->breakdown = 1;
    }
    return;
  }
  V beta = (V)(sc->rz[i1] / sc->rz[i0]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz[i2] = 0.0;
    sc->rr[i2] = 0.0;
  }
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  double part = 0.0;
  if (sr < npad) {
    int r = S.row[sr];
    V y[3];
    sliced_row<T, V, V, 4>(sr, S, K, z, y);
    if (r < nd) {
      V zv[4], pv[4], qv[4];
      ld4(z + 4 * (size_t)r, zv);
      ld4(p + 4 * (size_t)r, pv);
      ld4(q + 4 * (size_t)r, qv);
      for (int c = 0; c < 3; ++c) {
        pv[c] = zv[c] + beta * pv[c];
        qv[c] = y[c] + beta * qv[c];
        part += (double)pv[c] * (double)qv[c];
      }
      st4(p + 4 * (size_t)r, pv);
      st4(q + 4 * (size_t)r, qv);
    }
  }
  grid_sum1(part, &sc->pq[i1], gr);
}

// ---------------------------------------------------------------- BiCGStab
// Vectors padded to 4 components over 32*nslice rows, in FP64 or (the FP32
// inner solve of the mixed path) FP32; x keeps the caller's 3-component
// layout; scalars and dot products in FP64.

// y = K x (+ optional dots a.y into slot and y.y into slot2).  Skipped once
// the solve is done, or (check_s) once the half-step residual s has converged.
// Bounded to 4 resident blocks of 256 per SM (64 registers): left to itself
// the compiler took 72, which allows 3, and the launch ran at 0.337 against
// 0.281 ms (FP32, 41.7 M blocks)
template <class T, class V>
__global__ void __launch_bounds__(256, 4) k_spmv_dot(int nd, int npad, Sliced S, const T* __restrict__ K,
                           const V* __restrict__ x, V* y, const V* __restrict__ a,
                           double* slot, double* slot2, const Scal* sc, int check_s, GridRed gr) {
  if (sc->done || (check_s && sc->a[5] <= sc->thr)) return;
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  double p1 = 0.0, p2 = 0.0;
  if (sr < npad) {
    int r = S.row[sr];
    V v[3];
    sliced_row<T, V, V, 4>(sr, S, K, x, v);
    if (r >= nd) v[0] = v[1] = v[2] = (V)0;
    V yv[4] = {v[0], v[1], v[2], (V)0};
    st4(y + 4 * (size_t)r, yv);
    if (a) {
      V av[4];
      ld4(a + 4 * (size_t)r, av);
      p1 = (double)av[0] * v[0] + (double)av[1] * v[1] + (double)av[2] * v[2];
    }
    p2 = (double)v[0] * v[0] + (double)v[1] * v[1] + (double)v[2] * v[2];
  }
  grid_sum2(p1, p2, slot, slot2, gr);
}

// start: r = r0 = b (free components), x = 0, ||b||^2
template <class V, class X>
__global__ void k_bicg_init(int nd, int npad, const double* __restrict__ b, const int* __restrict__ mask,
                            X* x, V* r, V* r0, Scal* sc, GridRed gr) {
  double bb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    V rv[4] = {(V)0, (V)0, (V)0, (V)0};
    if (i < nd) {
      int mk = mask[i];
      for (int c = 0; c < 3; ++c) {
        rv[c] = ((mk >> c) & 1) ? (V)0 : (V)b[3 * (size_t)i + c];
        x[3 * (size_t)i + c] = (X)0;
        bb += (double)rv[c] * (double)rv[c];
      }
    }
    st4(r + 4 * (size_t)i, rv);
    st4(r0 + 4 * (size_t)i, rv);
  }
  grid_sum1(bb, &sc->bb, gr);
}

// BiCGStab scalar slots in Scal::a: 0 rho, 1 alpha, 2 omega, 3 rho1 (r0.r),
// 4 r0.v, 5 s.s, 6 t.s, 7 t.t; rr[0] = r.r.  Only k_bicg_rotate (one thread)
// writes `done`, so no block ever sees it change within a launch.
template <class V>
__global__ void k_bicg_p(int npad, V* p, const V* __restrict__ r, const V* __restrict__ v,
                         V* ph, const V* __restrict__ Dinv, const Scal* sc) {
  if (sc->done) return;
  V beta = (V)((sc->a[3] / sc->a[0]) * (sc->a[1] / sc->a[2]));
  V om = (V)sc->a[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    V pv[4], rv[4], vv[4], zv[4];
    ld4(p + 4 * (size_t)i, pv);
    ld4(r + 4 * (size_t)i, rv);
    ld4(v + 4 * (size_t)i, vv);
    for (int c = 0; c < 4; ++c) pv[c] = rv[c] + beta * (pv[c] - om * vv[c]);
    st4(p + 4 * (size_t)i, pv);
    if (Dinv) {  // else the multigrid V-cycle writes ph
      apply_dinv(Dinv, i, pv, zv);
      st4(ph + 4 * (size_t)i, zv);
    }
  }
}

template <class V>
__global__ void k_bicg_s(int npad, const V* __restrict__ r, const V* __restrict__ v, V* s,
                         V* sh_, const V* __restrict__ Dinv, Scal* sc, GridRed gr) {
  if (sc->done) return;
  double rv0 = sc->a[4];
  if (!(fabs(rv0) > 0.0) || !isfinite(rv0)) return;  // breakdown, recorded by k_bicg_rotate
  V alpha = (V)(sc->a[3] / rv0);
  double ss = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    V rv[4], vv[4], sv[4], zv[4];
    ld4(r + 4 * (size_t)i, rv);
    ld4(v + 4 * (size_t)i, vv);
    for (int c = 0; c < 4; ++c) {
      sv[c] = rv[c] - alpha * vv[c];
      ss += (double)sv[c] * (double)sv[c];
    }
    st4(s + 4 * (size_t)i, sv);
    if (Dinv) {
      apply_dinv(Dinv, i, sv, zv);
      st4(sh_ + 4 * (size_t)i, zv);
    }
  }
  grid_sum1(ss, &sc->a[5], gr);
}

// converged on s: x += alpha ph (the rest of the iteration is skipped)
template <class V, class X>
__global__ void k_bicg_check_s(int nd, X* x, const V* __restrict__ ph, const Scal* sc) {
  if (sc->done || !(sc->a[5] <= sc->thr)) return;
  double rv = sc->a[4];
  if (!(fabs(rv) > 0.0) || !isfinite(rv)) return;
  double alpha = sc->a[3] / rv;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nd; i += gridDim.x * blockDim.x)
    x[i] += (X)(alpha * (double)ph[4 * (size_t)(i / 3) + i % 3]);
}

template <class V, class X>
__global__ void k_bicg_x(int nd, int npad, X* x, V* r, const V* __restrict__ ph,
                         const V* __restrict__ shv, const V* __restrict__ s,
                         const V* __restrict__ t, const V* __restrict__ r0, const Scal* sc,
                         double* next_rho1, double* next_rr, GridRed gr) {
  if (sc->done || sc->a[5] <= sc->thr) return;
  double rv0 = sc->a[4];
  if (!(fabs(rv0) > 0.0) || !isfinite(rv0)) return;
  double tt = sc->a[7];
  double om = tt > 0.0 ? sc->a[6] / tt : 0.0;
  double alpha = sc->a[3] / rv0;
  double rr = 0.0, rho1 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    V pv[4], zv[4], sv[4], tv[4], r0v[4], rv[4];
    ld4(ph + 4 * (size_t)i, pv);
    ld4(shv + 4 * (size_t)i, zv);
    ld4(s + 4 * (size_t)i, sv);
    ld4(t + 4 * (size_t)i, tv);
    ld4(r0 + 4 * (size_t)i, r0v);
    for (int c = 0; c < 4; ++c) {
      rv[c] = sv[c] - (V)om * tv[c];
      rr += (double)rv[c] * (double)rv[c];
      rho1 += (double)r0v[c] * (double)rv[c];
    }
    st4(r + 4 * (size_t)i, rv);
    if (i < nd)
      for (int c = 0; c < 3; ++c) x[3 * (size_t)i + c] += (X)(alpha * (double)pv[c] + om * (double)zv[c]);
  }
  grid_sum2(rr, rho1, next_rr, next_rho1, gr);
}

// end of an iteration (one thread): decide convergence or breakdown, rotate
__global__ void k_bicg_rotate(Scal* sc, const double* next_rho1, const double* next_rr, int it) {
  if (sc->done) return;
  double rv = sc->a[4];
  if (!(fabs(rv) > 0.0) || !isfinite(rv)) {
    sc->breakdown = 1;
    sc->done = 1;
    sc->iters = it;
    return;
  }
  if (sc->a[5] <= sc->thr) {
    sc->rr[0] = sc->a[5];
    sc->done = 1;
    sc->iters = it;
    return;
  }
  double tt = sc->a[7];
  double om = tt > 0.0 ? sc->a[6] / tt : 0.0;
  sc->a[0] = sc->a[3];       // rho <- rho1
  sc->a[1] = sc->a[3] / rv;  // alpha
  sc->a[2] = om;             // omega
  sc->a[3] = *next_rho1;     // r0 . r of the new residual
  sc->rr[0] = *next_rr;
  sc->a[4] = sc->a[5] = sc->a[6] = sc->a[7] = 0.0;
  if (sc->rr[0] <= sc->thr) {
    sc->done = 1;
    sc->iters = it;
  } else if (!(om != 0.0) || !isfinite(sc->rr[0])) {
    sc->breakdown = 1;
    sc->done = 1;
    sc->iters = it;
  }
}

// ---------------------------------------------------------------- refinement helpers

// r = b - K x (FP64 x in 3 components, FP64 accumulation, any matrix
// precision), masked, written in 3 (R3) or 4 components; slot += r.r
template <class T, int RS>
__global__ void k_residual64(int nd, int npad, Sliced S, const T* __restrict__ K,
                             const double* __restrict__ x, const float4* __restrict__ xs,
                             const double* __restrict__ b, const int* __restrict__ mask, double* r,
                             double* slot, GridRed gr) {
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  double part = 0.0;
  if (sr < npad) {
    int rr = S.row[sr];
    double y[3];
    if constexpr (sizeof(T) == 4)
      sliced_row_df(sr, S, (const float*)K, xs, y);
    else
      sliced_row<T, double, double, 3>(sr, S, K, x, y);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (rr < nd) {
      int mk = mask[rr];
      for (int c = 0; c < 3; ++c) {
        v[c] = ((mk >> c) & 1) ? 0.0 : b[3 * (size_t)rr + c] - y[c];
        part += v[c] * v[c];
      }
    }
    if (RS == 4)
      st4(r + 4 * (size_t)rr, v);
    else if (rr < nd)
      for (int c = 0; c < 3; ++c) r[3 * (size_t)rr + c] = v[c];
  }
  grid_sum1(part, slot, gr);
}

__global__ void k_axpy_f2d(int n, double* x, const float* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)d[i];
}

__global__ void k_copy_d(int n, double* y, const double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i];
}

// for an FP32 matrix, the (hi, lo) float split of x used by the double-float
// residual (nullptr otherwise)
template <class T>
const float4* residual_split(mpm_ctx* c, const mpm_mesh* m, const T* K, const double* x) {
  (void)K;
  if constexpr (sizeof(T) != 4) {
    return nullptr;
  } else {
    int npad = 32 * m->nslice;
    float4* xs = grow<float4>(c, c->v[22], 2 * (size_t)npad);
    MPM_LAUNCH(k_split_df<<<grid_for(npad, 256), 256, 0, c->stream>>>(npad, m->ndof, x, xs));
    return xs;
  }
}

Sliced sliced_of(const mpm_mesh* m) { return sliced_view(m); }

template <class T, class V>
int run_pcg(mpm_ctx* c, const mpm_mesh* m, const T* K, const V* Dinv, const double* b, V* x,
            double tol, int maxit, Scal* sc_d, Scal* sc_h, double* relres, int* iters, V* r, V* z,
            V* p, V* q) {
  cudaStream_t st = c->stream;
  int nd = m->ndof, npad = 32 * m->nslice;
  Sliced S = sliced_of(m);
  MPM_CUDA(cudaMemsetAsync(sc_d, 0, sizeof(Scal), st));
  int vb = 4 * 152;
  GridRed gr = grid_red(c, 2, std::max(vb, grid_for(npad, 32 * SW)));
  MPM_LAUNCH(k_pcg_init<V><<<vb, 256, 0, st>>>(nd, npad, b, ptr<int>(m->dof_mask), Dinv, x, r, z, p, sc_d, gr));
  MPM_LAUNCH(k_pcg_q0<T, V><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, K, p, q, sc_d, gr));
  MPM_CUDA(cudaMemcpyAsync(sc_h, sc_d, sizeof(Scal), cudaMemcpyDeviceToHost, st));
  MPM_CUDA(cudaStreamSynchronize(st));
  double bb = sc_h->bb;
  if (bb == 0.0) {
    *relres = 0.0;
    *iters = 0;
    return MPM_OK;
  }
  double thr = tol * tol * bb;
  MPM_CUDA(cudaMemcpyAsync(&sc_d->thr, &thr, sizeof(double), cudaMemcpyHostToDevice, st));
  MPM_CUDA(cudaStreamSynchronize(st));
  int k = 0;
  const int batch = 32;
  while (k < maxit) {
    int kend = std::min(maxit, k + batch);
    for (; k < kend; ++k) {
      MPM_LAUNCH_P(MPM_PROF_PCG_UPDATE, k_pcg_a<V><<<vb, 256, 0, st>>>(nd, k, Dinv, x, r, z, p, q, sc_d, gr));
      MPM_LAUNCH_P(MPM_PROF_PCG_SPMV, k_pcg_b<T, V><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, k, S, K, z, p, q, sc_d, gr));
    }
    MPM_CUDA(cudaMemcpyAsync(sc_h, sc_d, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    if (sc_h->done) break;
  }
  if (!sc_h->done) {
    *iters = maxit;
    *relres = sqrt(sc_h->rr[maxit % 3] / bb);
    return MPM_ERR_KRYLOV;
  }
  *iters = sc_h->iters;
  *relres = sqrt(sc_h->rr[sc_h->iters % 3] / bb);
  return sc_h->breakdown ? MPM_ERR_KRYLOV : MPM_OK;
}

// PCG preconditioned by one multigrid V-cycle per iteration (mpm_mg.cu);
// the V-cycle kernels skip their work once the residual of the iteration has
// converged, so batches of launches cost nothing after convergence
template <class T>
int run_pcg_mg(mpm_ctx* c, const mpm_mesh* m, const T* K, const double* b, T* x, double tol,
               int maxit, Scal* sc_d, Scal* sc_h, double* relres, int* iters, T* r, T* z, T* p, T* q) {
  cudaStream_t st = c->stream;
  int nd = m->ndof, npad = 32 * m->nslice;
  Sliced S = sliced_of(m);
  MPM_CUDA(cudaMemsetAsync(sc_d, 0, sizeof(Scal), st));
  int vb = 4 * 152;
  GridRed gr = grid_red(c, 2, std::max(vb, grid_for(npad, 32 * SW)));
  MPM_LAUNCH(k_pcg_init_mg<T><<<vb, 256, 0, st>>>(nd, npad, b, ptr<int>(m->dof_mask), x, r, sc_d, gr));
  mg_apply<T>(c, m, K, r, z, nullptr, 0, &sc_d->rz[0]);
  MPM_LAUNCH(k_copy4<T><<<grid_for(npad, 256), 256, 0, st>>>(npad, z, p));
  MPM_LAUNCH(k_pcg_q0<T, T><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, K, p, q, sc_d, gr));
  MPM_CUDA(cudaMemcpyAsync(sc_h, sc_d, sizeof(Scal), cudaMemcpyDeviceToHost, st));
  MPM_CUDA(cudaStreamSynchronize(st));
  double bb = sc_h->bb;
  if (bb == 0.0) {
    *relres = 0.0;
    *iters = 0;
    return MPM_OK;
  }
  double thr = tol * tol * bb;
  MPM_CUDA(cudaMemcpyAsync(&sc_d->thr, &thr, sizeof(double), cudaMemcpyHostToDevice, st));
  int k = 0;
  const int batch = 4;
  while (k < maxit) {
    int kend = std::min(maxit, k + batch);
    for (; k < kend; ++k) {
      MPM_LAUNCH_P(MPM_PROF_PCG_UPDATE, k_pcg_a<T, false><<<vb, 256, 0, st>>>(nd, k, nullptr, x, r, z, p, q, sc_d, gr));
      mg_apply<T>(c, m, K, r, z, sc_d, k, &sc_d->rz[(k + 1) % 3]);
      MPM_LAUNCH_P(MPM_PROF_PCG_SPMV, k_pcg_b<T, T><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, k, S, K, z, p, q, sc_d, gr));
    }
    MPM_CUDA(cudaMemcpyAsync(sc_h, sc_d, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    if (sc_h->done) break;
  }
  if (!sc_h->done) {
    *iters = maxit;
    *relres = sqrt(sc_h->rr[maxit % 3] / bb);
    return MPM_ERR_KRYLOV;
  }
  *iters = sc_h->iters;
  *relres = sqrt(sc_h->rr[sc_h->iters % 3] / bb);
  return sc_h->breakdown ? MPM_ERR_KRYLOV : MPM_OK;
}

// z = B y by one V-cycle (vectors of 4 components over 32*nslice rows); an
// FP64 V-cycle on FP64 vectors, or the FP32 V-cycle on FP32 vectors
template <class T>
void mg_precondition(mpm_ctx* c, const mpm_mesh* m, const T* K, const T* y, T* z, const Scal* sc) {
  mg_apply<T>(c, m, K, y, z, sc, -1, nullptr);
}

// BiCGStab, right preconditioned by block Jacobi (Dinv) or, with Dinv null,
// by one multigrid V-cycle per half-step (mg_setup already run for K).  The
// vectors are T (the matrix precision): FP64, or FP32 for the inner solve of
// the mixed path; x (X) is the caller's 3-component solution.
template <class T, class X>
int run_bicgstab(mpm_ctx* c, const mpm_mesh* m, const T* K, const T* Dinv, const double* b,
                 X* x, double tol, int maxit, Scal* sc_d, Scal* sc_h, double* relres,
                 int* iters) {
  typedef T V;
  cudaStream_t st = c->stream;
  int nd = m->ndof, npad = 32 * m->nslice;
  size_t n4 = 4 * (size_t)npad;
  V* r = grow<V>(c, c->v[4], n4);
  V* r0 = grow<V>(c, c->v[5], n4);
  V* p = grow<V>(c, c->v[6], n4);
  V* v = grow<V>(c, c->v[7], n4);
  V* s = grow<V>(c, c->v[8], n4);
  V* t = grow<V>(c, c->v[9], n4);
  V* ph = grow<V>(c, c->v[10], n4);
  V* shv = grow<V>(c, c->v[11], n4);
  Sliced S = sliced_of(m);
  const int* mask = ptr<int>(m->dof_mask);
  MPM_CUDA(cudaMemsetAsync(sc_d, 0, sizeof(Scal), st));
  MPM_CUDA(cudaMemsetAsync(p, 0, sizeof(V) * n4, st));
  MPM_CUDA(cudaMemsetAsync(v, 0, sizeof(V) * n4, st));
  double* red = c->d_red + 40;  // rho1 / rr accumulators of the next iteration
  MPM_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
  int vb = 4 * 152, it = 0;
  GridRed gr = grid_red(c, 2, std::max(vb, grid_for(npad, 32 * SW)));
  // r = r0 = b (free components), x = 0, ||b||^2
  MPM_LAUNCH(k_bicg_init<V, X><<<vb, 256, 0, st>>>(nd, npad, b, mask, x, r, r0, sc_d, gr));
  MPM_CUDA(cudaMemcpyAsync(sc_h, sc_d, sizeof(Scal), cudaMemcpyDeviceToHost, st));
  MPM_CUDA(cudaStreamSynchronize(st));
  double bb = sc_h->bb;
  if (bb == 0.0) {
    *relres = 0.0;
    *iters = 0;
    return MPM_OK;
  }
  Scal init{};
  init.bb = bb;
  init.thr = tol * tol * bb;
  init.a[0] = init.a[1] = init.a[2] = 1.0;
  init.a[3] = bb;  // r0 . r at the start
  MPM_CUDA(cudaMemcpyAsync(sc_d, &init, sizeof(Scal), cudaMemcpyHostToDevice, st));
  const int batch = Dinv ? 16 : 4;
  while (it < maxit) {
    int iend = std::min(maxit, it + batch);
    for (; it < iend; ++it) {
      MPM_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
      MPM_LAUNCH(k_bicg_p<V><<<vb, 256, 0, st>>>(npad, p, r, v, ph, Dinv, sc_d));
      if (!Dinv) mg_precondition<T>(c, m, K, p, ph, sc_d);
      MPM_LAUNCH_P(MPM_PROF_BICG_SPMV, k_spmv_dot<T, V><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, K, ph, v, r0, &sc_d->a[4], nullptr, sc_d, 0, gr));
      MPM_LAUNCH(k_bicg_s<V><<<vb, 256, 0, st>>>(npad, r, v, s, shv, Dinv, sc_d, gr));
      MPM_LAUNCH(k_bicg_check_s<V, X><<<vb, 256, 0, st>>>(nd, x, ph, sc_d));
      if (!Dinv) mg_precondition<T>(c, m, K, s, shv, sc_d);
      MPM_LAUNCH_P(MPM_PROF_BICG_SPMV, k_spmv_dot<T, V><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, K, shv, t, s, &sc_d->a[6], &sc_d->a[7], sc_d, 1, gr));
      MPM_LAUNCH(k_bicg_x<V, X><<<vb, 256, 0, st>>>(nd, npad, x, r, ph, shv, s, t, r0, sc_d, red, red + 1, gr));
      MPM_LAUNCH(k_bicg_rotate<<<1, 1, 0, st>>>(sc_d, red, red + 1, it + 1));
    }
    MPM_CUDA(cudaMemcpyAsync(sc_h, sc_d, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    if (sc_h->done) break;
  }
  *iters = sc_h->done ? sc_h->iters : maxit;
  *relres = sqrt(sc_h->rr[0] / bb);
  if (!sc_h->done || sc_h->breakdown) return MPM_ERR_KRYLOV;
  return MPM_OK;
}

// ---------------------------------------------------------------- GMRES
// Restarted GMRES(m) right preconditioned by 3x3 block Jacobi (Sec. 6.4 names
// GMRES with a Jacobi preconditioner as the iterative route for the CPT's
// linear solves).  The Arnoldi basis is orthogonalised by classical
// Gram-Schmidt applied twice (CGS2: two passes of j + 1 dot products and one
// combined update each, instead of the j + 1 dependent steps of modified
// Gram-Schmidt); the dot products are fixed-order two-stage reductions, the
// small Hessenberg least-squares problem is solved on the host by Givens
// rotations.  Vectors are T (FP64, or FP32 for the inner solve of the mixed
// path) padded to 4 components over 32 nslice rows; sums in FP64.

// r = b - K x on the free components (x over 4-component rows), rows beyond
// nd and fixed components zero
template <class T, class V>
__global__ void k_gm_residual(int nd, int npad, Sliced S, const T* __restrict__ K, const V* __restrict__ x,
                              const double* __restrict__ b, const int* __restrict__ mask, V* r) {
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  if (sr >= npad) return;
  int i = S.row[sr];
  V y[3];
  sliced_row<T, V, V, 4>(sr, S, K, x, y);
  V rv[4] = {(V)0, (V)0, (V)0, (V)0};
  if (i < nd) {
    int mi = mask[i];
    for (int c = 0; c < 3; ++c)
      rv[c] = ((mi >> c) & 1) ? (V)0 : (V)(b[3 * (size_t)i + c] - (double)y[c]);
  }
  st4(r + 4 * (size_t)i, rv);
}

// w = K (Dinv v): the preconditioned direction z = Dinv v first (kept in z),
// then the row product
template <class V>
__global__ void k_gm_dinv(int nd, int npad, const V* __restrict__ Dinv, const V* __restrict__ v, V* z) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  V rv[4], zv[4] = {(V)0, (V)0, (V)0, (V)0};
  if (i < nd) {  // rows beyond nd: no preconditioner block
    ld4(v + 4 * (size_t)i, rv);
    apply_dinv(Dinv, i, rv, zv);
  }
  st4(z + 4 * (size_t)i, zv);
}

template <class T, class V>
__global__ void k_gm_spmv(int nd, int npad, Sliced S, const T* __restrict__ K, const V* __restrict__ z, V* w) {
  int sr = blockIdx.x * blockDim.x + threadIdx.x;  // storage row
  if (sr >= npad) return;
  int i = S.row[sr];
  V y[3];
  sliced_row<T, V, V, 4>(sr, S, K, z, y);
  V wv[4] = {y[0], y[1], y[2], (V)0};
  if (i >= nd) wv[0] = wv[1] = wv[2] = (V)0;
  st4(w + 4 * (size_t)i, wv);
}

// stage 1 of the dots V_i . w (i = blockIdx.y < nv; V_i at Vb + i n4): each
// block's partial sum of its strided entries, by the block's fixed tree
template <class V>
__global__ void k_gm_dots(long long n4, const V* __restrict__ Vb, const V* __restrict__ w, double* part) {
  __shared__ double sh[32];
  const V* vi = Vb + (size_t)blockIdx.y * n4;
  double s = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x)
    s += (double)vi[k] * (double)w[k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// stage 2: h[i] = the block partials of dot i added in block order
__global__ void k_gm_dots_fin(int nb, const double* __restrict__ part, double* h) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)blockIdx.x * nb + b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}

// w -= sum_i h[i] V_i (i < nv)
template <class V>
__global__ void k_gm_orth(long long n4, int nv, const V* __restrict__ Vb, const double* __restrict__ h, V* w) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n4) return;
  double s = (double)w[k];
  for (int i = 0; i < nv; ++i) s -= h[i] * (double)Vb[(size_t)i * n4 + k];
  w[k] = (V)s;
}

// y = a x
template <class V>
__global__ void k_gm_scale(long long n4, double a, const V* __restrict__ x, V* y) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n4) y[k] = (V)(a * (double)x[k]);
}

// u = sum_i y[i] V_i, then x += Dinv u over the rows (one thread per row)
template <class V>
__global__ void k_gm_update_x(int nd, long long n4, int nv, const V* __restrict__ Vb, const double* __restrict__ y,
                              const V* __restrict__ Dinv, V* x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  V u[4];
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += y[j] * (double)Vb[(size_t)j * n4 + 4 * (size_t)i + c];
    u[c] = (V)s;
  }
  V zv[4], xv[4];
  apply_dinv(Dinv, i, u, zv);
  ld4(x + 4 * (size_t)i, xv);
  for (int c = 0; c < 3; ++c) xv[c] += zv[c];
  st4(x + 4 * (size_t)i, xv);
}

// x (4-component rows) -> the caller's 3-component solution
template <class V, class X>
__global__ void k_gm_out(int nd, const V* __restrict__ x4, X* x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nd) return;
  x[i] = (X)x4[4 * (size_t)(i / 3) + i % 3];
}

template <class T>
int run_gmres(mpm_ctx* c, const mpm_mesh* m, const T* K, const T* Dinv, const double* b, T* xout,
              double tol, int maxit, int restart, double* relres, int* iters) {
  typedef T V;
  cudaStream_t st = c->stream;
  int nd = m->ndof, npad = 32 * m->nslice, mr = restart;
  long long n4 = 4LL * npad;
  V* Vb = grow<V>(c, c->v[28], (size_t)(mr + 1) * n4);
  V* w = grow<V>(c, c->v[29], n4);
  V* z = grow<V>(c, c->v[30], n4);
  V* x = grow<V>(c, c->v[31], n4);
  Sliced S = sliced_of(m);
  const int* mask = ptr<int>(m->dof_mask);
  int nbk = std::min(4 * 152, std::max(1, (int)((n4 + 255) / 256)));
  double* part = grow<double>(c, c->v[23], (size_t)(mr + 1) * nbk + 2 * (mr + 1));
  double* hd = part + (size_t)(mr + 1) * nbk;  // device h (mr + 1) and y (mr + 1)
  double* yd = hd + (mr + 1);
  double* hh = c->h_red;  // pinned host: up to 32 values
  if (mr + 1 > 32) throw CudaError(MPM_ERR_ARG, "GMRES restart too long");
  int gr = grid_for(npad, 256);
  int gv = (int)((n4 + 255) / 256);
  auto dots = [&](int nv, const V* base, const V* vec) {
    MPM_LAUNCH(k_gm_dots<V><<<dim3(nbk, nv), 256, 0, st>>>(n4, base, vec, part));
    MPM_LAUNCH(k_gm_dots_fin<<<nv, 256, 0, st>>>(nbk, part, hd));
    MPM_CUDA(cudaMemcpyAsync(hh, hd, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
  };
  MPM_CUDA(cudaMemsetAsync(x, 0, sizeof(V) * n4, st));
  // ||b|| over the free components
  MPM_LAUNCH(k_gm_residual<T, V><<<gr, 256, 0, st>>>(nd, npad, S, K, x, b, mask, w));
  dots(1, w, w);
  double bn = sqrt(hh[0]);
  *iters = 0;
  *relres = 0.0;
  if (bn == 0.0) {
    MPM_LAUNCH(k_gm_out<V, T><<<grid_for(3 * nd, 256), 256, 0, st>>>(nd, x, xout));
    return MPM_OK;
  }
  std::vector<double> H((size_t)(mr + 1) * mr), cs(mr), sn(mr), g(mr + 1), y(mr + 1);
  int total = 0;
  double beta = bn;
  bool conv = false;
  while (total < maxit && !conv) {
    // restart: V_0 = r / ||r||
    MPM_LAUNCH(k_gm_scale<V><<<gv, 256, 0, st>>>(n4, 1.0 / beta, w, Vb));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < mr && total < maxit; ++j) {
      V* vj1 = Vb + (size_t)(j + 1) * n4;
      MPM_LAUNCH(k_gm_dinv<V><<<gr, 256, 0, st>>>(nd, npad, Dinv, Vb + (size_t)j * n4, z));
      MPM_LAUNCH_P(MPM_PROF_BICG_SPMV, k_gm_spmv<T, V><<<gr, 256, 0, st>>>(nd, npad, S, K, z, w));
      double hcol[33];
      for (int i = 0; i <= j; ++i) hcol[i] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        dots(j + 1, Vb, w);
        for (int i = 0; i <= j; ++i) hcol[i] += hh[i];
        MPM_LAUNCH(k_gm_orth<V><<<gv, 256, 0, st>>>(n4, j + 1, Vb, hd, w));
      }
      dots(1, w, w);
      double hn = sqrt(hh[0]);
      hcol[j + 1] = hn;
      ++total;
      // apply the earlier rotations to the new column, then its own
      for (int i = 0; i < j; ++i) {
        double t0 = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = t0;
      }
      double den = hypot(hcol[j], hcol[j + 1]);
      cs[j] = den > 0.0 ? hcol[j] / den : 1.0;
      sn[j] = den > 0.0 ? hcol[j + 1] / den : 0.0;
      hcol[j] = den;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * mr + j] = hcol[i];
      if (fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
        conv = true;
        ++j;
        break;
      }
      MPM_LAUNCH(k_gm_scale<V><<<gv, 256, 0, st>>>(n4, 1.0 / hn, w, vj1));
    }
    // y = R^-1 g (upper triangular), x += Dinv (V y)
    int k = j;
    for (int i = k - 1; i >= 0; --i) {
      double sm = g[i];
      for (int l = i + 1; l < k; ++l) sm -= H[(size_t)i * mr + l] * y[l];
      y[i] = H[(size_t)i * mr + i] != 0.0 ? sm / H[(size_t)i * mr + i] : 0.0;
    }
    MPM_CUDA(cudaMemcpyAsync(yd, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    MPM_LAUNCH(k_gm_update_x<V><<<grid_for(nd, 256), 256, 0, st>>>(nd, n4, k, Vb, yd, Dinv, x));
    // the true residual of the restart (and of the end)
    MPM_LAUNCH(k_gm_residual<T, V><<<gr, 256, 0, st>>>(nd, npad, S, K, x, b, mask, w));
    dots(1, w, w);
    beta = sqrt(hh[0]);
    conv = beta <= tol * bn;
  }
  MPM_LAUNCH(k_gm_out<V, T><<<grid_for(3 * nd, 256), 256, 0, st>>>(nd, x, xout));
  *iters = total;
  *relres = beta / bn;
  return conv ? MPM_OK : MPM_ERR_KRYLOV;
}

}  // namespace

void solve(mpm_ctx* c, const mpm_mesh* mc, const mpm_material& mat, const void* K,
           const double* b, double* x, const mpm_solve_params& prm, mpm_solve_stats* out) {
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  cudaStream_t st = c->stream;
  int nd = m->ndof, n3 = 3 * nd, npad = 32 * m->nslice;
  size_t n4 = 4 * (size_t)npad;
  const int* rp = ptr<int>(m->row_ptr);
  const int* col = ptr<int>(m->col);
  Sliced S = sliced_of(m);
  int method = prm.method;
  // non-associated Drucker-Prager, the Willam-Warnke cone (its potential is
  // not its yield function) and Coulomb friction make K non-symmetric
  bool sym = !(mat.model == 2 && mat.psi != mat.phi) && mat.model != 3 &&
             !(mat.mu > 0.0 && mat.contact_on);
  if (method == 0) method = sym ? 1 : 2;
  bool mgb = method == 3 && !sym;  // multigrid-preconditioned BiCGStab
  const int GMRES_M = 30;          // restart length of method 4
  Scal* sc_d = grow<Scal>(c, c->v[20], 1);
  Scal* sc_h = (Scal*)(c->h_red + 32);  // pinned, 32 doubles fit Scal
  // partial sums of every grid sum of this solve in one buffer, sized once so
  // that no later request moves it
  grid_red(c, 4, std::max(4096, grid_for(npad, 32 * SW)));
  MPM_CUDA(cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), st));
  static_assert(sizeof(Scal) <= 32 * sizeof(double), "scalar block too large");
  out->iterations = 0;
  out->refinements = 0;
  out->status = MPM_OK;
  if (prm.precision == MPM_FP64) {
    const double* Kd = (const double*)K;
    double* Dinv = grow<double>(c, c->v[3], 12 * (size_t)npad);
    MPM_LAUNCH(k_block_jacobi<double, double><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, S, Kd, Dinv, c->d_err));
    int its = 0;
    double rel = 0.0;
    int sst;
    if (method == 4) {
      sst = run_gmres<double>(c, m, Kd, Dinv, b, x, prm.tol, prm.maxit, GMRES_M, &rel, &its);
    } else if (mgb) {
      mg_setup<double>(c, m, Kd, prm.mg_reuse != 0);
      sst = run_bicgstab<double, double>(c, m, Kd, nullptr, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its);
    } else if (method == 3) {
      mg_setup<double>(c, m, Kd, prm.mg_reuse != 0);
      sst = run_pcg_mg<double>(c, m, Kd, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its,
                               grow<double>(c, c->v[4], n4), grow<double>(c, c->v[5], n4),
                               grow<double>(c, c->v[6], n4), grow<double>(c, c->v[7], n4));
    } else if (method == 1)
      sst = run_pcg<double, double>(c, m, Kd, Dinv, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its,
                                    grow<double>(c, c->v[4], n4), grow<double>(c, c->v[5], n4),
                                    grow<double>(c, c->v[6], n4), grow<double>(c, c->v[7], n4));
    else
      sst = run_bicgstab<double, double>(c, m, Kd, Dinv, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its);
    out->iterations = its;
    out->relres = rel;
    out->status = sst;
    if (sst)
      set_error(c, std::string(method == 4 ? "GMRES" : method == 1 ? "PCG" : (mgb ? "multigrid BiCGStab" : (method == 3 ? "multigrid PCG" : "BiCGStab"))) +
                       " did not reach the tolerance (" +
                       std::to_string(its) + " iterations, relative residual " +
                       std::to_string(rel) + (sc_h->breakdown ? ", breakdown)" : ")"));
    return;
  }
  // mixed: FP32 inner solves (PCG for symmetric K, BiCGStab otherwise) inside
  // FP64 iterative refinement, the refinement residual accumulated in
  // double-float arithmetic from the FP32 matrix
  const float* Kf = (const float*)K;
  double inner = prm.inner_tol > 0 ? prm.inner_tol : 1e-3;
  double* r64 = grow<double>(c, c->v[12], n3);
  float* d32 = grow<float>(c, c->v[13], n3);
  double* slot = c->d_red + 44;
  GridRed gred = grid_red(c, 2, grid_for(npad, 32 * SW));
  bool gmres = method == 4;
  bool bicg = !sym && method != 1 && !gmres;
  float* Dinv = grow<float>(c, c->v[3], 12 * (size_t)npad);
  if (method == 3)
    mg_setup<float>(c, m, Kf, prm.mg_reuse != 0);
  else
    MPM_LAUNCH(k_block_jacobi<float, float><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, S, Kf, Dinv, c->d_err));
  float* r = grow<float>(c, c->v[4], n4);
  float* z = grow<float>(c, c->v[5], n4);
  float* pp = grow<float>(c, c->v[6], n4);
  float* q = grow<float>(c, c->v[7], n4);
  MPM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n3, st));
  MPM_CUDA(cudaMemsetAsync(slot, 0, sizeof(double), st));
  MPM_LAUNCH_P(MPM_PROF_REFINE, k_residual64<float, 3><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, Kf, x, residual_split(c, m, Kf, x), b, ptr<int>(m->dof_mask), r64, slot, gred));
  MPM_CUDA(cudaMemcpyAsync(c->h_red + 60, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  MPM_CUDA(cudaStreamSynchronize(st));
  double bb = c->h_red[60], rr = bb;
  int total = 0, rounds = 0, status = MPM_OK;
  bool breakdown = false;
  while (rr > prm.tol * prm.tol * bb && rr > 0.0) {
    if (total >= prm.maxit || rounds >= 50) {
      status = MPM_ERR_KRYLOV;
      break;
    }
    int its = 0;
    double rel = 0.0;
    int sst;
    if (gmres)
      sst = run_gmres<float>(c, m, Kf, Dinv, r64, d32, inner, prm.maxit - total, GMRES_M, &rel, &its);
    else if (bicg)
      sst = run_bicgstab<float, float>(c, m, Kf, method == 3 ? nullptr : Dinv, r64, d32, inner,
                                       prm.maxit - total, sc_d, sc_h, &rel, &its);
    else if (method == 3)
      sst = run_pcg_mg<float>(c, m, Kf, r64, d32, inner, prm.maxit - total, sc_d, sc_h, &rel, &its, r,
                              z, pp, q);
    else
      sst = run_pcg<float, float>(c, m, Kf, Dinv, r64, d32, inner, prm.maxit - total, sc_d, sc_h,
                                  &rel, &its, r, z, pp, q);
    total += its;
    ++rounds;
    breakdown = breakdown || sc_h->breakdown;
    if (sst && its == 0) {
      status = MPM_ERR_KRYLOV;
      break;
    }
    MPM_LAUNCH(k_axpy_f2d<<<grid_for(n3, 256), 256, 0, st>>>(n3, x, d32));
    MPM_CUDA(cudaMemsetAsync(slot, 0, sizeof(double), st));
    MPM_LAUNCH_P(MPM_PROF_REFINE, k_residual64<float, 3><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, Kf, x, residual_split(c, m, Kf, x), b, ptr<int>(m->dof_mask), r64, slot, gred));
    MPM_CUDA(cudaMemcpyAsync(c->h_red + 60, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    rr = c->h_red[60];
  }
  out->iterations = total;
  out->refinements = rounds;
  out->relres = bb > 0 ? sqrt(rr / bb) : 0.0;
  out->status = status;
  if (status)
    set_error(c, std::string("mixed-precision refinement (") + (gmres ? "GMRES" : bicg ? "BiCGStab" : "PCG") +
                     " inner solves) did not reach the tolerance" + (breakdown ? " (breakdown)" : ""));
}

// ---------------------------------------------------------------- allocation-free PCG
//
// A variant of the FP64 block-Jacobi PCG above for callers that must not
// allocate device memory during the solve.  Its work vectors, preconditioner
// blocks and scalars live in this file-scope array, reserved once when the
// library is loaded on a device and kept until the process exits.

namespace {

constexpr size_t kStaticBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_pcg_scratch[kStaticBytes];

// layout of the array: Krylov scalars, the grid-sum ticket, the per-block
// partial sums (kStaticParts doubles), then the work vectors
constexpr size_t kStaticScal = 256, kStaticTicket = 256, kStaticParts = 2048;
constexpr size_t kStaticHead = kStaticScal + kStaticTicket + kStaticParts * sizeof(double);

constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_pcg_scratch_dev[kMaxDevices];

// device address of g_pcg_scratch on the context's device, looked up once per
// device; the context's device must be the current one (the address belongs
// to the device current at the lookup)
unsigned char* static_scratch(mpm_ctx* c) {
  int dev = 0;
  MPM_CUDA(cudaGetDevice(&dev));
  if (dev != c->device)
    throw CudaError(MPM_ERR_ARG, "mpm_solve_static: the context's device (" + std::to_string(c->device) +
                                     ") is not the current device (" + std::to_string(dev) + ")");
  if (dev < 0 || dev >= kMaxDevices) throw CudaError(MPM_ERR_ARG, "device ordinal out of range");
  unsigned char* p = g_pcg_scratch_dev[dev].load(std::memory_order_acquire);
  if (!p) {
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&q, g_pcg_scratch);
    if (e != cudaSuccess)
      throw CudaError(MPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    // two threads racing here look up the same address
    g_pcg_scratch_dev[dev].store((unsigned char*)q, std::memory_order_release);
    p = (unsigned char*)q;
  }
  return p;
}

}  // namespace

}  // namespace mpm

using namespace mpm;

extern "C" int mpm_solve_static(mpm_ctx* c, const mpm_mesh* m, const double* K, const double* rhs,
                                double* x, double tol, int maxit, mpm_solve_stats* stats) {
  if (!c || !m || !K || !rhs || !x || !m->built || !(tol > 0) || maxit <= 0) return MPM_ERR_ARG;
  int nd = m->ndof, npad = 32 * m->nslice;
  // layout: scalars, ticket and partial sums (kStaticHead bytes), then r, z,
  // p, q (4 per row over the padded rows) and the 3x3 inverses (12 per row)
  size_t need = kStaticHead + sizeof(double) * (size_t)npad * (4 * 4 + 12);
  const size_t max_rows = (kStaticBytes - kStaticHead) / (28 * sizeof(double));
  if (need > kStaticBytes) {
    set_error(c, "mpm_solve_static: " + std::to_string(nd) + " dofs need " + std::to_string(need) +
                     " bytes of scratch, the static array holds " + std::to_string(kStaticBytes) +
                     " (at most " + std::to_string(max_rows / 32 * 32) + " dofs)");
    return MPM_ERR_ARG;
  }
  try {
    cudaStream_t st = c->stream;
    unsigned char* base = static_scratch(c);
    Scal* sc = (Scal*)base;
    unsigned* ticket = (unsigned*)(base + kStaticScal);
    GridRed gr{(double*)(base + kStaticScal + kStaticTicket), ticket};
    double* r = (double*)(base + kStaticHead);
    double* z = r + 4 * (size_t)npad;
    double* p = z + 4 * (size_t)npad;
    double* q = p + 4 * (size_t)npad;
    double* Dinv = q + 4 * (size_t)npad;
    const int* rp = ptr<int>(m->row_ptr);
    const int* col = ptr<int>(m->col);
    Sliced S = sliced_of(m);
    // the array keeps the previous call's contents: every vector below is
    // written before it is read, and the scalars start from zero
    MPM_CUDA(cudaMemsetAsync(sc, 0, sizeof(Scal), st));
    MPM_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
    MPM_LAUNCH(k_block_jacobi<double, double><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, S, K, Dinv, c->d_err));
    int vb = 4 * 152;
    // every grid sum below has at most max(vb, npad / 256) blocks of 2 values
    static_assert(2 * 4 * 152 <= kStaticParts, "partial sums of the vector kernels");
    static_assert((kStaticBytes / (28 * sizeof(double)) / 256 + 1) <= kStaticParts,
                  "partial sums of the row kernels");
    MPM_LAUNCH(k_pcg_init<double><<<vb, 256, 0, st>>>(nd, npad, rhs, ptr<int>(m->dof_mask), Dinv, x, r, z, p, sc, gr));
    MPM_LAUNCH(k_pcg_q0<double, double><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, S, K, p, q, sc, gr));
    Scal* h = (Scal*)(c->h_red + 32);
    MPM_CUDA(cudaMemcpyAsync(h, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    double bb = h->bb;
    mpm_solve_stats s{};
    if (bb > 0.0) {
      double thr = tol * tol * bb;
      MPM_CUDA(cudaMemcpyAsync(&sc->thr, &thr, sizeof(double), cudaMemcpyHostToDevice, st));
      int k = 0;
      while (k < maxit) {
        int kend = std::min(maxit, k + 32);
        for (; k < kend; ++k) {
          MPM_LAUNCH(k_pcg_a<double><<<vb, 256, 0, st>>>(nd, k, Dinv, x, r, z, p, q, sc, gr));
          MPM_LAUNCH(k_pcg_b<double, double><<<grid_for(npad, 32 * SW), 32 * SW, 0, st>>>(nd, npad, k, S, K, z, p, q, sc, gr));
        }
        MPM_CUDA(cudaMemcpyAsync(h, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        MPM_CUDA(cudaStreamSynchronize(st));
        if (h->done) break;
      }
      s.iterations = h->done ? h->iters : maxit;
      s.relres = sqrt(h->rr[s.iterations % 3] / bb);
      s.status = (!h->done || h->breakdown) ? MPM_ERR_KRYLOV : MPM_OK;
    }
    int e = check_device_error(c, "mpm_solve_static");
    if (stats) *stats = s;
    if (e) return e;
    if (s.status) set_error(c, "mpm_solve_static: PCG did not reach the tolerance");
    return s.status;
  } catch (const CudaError& e) {
    set_error(c, e.what());
    return e.code;
  }
}
