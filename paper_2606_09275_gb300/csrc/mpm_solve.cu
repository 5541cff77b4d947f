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
#include <cmath>
#include <string>

#include "mpm_internal.cuh"

namespace mpm {
namespace {

constexpr int SW = 8;  // warps (rows) per block of the row kernels

struct Scal {
  double rz[3], pq[3], rr[3];
  double bb, thr;    // ||b||^2 and tol^2 ||b||^2
  double a[8];       // BiCGStab scalars
  int done, iters, breakdown, pad;
};

template <class T, class V, class A>
__device__ inline void row_dot(int r, int lane, const int* __restrict__ rp, const int* __restrict__ col,
                               const T* __restrict__ K, const V* __restrict__ x, A& y0, A& y1, A& y2) {
  int s0 = rp[r], nb = rp[r + 1] - s0;
  const T* b = K + 9 * (size_t)s0;
  y0 = y1 = y2 = (A)0;
  for (int k = lane; k < nb; k += 32) {
    int c = col[s0 + k];
    A x0 = (A)x[3 * (size_t)c], x1 = (A)x[3 * (size_t)c + 1], x2 = (A)x[3 * (size_t)c + 2];
    y0 += (A)b[k] * x0 + (A)b[nb + k] * x1 + (A)b[2 * (size_t)nb + k] * x2;
    y1 += (A)b[3 * (size_t)nb + k] * x0 + (A)b[4 * (size_t)nb + k] * x1 + (A)b[5 * (size_t)nb + k] * x2;
    y2 += (A)b[6 * (size_t)nb + k] * x0 + (A)b[7 * (size_t)nb + k] * x1 + (A)b[8 * (size_t)nb + k] * x2;
  }
  y0 = warp_sum(y0);
  y1 = warp_sum(y1);
  y2 = warp_sum(y2);
}

// block-Jacobi: inverse of each 3x3 diagonal block (row-major, 9 per dof)
template <class T, class V>
__global__ void k_block_jacobi(int nd, const int* __restrict__ rp, const int* __restrict__ col,
                               const T* __restrict__ K, V* Dinv, int* err) {
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
  double a[9];
  for (int e = 0; e < 9; ++e) a[e] = k >= 0 ? (double)K[9 * (size_t)s0 + (size_t)e * nb + k] : (e % 4 == 0);
  double c0 = a[4] * a[8] - a[5] * a[7], c1 = a[5] * a[6] - a[3] * a[8], c2 = a[3] * a[7] - a[4] * a[6];
  double det = a[0] * c0 + a[1] * c1 + a[2] * c2;
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    atomicOr(err, EB_KRYLOV);
    det = 1.0;
  }
  double id = 1.0 / det;
  V* o = Dinv + 9 * (size_t)r;
  o[0] = (V)(c0 * id);
  o[1] = (V)((a[2] * a[7] - a[1] * a[8]) * id);
  o[2] = (V)((a[1] * a[5] - a[2] * a[4]) * id);
  o[3] = (V)(c1 * id);
  o[4] = (V)((a[0] * a[8] - a[2] * a[6]) * id);
  o[5] = (V)((a[2] * a[3] - a[0] * a[5]) * id);
  o[6] = (V)(c2 * id);
  o[7] = (V)((a[1] * a[6] - a[0] * a[7]) * id);
  o[8] = (V)((a[0] * a[4] - a[1] * a[3]) * id);
}

// ---------------------------------------------------------------- PCG

// setup: r = b (free components), x = 0, z = M r, p = z, rz_0, ||b||^2
template <class V>
__global__ void k_pcg_init(int nd, const double* __restrict__ b, const int* __restrict__ mask,
                           const V* __restrict__ Dinv, V* x, V* r, V* z, V* p, Scal* sc) {
  __shared__ double sh[32];
  double rz = 0.0, bb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
    int mk = mask[i];
    V rv[3];
    for (int c = 0; c < 3; ++c) {
      rv[c] = ((mk >> c) & 1) ? (V)0 : (V)b[3 * (size_t)i + c];
      r[3 * (size_t)i + c] = rv[c];
      x[3 * (size_t)i + c] = (V)0;
      bb += (double)rv[c] * (double)rv[c];
    }
    const V* D = Dinv + 9 * (size_t)i;
    for (int c = 0; c < 3; ++c) {
      V zc = D[3 * c] * rv[0] + D[3 * c + 1] * rv[1] + D[3 * c + 2] * rv[2];
      z[3 * (size_t)i + c] = zc;
      p[3 * (size_t)i + c] = zc;
      rz += (double)rv[c] * (double)zc;
    }
  }
  rz = block_sum(rz, sh);
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&sc->rz[0], rz);
    atomicAdd(&sc->bb, bb);
  }
}

// q = K p, pq_0
template <class T, class V>
__global__ void k_pcg_q0(int nd, const int* __restrict__ rp, const int* __restrict__ col,
                         const T* __restrict__ K, const V* __restrict__ p, V* q, Scal* sc) {
  __shared__ double sh[32];
  int r = blockIdx.x * SW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  double part = 0.0;
  if (r < nd) {
    V y0, y1, y2;
    row_dot<T, V, V>(r, lane, rp, col, K, p, y0, y1, y2);
    if (lane < 3) {
      V y = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
      q[3 * (size_t)r + lane] = y;
      part = (double)y * (double)p[3 * (size_t)r + lane];
    }
  }
  part = block_sum(part, sh);
  if (threadIdx.x == 0) atomicAdd(&sc->pq[0], part);
}

// A_k: alpha = rz_k/pq_k; x += alpha p; r -= alpha q; z = M r; rz_{k+1}, rr_{k+1}
template <class V>
__global__ void k_pcg_a(int nd, int k, const V* __restrict__ Dinv, V* x, V* r, V* z,
                        const V* __restrict__ p, const V* __restrict__ q, Scal* sc) {
  __shared__ double sh[32];
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
    V rv[3];
    for (int c = 0; c < 3; ++c) {
      size_t j = 3 * (size_t)i + c;
      x[j] += alpha * p[j];
      rv[c] = r[j] - alpha * q[j];
      r[j] = rv[c];
      rr += (double)rv[c] * (double)rv[c];
    }
    const V* D = Dinv + 9 * (size_t)i;
    for (int c = 0; c < 3; ++c) {
      V zc = D[3 * c] * rv[0] + D[3 * c + 1] * rv[1] + D[3 * c + 2] * rv[2];
      z[3 * (size_t)i + c] = zc;
      rz += (double)rv[c] * (double)zc;
    }
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&sc->rz[i1], rz);
    atomicAdd(&sc->rr[i1], rr);
  }
}

// B_k: converged? else beta = rz_{k+1}/rz_k; w = K z; p = z + beta p;
// q = w + beta q; pq_{k+1}
template <class T, class V>
__global__ void k_pcg_b(int nd, int k, const int* __restrict__ rp, const int* __restrict__ col,
                        const T* __restrict__ K, const V* __restrict__ z, V* p, V* q, Scal* sc) {
  __shared__ double sh[32];
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
  int r = blockIdx.x * SW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  double part = 0.0;
  if (r < nd) {
    V y0, y1, y2;
    row_dot<T, V, V>(r, lane, rp, col, K, z, y0, y1, y2);
    if (lane < 3) {
      V y = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
      size_t j = 3 * (size_t)r + lane;
      V pn = z[j] + beta * p[j];
      V qn = y + beta * q[j];
      p[j] = pn;
      q[j] = qn;
      part = (double)pn * (double)qn;
    }
  }
  part = block_sum(part, sh);
  if (threadIdx.x == 0) atomicAdd(&sc->pq[i1], part);
}

// ---------------------------------------------------------------- BiCGStab

// generic y = K x (+ optional dots a.y into slot and y.y into slot2).  Skipped
// once the solve is done, or (check_s) once the half-step residual s has converged.
template <class T>
__global__ void k_spmv_dot(int nd, const int* __restrict__ rp, const int* __restrict__ col,
                           const T* __restrict__ K, const double* __restrict__ x, double* y,
                           const double* __restrict__ a, double* slot, double* slot2,
                           const Scal* sc, int check_s) {
  __shared__ double sh[32];
  if (sc->done || (check_s && sc->a[5] <= sc->thr)) return;
  int r = blockIdx.x * SW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  double p1 = 0.0, p2 = 0.0;
  if (r < nd) {
    double y0, y1, y2;
    row_dot<T, double, double>(r, lane, rp, col, K, x, y0, y1, y2);
    if (lane < 3) {
      double v = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
      size_t j = 3 * (size_t)r + lane;
      y[j] = v;
      if (a) p1 = a[j] * v;
      p2 = v * v;
    }
  }
  if (slot) {
    p1 = block_sum(p1, sh);
    if (threadIdx.x == 0) atomicAdd(slot, p1);
  }
  if (slot2) {
    p2 = block_sum(p2, sh);
    if (threadIdx.x == 0) atomicAdd(slot2, p2);
  }
}

// BiCGStab scalar slots in Scal::a: 0 rho, 1 alpha, 2 omega, 3 rho1 (r0.r),
// 4 r0.v, 5 s.s, 6 t.s, 7 t.t; rr[0] = r.r.  Only k_bicg_rotate (one thread)
// writes `done`, so no block ever sees it change within a launch.
__global__ void k_bicg_p(int nd, double* p, const double* __restrict__ r, const double* __restrict__ v,
                         double* ph, const double* __restrict__ Dinv, const Scal* sc) {
  if (sc->done) return;
  double beta = (sc->a[3] / sc->a[0]) * (sc->a[1] / sc->a[2]);
  double om = sc->a[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
    double pv[3];
    for (int c = 0; c < 3; ++c) {
      size_t j = 3 * (size_t)i + c;
      pv[c] = r[j] + beta * (p[j] - om * v[j]);
      p[j] = pv[c];
    }
    const double* D = Dinv + 9 * (size_t)i;
    for (int c = 0; c < 3; ++c) ph[3 * (size_t)i + c] = D[3 * c] * pv[0] + D[3 * c + 1] * pv[1] + D[3 * c + 2] * pv[2];
  }
}

__global__ void k_bicg_s(int nd, const double* __restrict__ r, const double* __restrict__ v, double* s,
                         double* sh_, const double* __restrict__ Dinv, Scal* sc) {
  __shared__ double sh[32];
  if (sc->done) return;
  double rv = sc->a[4];
  if (!(fabs(rv) > 0.0) || !isfinite(rv)) return;  // breakdown, recorded by k_bicg_rotate
  double alpha = sc->a[3] / rv;
  double ss = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
    double sv[3];
    for (int c = 0; c < 3; ++c) {
      size_t j = 3 * (size_t)i + c;
      sv[c] = r[j] - alpha * v[j];
      s[j] = sv[c];
      ss += sv[c] * sv[c];
    }
    const double* D = Dinv + 9 * (size_t)i;
    for (int c = 0; c < 3; ++c) sh_[3 * (size_t)i + c] = D[3 * c] * sv[0] + D[3 * c + 1] * sv[1] + D[3 * c + 2] * sv[2];
  }
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) atomicAdd(&sc->a[5], ss);
}

// converged on s: x += alpha ph (the rest of the iteration is skipped)
__global__ void k_bicg_check_s(int nd, double* x, const double* __restrict__ ph, const Scal* sc) {
  if (sc->done || !(sc->a[5] <= sc->thr)) return;
  double rv = sc->a[4];
  if (!(fabs(rv) > 0.0) || !isfinite(rv)) return;
  double alpha = sc->a[3] / rv;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nd; i += gridDim.x * blockDim.x)
    x[i] += alpha * ph[i];
}

__global__ void k_bicg_x(int nd, double* x, double* r, const double* __restrict__ ph,
                         const double* __restrict__ shv, const double* __restrict__ s,
                         const double* __restrict__ t, const double* __restrict__ r0, const Scal* sc,
                         double* next_rho1, double* next_rr) {
  __shared__ double sh[32];
  if (sc->done || sc->a[5] <= sc->thr) return;
  double rv = sc->a[4];
  if (!(fabs(rv) > 0.0) || !isfinite(rv)) return;
  double tt = sc->a[7];
  double om = tt > 0.0 ? sc->a[6] / tt : 0.0;
  double alpha = sc->a[3] / rv;
  double rr = 0.0, rho1 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nd; i += gridDim.x * blockDim.x) {
    x[i] += alpha * ph[i] + om * shv[i];
    double rvv = s[i] - om * t[i];
    r[i] = rvv;
    rr += rvv * rvv;
    rho1 += r0[i] * rvv;
  }
  rr = block_sum(rr, sh);
  rho1 = block_sum(rho1, sh);
  if (threadIdx.x == 0) {
    atomicAdd(next_rr, rr);
    atomicAdd(next_rho1, rho1);
  }
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

// r = b - K x  (FP64 x, FP64 accumulation, any matrix precision), masked; slot += r.r
template <class T>
__global__ void k_residual64(int nd, const int* __restrict__ rp, const int* __restrict__ col,
                             const T* __restrict__ K, const double* __restrict__ x,
                             const double* __restrict__ b, const int* __restrict__ mask, double* r,
                             double* slot) {
  __shared__ double sh[32];
  int rr = blockIdx.x * SW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  double part = 0.0;
  if (rr < nd) {
    double y0, y1, y2;
    row_dot<T, double, double>(rr, lane, rp, col, K, x, y0, y1, y2);
    if (lane < 3) {
      double y = lane == 0 ? y0 : (lane == 1 ? y1 : y2);
      size_t j = 3 * (size_t)rr + lane;
      double v = ((mask[rr] >> lane) & 1) ? 0.0 : b[j] - y;
      r[j] = v;
      part = v * v;
    }
  }
  part = block_sum(part, sh);
  if (threadIdx.x == 0) atomicAdd(slot, part);
}

__global__ void k_axpy_f2d(int n, double* x, const float* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)d[i];
}

__global__ void k_copy_d(int n, double* y, const double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i];
}

template <class T, class V>
int run_pcg(mpm_ctx* c, const mpm_mesh* m, const T* K, const V* Dinv, const double* b, V* x,
            double tol, int maxit, Scal* sc_d, Scal* sc_h, double* relres, int* iters) {
  cudaStream_t st = c->stream;
  int nd = m->ndof;
  V* r = grow<V>(c, c->v[4], 3 * (size_t)nd);
  V* z = grow<V>(c, c->v[5], 3 * (size_t)nd);
  V* p = grow<V>(c, c->v[6], 3 * (size_t)nd);
  V* q = grow<V>(c, c->v[7], 3 * (size_t)nd);
  const int* rp = ptr<int>(m->row_ptr);
  const int* col = ptr<int>(m->col);
  MPM_CUDA(cudaMemsetAsync(sc_d, 0, sizeof(Scal), st));
  int vb = 4 * 152;
  MPM_LAUNCH(k_pcg_init<V><<<vb, 256, 0, st>>>(nd, b, ptr<int>(m->dof_mask), Dinv, x, r, z, p, sc_d));
  MPM_LAUNCH(k_pcg_q0<T, V><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, K, p, q, sc_d));
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
      MPM_LAUNCH_P(MPM_PROF_PCG_UPDATE, k_pcg_a<V><<<vb, 256, 0, st>>>(nd, k, Dinv, x, r, z, p, q, sc_d));
      MPM_LAUNCH_P(MPM_PROF_PCG_SPMV, k_pcg_b<T, V><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, k, rp, col, K, z, p, q, sc_d));
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

template <class T>
int run_bicgstab(mpm_ctx* c, const mpm_mesh* m, const T* K, const double* Dinv, const double* b,
                 double* x, double tol, int maxit, Scal* sc_d, Scal* sc_h, double* relres,
                 int* iters) {
  cudaStream_t st = c->stream;
  int nd = m->ndof, n3 = 3 * nd;
  double* r = grow<double>(c, c->v[4], n3);
  double* r0 = grow<double>(c, c->v[5], n3);
  double* p = grow<double>(c, c->v[6], n3);
  double* v = grow<double>(c, c->v[7], n3);
  double* s = grow<double>(c, c->v[8], n3);
  double* t = grow<double>(c, c->v[9], n3);
  double* ph = grow<double>(c, c->v[10], n3);
  double* shv = grow<double>(c, c->v[11], n3);
  const int* rp = ptr<int>(m->row_ptr);
  const int* col = ptr<int>(m->col);
  const int* mask = ptr<int>(m->dof_mask);
  MPM_CUDA(cudaMemsetAsync(sc_d, 0, sizeof(Scal), st));
  MPM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n3, st));
  MPM_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * n3, st));
  MPM_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * n3, st));
  double* red = c->d_red + 40;  // rho1 / rr accumulators of the next iteration
  MPM_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
  // r = r0 = b (free), ||b||^2 via r = b - K*0
  MPM_LAUNCH_P(MPM_PROF_REFINE, k_residual64<T><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, K, x, b, mask, r, &sc_d->bb));
  MPM_LAUNCH(k_copy_d<<<grid_for(n3, 256), 256, 0, st>>>(n3, r0, r));
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
  int vb = 4 * 152, it = 0;
  const int batch = 16;
  while (it < maxit) {
    int iend = std::min(maxit, it + batch);
    for (; it < iend; ++it) {
      MPM_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
      MPM_LAUNCH(k_bicg_p<<<vb, 256, 0, st>>>(nd, p, r, v, ph, Dinv, sc_d));
      MPM_LAUNCH_P(MPM_PROF_BICG_SPMV, k_spmv_dot<T><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, K, ph, v, r0, &sc_d->a[4],
                                                          nullptr, sc_d, 0));
      MPM_LAUNCH(k_bicg_s<<<vb, 256, 0, st>>>(nd, r, v, s, shv, Dinv, sc_d));
      MPM_LAUNCH(k_bicg_check_s<<<vb, 256, 0, st>>>(nd, x, ph, sc_d));
      MPM_LAUNCH_P(MPM_PROF_BICG_SPMV, k_spmv_dot<T><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, K, shv, t, s, &sc_d->a[6],
                                                          &sc_d->a[7], sc_d, 1));
      MPM_LAUNCH(k_bicg_x<<<vb, 256, 0, st>>>(nd, x, r, ph, shv, s, t, r0, sc_d, red, red + 1));
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

}  // namespace

void solve(mpm_ctx* c, const mpm_mesh* mc, const mpm_material& mat, const void* K,
           const double* b, double* x, const mpm_solve_params& prm, mpm_solve_stats* out) {
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  cudaStream_t st = c->stream;
  int nd = m->ndof, n3 = 3 * nd;
  const int* rp = ptr<int>(m->row_ptr);
  const int* col = ptr<int>(m->col);
  int method = prm.method;
  if (method == 0) method = (mat.model == 2 && mat.psi != mat.phi) ? 2 : 1;
  Scal* sc_d = grow<Scal>(c, c->v[20], 1);
  Scal* sc_h = (Scal*)(c->h_red + 32);  // pinned, 32 doubles fit Scal
  static_assert(sizeof(Scal) <= 32 * sizeof(double), "scalar block too large");
  out->iterations = 0;
  out->refinements = 0;
  out->status = MPM_OK;
  if (prm.precision == MPM_FP64) {
    const double* Kd = (const double*)K;
    double* Dinv = grow<double>(c, c->v[3], 9 * (size_t)nd);
    MPM_LAUNCH(k_block_jacobi<double, double><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, Kd, Dinv, c->d_err));
    int its = 0;
    double rel = 0.0;
    int s = method == 1 ? run_pcg<double, double>(c, m, Kd, Dinv, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its)
                        : run_bicgstab<double>(c, m, Kd, Dinv, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its);
    out->iterations = its;
    out->relres = rel;
    out->status = s;
    if (s)
      set_error(c, std::string(method == 1 ? "PCG" : "BiCGStab") + " did not reach the tolerance (" +
                       std::to_string(its) + " iterations, relative residual " +
                       std::to_string(rel) + (sc_h->breakdown ? ", breakdown)" : ")"));
    return;
  }
  // mixed: FP32 inner solves inside FP64 iterative refinement
  const float* Kf = (const float*)K;
  double inner = prm.inner_tol > 0 ? prm.inner_tol : 1e-3;
  double* r64 = grow<double>(c, c->v[12], n3);
  float* d32 = grow<float>(c, c->v[13], n3);
  double* slot = c->d_red + 44;
  if (method == 1) {
    float* Dinv = grow<float>(c, c->v[3], 9 * (size_t)nd);
    MPM_LAUNCH(k_block_jacobi<float, float><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, Kf, Dinv, c->d_err));
    MPM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n3, st));
    MPM_CUDA(cudaMemsetAsync(slot, 0, sizeof(double), st));
    MPM_LAUNCH_P(MPM_PROF_REFINE, k_residual64<float><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, Kf, x, b, ptr<int>(m->dof_mask), r64, slot));
    MPM_CUDA(cudaMemcpyAsync(c->h_red + 60, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    double bb = c->h_red[60], rr = bb;
    int total = 0, rounds = 0, status = MPM_OK;
    while (rr > prm.tol * prm.tol * bb && rr > 0.0) {
      if (total >= prm.maxit || rounds >= 50) {
        status = MPM_ERR_KRYLOV;
        break;
      }
      int its = 0;
      double rel = 0.0;
      int s = run_pcg<float, float>(c, m, Kf, Dinv, r64, d32, inner, prm.maxit - total, sc_d, sc_h, &rel, &its);
      total += its;
      ++rounds;
      if (s && its == 0) {
        status = MPM_ERR_KRYLOV;
        break;
      }
      MPM_LAUNCH(k_axpy_f2d<<<grid_for(n3, 256), 256, 0, st>>>(n3, x, d32));
      MPM_CUDA(cudaMemsetAsync(slot, 0, sizeof(double), st));
      MPM_LAUNCH_P(MPM_PROF_REFINE, k_residual64<float><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, Kf, x, b, ptr<int>(m->dof_mask), r64, slot));
      MPM_CUDA(cudaMemcpyAsync(c->h_red + 60, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
      MPM_CUDA(cudaStreamSynchronize(st));
      rr = c->h_red[60];
    }
    out->iterations = total;
    out->refinements = rounds;
    out->relres = bb > 0 ? sqrt(rr / bb) : 0.0;
    out->status = status;
    if (status) set_error(c, "mixed-precision refinement did not reach the tolerance");
    return;
  }
  // non-symmetric mixed: BiCGStab on the FP32 matrix with FP64 vectors
  double* Dinv = grow<double>(c, c->v[3], 9 * (size_t)nd);
  MPM_LAUNCH(k_block_jacobi<float, double><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, Kf, Dinv, c->d_err));
  int its = 0;
  double rel = 0.0;
  int s = run_bicgstab<float>(c, m, Kf, Dinv, b, x, prm.tol, prm.maxit, sc_d, sc_h, &rel, &its);
  out->iterations = its;
  out->relres = rel;
  out->status = s;
  if (s)
    set_error(c, "BiCGStab (FP32 matrix) did not reach the tolerance (" + std::to_string(its) +
                     " iterations, relative residual " + std::to_string(rel) +
                     (sc_h->breakdown ? ", breakdown)" : ")"));
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

constexpr int kMaxDevices = 64;
unsigned char* g_pcg_scratch_dev[kMaxDevices] = {};

// device address of g_pcg_scratch on the current device (looked up once per device)
unsigned char* static_scratch(mpm_ctx* c) {
  int dev = 0;
  MPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw CudaError(MPM_ERR_ARG, "device ordinal out of range");
  if (!g_pcg_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
    if (e != cudaSuccess)
      throw CudaError(MPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_pcg_scratch_dev[dev] = (unsigned char*)p;
  }
  return g_pcg_scratch_dev[dev];
}

}  // namespace

}  // namespace mpm

using namespace mpm;

extern "C" int mpm_solve_static(mpm_ctx* c, const mpm_mesh* m, const double* K, const double* rhs,
                                double* x, double tol, int maxit, mpm_solve_stats* stats) {
  if (!c || !m || !K || !rhs || !x || !m->built || !(tol > 0) || maxit <= 0) return MPM_ERR_ARG;
  int nd = m->ndof;
  // layout: scalars (256 B), then r, z, p, q (3 nd each) and the 3x3 inverses (9 nd)
  size_t need = 256 + sizeof(double) * (size_t)nd * (4 * 3 + 9);
  if (need > kStaticBytes) {
    set_error(c, "mpm_solve_static: " + std::to_string(nd) + " dofs need " + std::to_string(need) +
                     " bytes of scratch, the static array holds " + std::to_string(kStaticBytes) +
                     " (at most " + std::to_string((kStaticBytes - 256) / (21 * sizeof(double))) +
                     " dofs)");
    return MPM_ERR_ARG;
  }
  try {
    cudaStream_t st = c->stream;
    unsigned char* base = static_scratch(c);
    Scal* sc = (Scal*)base;
    double* r = (double*)(base + 256);
    double* z = r + 3 * (size_t)nd;
    double* p = z + 3 * (size_t)nd;
    double* q = p + 3 * (size_t)nd;
    double* Dinv = q + 3 * (size_t)nd;
    const int* rp = ptr<int>(m->row_ptr);
    const int* col = ptr<int>(m->col);
    // the array keeps the previous call's contents: every vector below is
    // written before it is read, and the scalars start from zero
    MPM_CUDA(cudaMemsetAsync(sc, 0, sizeof(Scal), st));
    MPM_LAUNCH(k_block_jacobi<double, double><<<grid_for(nd, 256), 256, 0, st>>>(nd, rp, col, K, Dinv, c->d_err));
    int vb = 4 * 152;
    MPM_LAUNCH(k_pcg_init<double><<<vb, 256, 0, st>>>(nd, rhs, ptr<int>(m->dof_mask), Dinv, x, r, z, p, sc));
    MPM_LAUNCH(k_pcg_q0<double, double><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, rp, col, K, p, q, sc));
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
          MPM_LAUNCH(k_pcg_a<double><<<vb, 256, 0, st>>>(nd, k, Dinv, x, r, z, p, q, sc));
          MPM_LAUNCH(k_pcg_b<double, double><<<grid_for(nd, SW), 32 * SW, 0, st>>>(nd, k, rp, col, K, z, p, q, sc));
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
