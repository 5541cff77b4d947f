// One load step or Newmark time step (Sec. 2.4): rebuild the mesh for the body
// pose (Sec. 5), Newton-Raphson with the line search (with a free rigid body's
// increment among the unknowns), then the point update.
#include <algorithm>
#include <cmath>
#include <string>

#include "mpm_internal.cuh"

namespace mpm {
namespace {

// y = a + eta b (y may alias a)
__global__ void k_axpy_out(int n, double* y, const double* a, double eta, const double* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] + eta * b[i];
}

__global__ void k_neg(int n, double* y, const double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = -x[i];
}

// a . b over n entries by the fixed-order grid sum into *out (zeroed first)
__global__ void k_dot(int n, const double* __restrict__ a, const double* __restrict__ b, double* out,
                      GridRed gr) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += a[i] * b[i];
  grid_sum1(s, out, gr);
}

// host LU with partial pivoting of the small Schur system (n <= 6), in place
bool small_solve(int n, double* A, double* b) {
  for (int k = 0; k < n; ++k) {
    int pm = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[pm * n + k])) pm = i;
    if (A[pm * n + k] == 0.0) return false;
    if (pm != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[pm * n + j]);
      std::swap(b[k], b[pm]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double sm = b[i];
    for (int j = i + 1; j < n; ++j) sm -= A[i * n + j] * b[j];
    b[i] = sm / A[i * n + i];
  }
  return true;
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  void start() { cudaEventRecord(a, s); }
  double stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

}  // namespace

// the contact candidates' extra band for a free body over a time step of dt
// (beyond the 4 finest cells every build keeps): twice its motion at constant
// velocity and under gravity alone
double free_body_band(const mpm_rigid& bd, const mpm_material& mat, double dt) {
  double v2 = 0.0, g2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    v2 += bd.v[d] * bd.v[d];
    g2 += mat.g[d] * mat.g[d];
  }
  return 2.0 * (sqrt(v2) * dt + sqrt(g2) * dt * dt);
}

}  // namespace mpm

namespace mpm {

// Newton-Raphson with the line search of Sec. 2.4 on a built mesh; leaves the
// converged increment in du (device [3*ndof], grown in c->v[14]).  A time step
// (prm->dt > 0) adds the Newmark inertia; a free body adds its increment q to
// the unknowns, eliminated per iteration through the coupling blocks (one
// extra solve per free component; see mpm_step in the header).
void newton(mpm_ctx* c, mpm_mesh* m, const mpm_material* mat, const mpm_rigid& bd,
            const mpm_step_params* prm, mpm_step_stats& st, double** du_out) {
  cudaStream_t s = c->stream;
  Timer tm(s);
  int status = MPM_OK;
    int n3 = 3 * m->ndof;
    int prec = prm->lin.precision;
    double* du = grow<double>(c, c->v[14], n3);
    double* R = grow<double>(c, c->v[15], n3);
    double* Rt = grow<double>(c, c->v[16], n3);
    double* dx = grow<double>(c, c->v[17], n3);
    double* trial = grow<double>(c, c->v[18], n3);
    double* rhs = grow<double>(c, c->v[19], n3);
    void* K = grow_bytes(c, c->v[21], (size_t)m->nslot * 9 * (prec == MPM_MIXED ? 4 : 8));
    MPM_CUDA(cudaMemsetAsync(du, 0, sizeof(double) * n3, s));
    // the time step and the free body's unknowns
    int fb[6], nb = 0;
    for (int j = 0; j < 6; ++j)
      if (bd.free & (1 << j)) fb[nb++] = j;
    Dyn dyn;
    dyn.dt = prm->dt;
    dyn.body = nb > 0;
    for (int d = 0; d < 3; ++d) dyn.q[d] = (bd.free & (1 << d)) ? 0.0 : bd.step_d[d];
    const Dyn* dp = (prm->dt > 0.0 || nb) ? &dyn : nullptr;
    double *Z = nullptr, *dots = nullptr;
    if (nb) {
      dyn.Kgb = grow<double>(c, c->v[24], 6 * (size_t)n3);
      dyn.Kbg = grow<double>(c, c->v[25], 6 * (size_t)n3);
      Z = grow<double>(c, c->v[26], 6 * (size_t)n3);
      dots = grow<double>(c, c->v[27], 64);
    }
    double wref = 0.0;
    for (int d = 0; d < 3 && nb; ++d) wref += pow(bd.mass * prm->load * mat->g[d], 2.0);
    wref = sqrt(wref);
    auto body_norm = [&](double r, const AsmOut& oo) {
      for (int j = 0; j < nb; ++j) r = hypot(r, oo.Rb[fb[j]]);
      return r;
    };
    AsmOut o{};
    tm.start();
    assemble(c, m, *mat, bd, du, prm->load, prec, R, nullptr, &o, true, false, dp);
    st.ms_assemble += tm.stop();
    status = check_device_error(c, "assembly");
    if (status) throw CudaError(status, c->err);
    double rn = body_norm(sqrt(c->h_red[16]), o);
    bool conv = false;
    for (int it = 0; it <= prm->maxit; ++it) {
      double fref = std::max(std::max(o.fint_norm, o.fextc_norm), std::max(o.finert_norm, wref));
      st.res_hist[it] = fref > 0 ? rn / fref : rn;
      for (int d = 0; d < 3; ++d) st.reaction[d] = o.reaction[d];
      if (rn <= prm->tol * fref || fref == 0.0) {
        conv = true;
        st.newton_its = it;
        break;
      }
      if (it == prm->maxit) break;
      // consistent tangent at the current increment, built from the state that
      // the last residual evaluation (at this increment) left; R stays as it is
      tm.start();
      assemble(c, m, *mat, bd, du, prm->load, prec, R, K, &o, false, true, dp);
      st.ms_assemble += tm.stop();
      status = check_device_error(c, "tangent assembly");
      if (status) throw CudaError(status, c->err);
      MPM_LAUNCH(k_neg<<<grid_for(n3, 256), 256, 0, s>>>(n3, rhs, R));
      mpm_solve_stats ss{};
      tm.start();
      solve(c, m, *mat, K, rhs, dx, prm->lin, &ss);
      st.lin_its += ss.iterations;
      status = check_device_error(c, "linear solve");
      if (status) throw CudaError(status, c->err);
      if (ss.status) throw CudaError(ss.status, c->err);
      double dq[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (nb) {
        // Z_l = K^-1 dR/dq_l, then the Schur system of the free components
        for (int l = 0; l < nb; ++l) {
          mpm_solve_stats sz{};
          solve(c, m, *mat, K, dyn.Kgb + (size_t)fb[l] * n3, Z + (size_t)l * n3, prm->lin, &sz);
          st.lin_its += sz.iterations;
          status = check_device_error(c, "linear solve");
          if (status) throw CudaError(status, c->err);
          if (sz.status) throw CudaError(sz.status, c->err);
        }
        MPM_CUDA(cudaMemsetAsync(dots, 0, 64 * sizeof(double), s));
        int gb = std::min(grid_for(n3, 256), 4 * 152);
        for (int j = 0; j < nb; ++j) {
          const double* kr = dyn.Kbg + (size_t)fb[j] * n3;
          MPM_LAUNCH(k_dot<<<gb, 256, 0, s>>>(n3, kr, dx, dots + 7 * j, grid_red(c, 1, gb)));
          for (int l = 0; l < nb; ++l)
            MPM_LAUNCH(k_dot<<<gb, 256, 0, s>>>(n3, kr, Z + (size_t)l * n3, dots + 7 * j + 1 + l,
                                               grid_red(c, 1, gb)));
        }
        double hd[64];
        MPM_CUDA(cudaMemcpyAsync(hd, dots, sizeof(hd), cudaMemcpyDeviceToHost, s));
        MPM_CUDA(cudaStreamSynchronize(s));
        double Sm[36], rb[6];
        for (int j = 0; j < nb; ++j) {
          rb[j] = -o.Rb[fb[j]] - hd[7 * j];
          for (int l = 0; l < nb; ++l) Sm[nb * j + l] = o.Kbb[6 * fb[j] + fb[l]] - hd[7 * j + 1 + l];
        }
        if (!small_solve(nb, Sm, rb)) throw CudaError(MPM_ERR_KRYLOV, "singular rigid-body Schur system");
        for (int l = 0; l < nb; ++l) {
          dq[fb[l]] = rb[l];
          MPM_LAUNCH(k_axpy_out<<<grid_for(n3, 256), 256, 0, s>>>(n3, dx, dx, -rb[l], Z + (size_t)l * n3));
        }
      }
      st.ms_solve += tm.stop();
      // line search (Sec. 2.4): eta = 1, else the lowest residual of {0.5, 0.25, 0.1}
      const double etas[4] = {1.0, 0.5, 0.25, 0.1};
      double best = -1.0, beta_ = 1.0;
      int ibest = 0, ilast = 0;
      AsmOut obest{};
      tm.start();
      for (int e = 0; e < 4; ++e) {
        MPM_LAUNCH(k_axpy_out<<<grid_for(n3, 256), 256, 0, s>>>(n3, trial, du, etas[e], dx));
        Dyn dt_ = dyn;
        dt_.Kgb = dt_.Kbg = nullptr;
        for (int j = 0; j < 6; ++j) dt_.q[j] = dyn.q[j] + etas[e] * dq[j];
        AsmOut ot{};
        assemble(c, m, *mat, bd, trial, prm->load, prec, Rt, nullptr, &ot, true, false, dp ? &dt_ : nullptr);
        double r1 = body_norm(sqrt(c->h_red[16]), ot);
        int es = check_device_error(c, "line search");
        if (es) r1 = INFINITY;
        ilast = e;
        if (best < 0.0 || r1 < best) {
          best = r1;
          beta_ = etas[e];
          ibest = e;
          obest = ot;
        }
        if (e == 0 && r1 < rn) break;
      }
      st.eta_hist[it] = beta_;
      MPM_LAUNCH(k_axpy_out<<<grid_for(n3, 256), 256, 0, s>>>(n3, du, du, beta_, dx));
      for (int j = 0; j < 6; ++j) dyn.q[j] += beta_ * dq[j];
      if (ibest == ilast && std::isfinite(best)) {
        std::swap(R, Rt);  // the accepted trial's residual is the last one computed
        o = obest;
        rn = best;
      } else {
        assemble(c, m, *mat, bd, du, prm->load, prec, R, nullptr, &o, true, false, dp);
        status = check_device_error(c, "assembly");
        if (status) throw CudaError(status, c->err);
        rn = body_norm(sqrt(c->h_red[16]), o);
      }
      st.ms_assemble += tm.stop();
    }
    if (!conv) {
      st.newton_its = prm->maxit;
      throw CudaError(MPM_ERR_NEWTON, "Newton iterations exhausted");
    }
    for (int j = 0; j < 6; ++j) st.body_q[j] = dyn.q[j];
    if (nb) {
      double dt = prm->dt, c2 = 2.0 / (dt * dt), qn = 0.0;
      for (int d = 0; d < 3; ++d) {
        st.body_v[d] = bd.v[d] + dt * (c2 * (dyn.q[d] - dt * bd.v[d]));
        st.body_w[d] = bd.w[d] + dt * (c2 * (dyn.q[3 + d] - dt * bd.w[d]));
        qn += dyn.q[d] * dyn.q[d];
      }
      if (sqrt(qn) > free_body_band(bd, *mat, dt))
        throw CudaError(MPM_ERR_SUPPORT, "the free body moved farther than the contact candidates' band "
                                         "allows; take a smaller time step");
    }
  *du_out = du;
}

}  // namespace mpm

using namespace mpm;

extern "C" int mpm_step(mpm_ctx* c, const mpm_domain* dom, const mpm_rigid* body,
                        const mpm_adapt* ad, const mpm_material* mat, mpm_points* pts,
                        const mpm_step_params* prm, mpm_step_stats* stats) {
  if (!c || !dom || !ad || !mat || !pts || !prm) return MPM_ERR_ARG;
  if (!(prm->tol > 0) || prm->maxit < 0 || prm->maxit > 63) {
    set_error(c, "step: need tol > 0 and 0 <= maxit <= 63");
    return MPM_ERR_ARG;
  }
  mpm_step_stats st{};
  mpm_rigid nob{};
  const mpm_rigid& bd = body ? *body : nob;
  if (!(prm->dt >= 0.0) || (prm->dt > 0.0 && !pts->v)) {
    set_error(c, "step: need dt >= 0, and point velocities for a time step");
    return MPM_ERR_ARG;
  }
  if (bd.free && (!(prm->dt > 0.0) || bd.kind == 0 || !mat->contact_on || !(bd.mass > 0.0) ||
                  (bd.free & ~63) || ((bd.free & 56) && (bd.kind != 4 || !(bd.inertia > 0.0))))) {
    set_error(c, "step: a free body needs a time step, contact, a mass, and for free rotation a sphere "
                 "with a rotational inertia");
    return MPM_ERR_ARG;
  }
  int status = MPM_OK;
  try {
    cudaStream_t s = c->stream;
    Timer tm(s);
    if (!c->step_mesh) {
      c->step_mesh = new mpm_mesh();
      c->step_mesh->ctx = c;
    }
    mpm_mesh* m = c->step_mesh;
    tm.start();
    build_mesh(c, m, *dom, bd, *ad, *mat, pts, 0, bd.free ? free_body_band(bd, *mat, prm->dt) : 0.0);
    status = check_device_error(c, "mesh build");
    st.ms_build = tm.stop();
    st.npts = m->np;
    st.ndof = m->ndof;
    st.nnzb = m->nnzb;
    st.nsrc = m->nsrc;
    st.npair = m->npair;
    st.nslot = m->nslot;
    if (status) throw CudaError(status, c->err);
    double* du = nullptr;
    newton(c, m, mat, bd, prm, st, &du);
    if (m->mg && m->mg->gen == m->gen && m->mg->nlev > 0) {
      st.mg_rows1 = m->mg->lev[0].nrow;
      st.mg_stencil1 = m->mg->lev[0].S;
    }
    if (prm->du_out) {
      long long n3 = 3LL * m->ndof;
      if (n3 > prm->du_capacity)
        throw CudaError(MPM_ERR_CAPACITY, "step: du_out holds " + std::to_string(prm->du_capacity) +
                                              " doubles, the increment has " + std::to_string(n3));
      MPM_CUDA(cudaMemcpyAsync(prm->du_out, du, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s));
    }
    tm.start();
    point_update(c, m, *mat, du, pts, prm->dt);
    status = check_device_error(c, "point update");
    st.ms_update = tm.stop();
    if (status) throw CudaError(status, c->err);
  } catch (const CudaError& e) {
    set_error(c, e.what());
    status = e.code;
  } catch (const std::exception& e) {
    set_error(c, e.what());
    status = MPM_ERR_ARG;
  }
  st.status = status;
  if (stats) *stats = st;
  return status;
}
