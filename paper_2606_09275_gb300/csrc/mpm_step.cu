// One quasi-static load step (Sec. 2.4): rebuild the mesh for the body pose
// (Sec. 5), Newton-Raphson with the line search, then the point update.
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
}  // namespace mpm

namespace mpm {

// Newton-Raphson with the line search of Sec. 2.4 on a built mesh; leaves the
// converged increment in du (device [3*ndof], grown in c->v[14]).
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
    AsmOut o{};
    tm.start();
    assemble(c, m, *mat, bd, du, prm->load, prec, R, nullptr, &o, true);
    st.ms_assemble += tm.stop();
    status = check_device_error(c, "assembly");
    if (status) throw CudaError(status, c->err);
    double rn = sqrt(c->h_red[16]);
    bool conv = false;
    for (int it = 0; it <= prm->maxit; ++it) {
      double fref = std::max(o.fint_norm, o.fextc_norm);
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
      assemble(c, m, *mat, bd, du, prm->load, prec, R, K, &o, false, true);
      st.ms_assemble += tm.stop();
      status = check_device_error(c, "tangent assembly");
      if (status) throw CudaError(status, c->err);
      MPM_LAUNCH(k_neg<<<grid_for(n3, 256), 256, 0, s>>>(n3, rhs, R));
      mpm_solve_stats ss{};
      tm.start();
      solve(c, m, *mat, K, rhs, dx, prm->lin, &ss);
      st.ms_solve += tm.stop();
      st.lin_its += ss.iterations;
      status = check_device_error(c, "linear solve");
      if (status) throw CudaError(status, c->err);
      if (ss.status) throw CudaError(ss.status, c->err);
      // line search (Sec. 2.4): eta = 1, else the lowest residual of {0.5, 0.25, 0.1}
      const double etas[4] = {1.0, 0.5, 0.25, 0.1};
      double best = -1.0, beta_ = 1.0;
      int ibest = 0, ilast = 0;
      AsmOut obest{};
      tm.start();
      for (int e = 0; e < 4; ++e) {
        MPM_LAUNCH(k_axpy_out<<<grid_for(n3, 256), 256, 0, s>>>(n3, trial, du, etas[e], dx));
        AsmOut ot{};
        assemble(c, m, *mat, bd, trial, prm->load, prec, Rt, nullptr, &ot, true);
        double r1 = sqrt(c->h_red[16]);
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
      if (ibest == ilast && std::isfinite(best)) {
        std::swap(R, Rt);  // the accepted trial's residual is the last one computed
        o = obest;
        rn = best;
      } else {
        assemble(c, m, *mat, bd, du, prm->load, prec, R, nullptr, &o, true);
        status = check_device_error(c, "assembly");
        if (status) throw CudaError(status, c->err);
        rn = sqrt(c->h_red[16]);
      }
      st.ms_assemble += tm.stop();
    }
    if (!conv) {
      st.newton_its = prm->maxit;
      throw CudaError(MPM_ERR_NEWTON, "Newton iterations exhausted");
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
    build_mesh(c, m, *dom, bd, *ad, *mat, pts, 0);
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
    point_update(c, m, *mat, du, pts);
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
