// Context lifetime, error reporting, mesh queries and the C ABI entry points.
#include <cstdio>
#include <cstring>
#include <vector>

#include <cstdlib>

#include "mpm_internal.cuh"

namespace mpm {

void set_error(mpm_ctx* c, const std::string& m) {
  if (c) c->err = m;
}

void sync(mpm_ctx* c) { MPM_CUDA(cudaStreamSynchronize(c->stream)); }

// Reads and clears the device error word; maps its bits to a status.
int check_device_error(mpm_ctx* c, const char* where) {
  MPM_CUDA(cudaMemcpyAsync(c->h_int + 1, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MPM_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  int e = c->h_int[1];
  if (!e) return MPM_OK;
  int st = MPM_ERR_SUPPORT;
  const char* what = "support/overlap/constraint list overflow";
  if (e & EB_NAN) {
    st = MPM_ERR_NAN;
    what = "non-finite value or non-positive det F";
  } else if (e & EB_DOMAIN) {
    st = MPM_ERR_DOMAIN;
    what = "a GIMP domain lies outside the cube";
  } else if (e & EB_BALANCE) {
    st = MPM_ERR_BALANCE;
    what = "hanging node not at an edge or face midpoint (unbalanced octree)";
  } else if (e & EB_KRYLOV) {
    st = MPM_ERR_KRYLOV;
    what = "Krylov breakdown";
  } else if (e & EB_ROW) {
    what = "stiffness row longer than the pattern builder holds";
  }
  set_error(c, std::string(where) + ": " + what);
  return st;
}

void prof_flush(mpm_ctx* c) {
  if (c->prof.empty()) return;
  MPM_CUDA(cudaStreamSynchronize(c->stream));
  for (ProfEv& e : c->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      c->prof_ms[e.cls] += ms;
      c->prof_n[e.cls] += 1;
    }
    c->evpool.push_back(e.a);
    c->evpool.push_back(e.b);
  }
  c->prof.clear();
}

}  // namespace mpm

using namespace mpm;

extern "C" int mpm_profile(mpm_ctx* c, int enable) {
  if (!c) return MPM_ERR_ARG;
  try {
    prof_flush(c);
  } catch (const CudaError& e) {
    set_error(c, e.what());
    return e.code;
  }
  if (enable) {
    for (int i = 0; i < MPM_PROF_NCLASS; ++i) {
      c->prof_ms[i] = 0.0;
      c->prof_n[i] = 0;
    }
  }
  c->prof_on = enable != 0;
  return MPM_OK;
}

extern "C" int mpm_profile_read(mpm_ctx* c, long long* launches, double* ms) {
  if (!c || !launches || !ms) return MPM_ERR_ARG;
  try {
    prof_flush(c);
  } catch (const CudaError& e) {
    set_error(c, e.what());
    return e.code;
  }
  for (int i = 0; i < MPM_PROF_NCLASS; ++i) {
    launches[i] = c->prof_n[i];
    ms[i] = c->prof_ms[i];
  }
  return MPM_OK;
}

extern "C" int mpm_launch_count(const mpm_ctx* c, long long* n) {
  if (!c || !n) return MPM_ERR_ARG;
  *n = c->nlaunch;
  return MPM_OK;
}

#define MPM_GUARD(ctx, ...)                                  \
  try {                                                      \
    __VA_ARGS__                                              \
  } catch (const CudaError& e) {                             \
    set_error(ctx, e.what());                                \
    return e.code;                                           \
  } catch (const std::exception& e) {                        \
    set_error(ctx, e.what());                                \
    return MPM_ERR_ARG;                                      \
  }

extern "C" int mpm_create(mpm_ctx** out, void* stream) {
  if (!out) return MPM_ERR_ARG;
  mpm_ctx* c = new mpm_ctx();
  try {
    c->stream = (cudaStream_t)stream;
    MPM_CUDA(cudaGetDevice(&c->device));
    MPM_CUDA(cudaMallocAsync((void**)&c->d_err, sizeof(int), c->stream));
    MPM_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    MPM_CUDA(cudaMallocAsync((void**)&c->d_red, 64 * sizeof(double), c->stream));
    // CUDA graphs for the V-cycle (MPM_GRAPHS=0 in the environment: plain
    // launches, for comparison)
    const char* eg = getenv("MPM_GRAPHS");
    if (!(eg && eg[0] == '0')) MPM_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    MPM_CUDA(cudaMallocAsync((void**)&c->d_ticket, 16, c->stream));
    MPM_CUDA(cudaMemsetAsync(c->d_ticket, 0, 16, c->stream));
    grid_red(c, 4, 4096);
    MPM_CUDA(cudaMallocHost((void**)&c->h_red, 64 * sizeof(double)));
    MPM_CUDA(cudaMallocHost((void**)&c->h_int, 64 * sizeof(int)));
    MPM_CUDA(cudaStreamSynchronize(c->stream));
  } catch (const CudaError& e) {
    int code = e.code;
    delete c;
    *out = nullptr;
    return code;
  }
  *out = c;
  return MPM_OK;
}

namespace mpm {
void mesh_release(mpm_mesh* m) {
  mpm_ctx* c = m->ctx;
  mg_release(c, m);
  for (SplitRound& r : m->split_log) {
    free_buf(c, r.flag);
    free_buf(c, r.rank);
  }
  m->split_log.clear();
  Buf* bufs[] = {&m->leaf_key, &m->leaf_lev, &m->leaf_tmp_key, &m->leaf_tmp_lev, &m->flag,
                 &m->scan, &m->node_key, &m->corner, &m->hang, &m->owner, &m->cptr, &m->cidx,
                 &m->cw, &m->node_dof, &m->dof_node, &m->dof_mask, &m->perm, &m->pcell, &m->px,
                 &m->plp, &m->pl0, &m->pF, &m->pbe, &m->pV0, &m->pmass, &m->pE, &m->pys,
                 &m->nsup, &m->sidx, &m->S, &m->dS, &m->populated, &m->betaK,
                 &m->isB, &m->gface, &m->gdof, &m->gn, &m->row_ptr, &m->col, &m->kg, &m->rowcnt,
                 &m->src_key, &m->src_ptr, &m->fext, &m->cand, &m->cb_n, &m->cb_idx, &m->cb_phi,
                 &m->cb_y0, &m->dF, &m->dFinv, &m->tau, &m->Aalg, &m->gx, &m->slice_w, &m->slice_base, &m->scol, &m->srow, &m->spos,
                 &m->lawst, &m->ct_row, &m->ct_ptr, &m->ct_ent, &m->cc_f, &m->cc_k, &m->cc_on,
                 &m->gJ, &m->gcoef, &m->Mf, &m->V0t, &m->dS32, &m->pv, &m->cc_t, &m->cc_d, &m->cc_b, &m->pma, &m->tri_fn, &m->tri_en, &m->tri_vn};
  for (Buf* b : bufs) free_buf(c, *b);
}
}  // namespace mpm

extern "C" int mpm_destroy(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  if (c->step_mesh) {
    mesh_release(c->step_mesh);
    delete c->step_mesh;
  }
  for (mpm_mesh* m : c->meshes) {
    mesh_release(m);
    delete m;
  }
  c->meshes.clear();
  free_buf(c, c->cub_tmp);
  free_buf(c, c->part);
  for (auto& b : c->tmp) free_buf(c, b);
  for (auto& b : c->v) free_buf(c, b);
  try {
    prof_flush(c);
  } catch (...) {
  }
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->d_err) cudaFreeAsync(c->d_err, c->stream);
  if (c->d_red) cudaFreeAsync(c->d_red, c->stream);
  if (c->d_ticket) cudaFreeAsync(c->d_ticket, c->stream);
  cudaStreamSynchronize(c->stream);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->h_int) cudaFreeHost(c->h_int);
  delete c;
  return MPM_OK;
}

extern "C" const char* mpm_last_error(const mpm_ctx* c) { return c ? c->err.c_str() : "no context"; }

static bool valid_domain(mpm_ctx* c, const mpm_domain* d) {
  if (!d || !(d->L > 0) || d->depth_min < 0 || d->depth_max < d->depth_min || d->depth_max > 20 ||
      d->nbc < 0 || d->nbc > 8) {
    set_error(c, "invalid domain (need L > 0, 0 <= depth_min <= depth_max <= 20, nbc <= 8)");
    return false;
  }
  for (int b = 0; b < d->nbc; ++b) {
    double v = d->bc_pos[b] * ldexp(1.0, d->depth_max) / d->L;
    if (d->bc_axis[b] < 0 || d->bc_axis[b] > 2 || fabs(v - floor(v + 0.5)) > 1e-9) {
      set_error(c, "Dirichlet plane not on a finest-grid plane");
      return false;
    }
  }
  return true;
}

extern "C" int mpm_octree_build(mpm_ctx* c, const mpm_domain* dom, const mpm_rigid* body,
                                const mpm_adapt* ad, const mpm_material* mat, mpm_points* pts,
                                int flags, mpm_mesh** mesh) {
  if (!c || !mesh || !pts || !ad || !mat) return MPM_ERR_ARG;
  if (!valid_domain(c, dom)) return MPM_ERR_ARG;
  if (pts->count <= 0 || pts->capacity < pts->count) {
    set_error(c, "invalid point arrays (count <= 0 or capacity < count)");
    return MPM_ERR_ARG;
  }
  mpm_rigid nob{};
  MPM_GUARD(c, {
    if (!*mesh) {
      *mesh = new mpm_mesh();
      (*mesh)->ctx = c;
      c->meshes.push_back(*mesh);
    }
    build_mesh(c, *mesh, *dom, body ? *body : nob, *ad, *mat, pts, flags);
    int st = check_device_error(c, "mpm_octree_build");
    if (st) return st;
    return (int)MPM_OK;
  })
}

extern "C" int mpm_mesh_free(mpm_mesh* m) {
  if (!m) return MPM_ERR_ARG;
  mpm_ctx* c = m->ctx;
  for (size_t i = 0; i < c->meshes.size(); ++i)
    if (c->meshes[i] == m) {
      c->meshes.erase(c->meshes.begin() + i);
      break;
    }
  try {
    mesh_release(m);
    cudaStreamSynchronize(c->stream);
  } catch (...) {
  }
  delete m;
  return MPM_OK;
}

extern "C" int mpm_mesh_counts(const mpm_mesh* m, mpm_mesh_info* info) {
  if (!m || !info) return MPM_ERR_ARG;
  info->nleaf = m->nleaf;
  info->nnode = m->nnode;
  info->nhang = m->nhang;
  info->ndof = m->ndof;
  info->nnzb = m->nnzb;
  info->nghost = m->nghost;
  info->npts = m->np;
  info->maxs = m->maxs;
  info->ncontact = m->ncand;
  info->maxrow = m->maxrow;
  info->nslot = (int)m->nslot;
  return MPM_OK;
}

extern "C" int mpm_blocks_export(mpm_ctx* c, const mpm_mesh* m, const void* K, int precision,
                                 double* host) {
  if (!c || !m || !K || !host || !m->built) return MPM_ERR_ARG;
  MPM_GUARD(c, {
    double* d = grow<double>(c, c->tmp[6], 9 * (size_t)m->nnzb);
    blocks_export(c, m, K, precision, d);
    MPM_CUDA(cudaMemcpyAsync(host, d, sizeof(double) * 9 * (size_t)m->nnzb, cudaMemcpyDeviceToHost, c->stream));
    MPM_CUDA(cudaStreamSynchronize(c->stream));
    return (int)MPM_OK;
  })
}

namespace {

__global__ void k_export_leaves(int n, const uint64_t* key, const int* lev, int* out_lev,
                                int* out_anchor) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (out_lev) out_lev[i] = lev[i];
  if (out_anchor) {
    int a[3];
    demorton(key[i], a);
    out_anchor[3 * i] = a[0];
    out_anchor[3 * i + 1] = a[1];
    out_anchor[3 * i + 2] = a[2];
  }
}

__global__ void k_export_node_coord(int n, const uint64_t* key, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a[3];
  demorton(key[i], a);
  out[3 * i] = a[0];
  out[3 * i + 1] = a[1];
  out[3 * i + 2] = a[2];
}

// point arrays are stored in cell order: scatter back to the caller's order
template <class T>
__global__ void k_unpermute(int np, int width, const int* perm, const T* in, T* out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)np * width) return;
  int w = (int)(i / width), k = (int)(i % width);
  out[(long long)perm[w] * width + k] = in[i];
}

}  // namespace

extern "C" int mpm_mesh_export(const mpm_mesh* mc, int what, void* dst, size_t bytes) {
  if (!mc || !dst) return MPM_ERR_ARG;
  mpm_mesh* m = const_cast<mpm_mesh*>(mc);
  mpm_ctx* c = m->ctx;
  MPM_GUARD(c, {
    size_t need = 0;
    const void* src = nullptr;
    Buf& t = c->tmp[7];
    switch (what) {
      case MPM_EXPORT_LEAF_LEVEL:
        need = sizeof(int) * m->nleaf;
        src = m->leaf_lev.p;
        break;
      case MPM_EXPORT_LEAF_ANCHOR: {
        need = sizeof(int) * 3 * m->nleaf;
        int* o = grow<int>(c, t, 3 * (size_t)m->nleaf);
        MPM_LAUNCH(k_export_leaves<<<grid_for(m->nleaf, 256), 256, 0, c->stream>>>(
            m->nleaf, ptr<uint64_t>(m->leaf_key), ptr<int>(m->leaf_lev), nullptr, o));
        src = o;
        break;
      }
      case MPM_EXPORT_NODE_COORD: {
        need = sizeof(int) * 3 * m->nnode;
        int* o = grow<int>(c, t, 3 * (size_t)m->nnode);
        MPM_LAUNCH(k_export_node_coord<<<grid_for(m->nnode, 256), 256, 0, c->stream>>>(
            m->nnode, ptr<uint64_t>(m->node_key), o));
        src = o;
        break;
      }
      case MPM_EXPORT_NODE_HANG:
        need = sizeof(int) * m->nnode;
        src = m->hang.p;
        break;
      case MPM_EXPORT_NODE_DOF:
        need = sizeof(int) * m->nnode;
        src = m->node_dof.p;
        break;
      case MPM_EXPORT_CPTR:
        need = sizeof(int) * (m->nnode + 1);
        src = m->cptr.p;
        break;
      case MPM_EXPORT_CIDX:
        need = sizeof(int) * m->ncon;
        src = m->cidx.p;
        break;
      case MPM_EXPORT_CW:
        need = sizeof(double) * m->ncon;
        src = m->cw.p;
        break;
      case MPM_EXPORT_NSUP: {
        need = sizeof(int) * m->np;
        int* o = grow<int>(c, t, m->np);
        MPM_LAUNCH(k_unpermute<int><<<grid_for(m->np, 256), 256, 0, c->stream>>>(
            m->np, 1, ptr<int>(m->perm), ptr<int>(m->nsup), o));
        src = o;
        break;
      }
      case MPM_EXPORT_SIDX: {
        need = sizeof(int) * (size_t)m->np * MAXS;
        int* o = grow<int>(c, t, (size_t)m->np * MAXS);
        MPM_LAUNCH(k_unpermute<int><<<grid_for((long long)m->np * MAXS, 256), 256, 0, c->stream>>>(
            m->np, MAXS, ptr<int>(m->perm), ptr<int>(m->sidx), o));
        src = o;
        break;
      }
      case MPM_EXPORT_S: {
        need = sizeof(double) * (size_t)m->np * MAXS;
        double* o = grow<double>(c, t, (size_t)m->np * MAXS);
        MPM_LAUNCH(k_unpermute<double><<<grid_for((long long)m->np * MAXS, 256), 256, 0, c->stream>>>(
            m->np, MAXS, ptr<int>(m->perm), ptr<double>(m->S), o));
        src = o;
        break;
      }
      case MPM_EXPORT_DS: {
        need = sizeof(double) * (size_t)m->np * MAXS * 3;
        double* o = grow<double>(c, t, (size_t)m->np * MAXS * 3);
        MPM_LAUNCH(k_unpermute<double><<<grid_for((long long)m->np * MAXS * 3, 256), 256, 0, c->stream>>>(
            m->np, MAXS * 3, ptr<int>(m->perm), ptr<double>(m->dS), o));
        src = o;
        break;
      }
      case MPM_EXPORT_ROW_PTR:
        need = sizeof(int) * (m->ndof + 1);
        src = m->row_ptr.p;
        break;
      case MPM_EXPORT_COL:
        need = sizeof(int) * m->nnzb;
        src = m->col.p;
        break;
      case MPM_EXPORT_GHOST:
        need = sizeof(double) * m->nnzb;
        src = m->kg.p;
        break;
      case MPM_EXPORT_BCMASK:
        need = sizeof(int) * m->ndof;
        src = m->dof_mask.p;
        break;
      case MPM_EXPORT_POPULATED:
        need = sizeof(int) * m->nleaf;
        src = m->populated.p;
        break;
      case MPM_EXPORT_GHOST_FACES:
        need = sizeof(int) * 4 * m->nghost;
        src = m->gface.p;
        break;
      case MPM_EXPORT_MG_LEVELS: {
        // host data: depth, rows, stencil radius, stencil size per coarse level
        int info[32] = {0};
        const MGData* G = (m->mg && m->mg->gen == m->gen) ? m->mg : nullptr;
        if (G)
          for (int l = 0; l < G->nlev; ++l) {
            info[4 * l] = G->lev[l].d;
            info[4 * l + 1] = G->lev[l].nrow;
            info[4 * l + 2] = G->lev[l].R;
            info[4 * l + 3] = G->lev[l].S;
          }
        if (bytes < sizeof(info)) {
          set_error(c, "export buffer too small");
          return (int)MPM_ERR_ARG;
        }
        memcpy(dst, info, sizeof(info));
        return (int)MPM_OK;
      }
      default:
        set_error(c, "unknown export selector");
        return (int)MPM_ERR_ARG;
    }
    if (bytes < need) {
      set_error(c, "export buffer too small");
      return (int)MPM_ERR_ARG;
    }
    if (need) MPM_CUDA(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, c->stream));
    MPM_CUDA(cudaStreamSynchronize(c->stream));
    return (int)MPM_OK;
  })
}

extern "C" int mpm_assemble(mpm_ctx* c, const mpm_mesh* m, const mpm_material* mat,
                            const mpm_rigid* body, const double* du, double load, int precision,
                            double* R, void* K, double* reaction, double* fint_norms) {
  if (!c || !m || !mat || !du || !R || !m->built) return MPM_ERR_ARG;
  if (precision != MPM_FP64 && precision != MPM_MIXED) return MPM_ERR_ARG;
  mpm_rigid nob{};
  MPM_GUARD(c, {
    AsmOut o{};
    bool host_out = reaction || fint_norms;
    assemble(c, m, *mat, body ? *body : nob, du, load, precision, R, K, &o, host_out);
    int st = check_device_error(c, "mpm_assemble");
    if (st) return st;
    if (reaction)
      for (int d = 0; d < 3; ++d) reaction[d] = o.reaction[d];
    if (fint_norms) {
      fint_norms[0] = o.fint_norm;
      fint_norms[1] = o.fextc_norm;
    }
    return (int)MPM_OK;
  })
}

extern "C" int mpm_assemble_body(mpm_ctx* c, const mpm_mesh* m, const mpm_material* mat,
                                 const mpm_rigid* body, const double* du, const double* q, double dt,
                                 double load, int precision, double* R, void* K, double* reaction,
                                 double* fint_norms, double* Rb, double* Kbb, double* Kgb, double* Kbg) {
  if (!c || !m || !mat || !body || !du || !q || !R || !m->built || !(dt > 0.0)) return MPM_ERR_ARG;
  if (precision != MPM_FP64 && precision != MPM_MIXED) return MPM_ERR_ARG;
  MPM_GUARD(c, {
    Dyn dyn;
    dyn.dt = dt;
    dyn.body = body->free != 0 && body->kind != 0;
    for (int j = 0; j < 6; ++j) dyn.q[j] = q[j];
    dyn.Kgb = Kgb;
    dyn.Kbg = Kbg;
    AsmOut o{};
    assemble(c, m, *mat, *body, du, load, precision, R, K, &o, true, false, &dyn);
    int st = check_device_error(c, "mpm_assemble_body");
    if (st) return st;
    if (reaction)
      for (int d = 0; d < 3; ++d) reaction[d] = o.reaction[d];
    if (fint_norms) {
      fint_norms[0] = o.fint_norm;
      fint_norms[1] = o.fextc_norm;
      fint_norms[2] = o.finert_norm;
    }
    if (Rb)
      for (int j = 0; j < 6; ++j) Rb[j] = o.Rb[j];
    if (Kbb)
      for (int j = 0; j < 36; ++j) Kbb[j] = o.Kbb[j];
    return (int)MPM_OK;
  })
}

extern "C" int mpm_solve(mpm_ctx* c, const mpm_mesh* m, const mpm_material* mat, const void* K,
                         const double* rhs, double* x, const mpm_solve_params* prm,
                         mpm_solve_stats* st) {
  if (!c || !m || !mat || !K || !rhs || !x || !prm || !m->built) return MPM_ERR_ARG;
  if (!(prm->tol > 0) || prm->maxit <= 0) {
    set_error(c, "solve: need tol > 0 and maxit > 0");
    return MPM_ERR_ARG;
  }
  MPM_GUARD(c, {
    mpm_solve_stats s{};
    solve(c, m, *mat, K, rhs, x, *prm, &s);
    int e = check_device_error(c, "mpm_solve");
    if (st) *st = s;
    if (e) return e;
    return s.status;
  })
}
