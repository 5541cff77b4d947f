/*
 * Oracle: assembly of Eq. (MPMweak) (static part), penalty contact (Sec. 2.3),
 * the ghost term (Sec. 4), strong Dirichlet conditions and the Newton-Raphson
 * load step with line search (Sec. 2.4).  TEST INFRASTRUCTURE ONLY.
 *
 * Readings:
 *  - load steps (dt = 0) are quasi-static: the inertia term of Eq. (MPMweak)
 *    is dropped; time steps (dt > 0) keep it with Newmark's gamma = 1,
 *    beta = 1/2 (Sec. 2.4) applied to each material point's displacement over
 *    the step, du_p = sum_v S_vp du_v: its acceleration at the step end is
 *    a_p = 2 (du_p - dt v_p) / dt^2, so the inertia term is
 *    sum_p S_vp m_p a_p and its tangent the consistent mass times 2 / dt^2;
 *    the velocity update is v_p += dt a_p;
 *  - a free rigid body (Sec. 2.3, 2.4) obeys the same Newmark scheme,
 *    m_b a = m_b g + (contact force on the body), J_b alpha = (contact moment
 *    about its centre); the contact forces couple it to the material and
 *    every Newton iteration solves the bordered system of the material and
 *    body increments (its body part by block elimination);
 *  - updated Lagrangian: S and grad S are fixed at the step start; gradients
 *    in the current configuration are grad_x S = grad S . dF^{-1};
 *    V_p sigma_p = V0_p tau_p;
 *  - ghost: K_G added to the tangent and K_G du to the residual;
 *  - contact: the 8 corners of each GIMP domain are the contact nodes,
 *    eps_N = pf E_p (V0_p)^(2/3), force spread to the grid by the
 *    background basis at the corner; Coulomb friction with
 *    eps_T = pt E_p (V0_p)^(2/3) against the body's own displacement at the
 *    node over the step, q_T + q_R x (y - X) (the rotation linearised over
 *    one step);
 *  - line search: eta = 1, else the best of {0.5, 0.25, 0.1};
 *  - convergence: ||R_free|| <= tol * max(||f_int||, ||f_ext + f_c||), with
 *    ||f_inert|| (time steps) and the body's weight (a free body) in the max;
 *    a free body's residual components join R_free.
 */
#include "o_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

o_model* o_create(const o_params* prm) {
  o_model* m = (o_model*)calloc(1, sizeof(o_model));
  m->p = *prm;
  m->D = prm->depth_max;
  m->unit = prm->L / ldexp(1.0, m->D);
  m->scale = ldexp(1.0, m->D) / prm->L;
  return m;
}

void o_nodes_release(o_nodes* nd);

void o_free(o_model* m) {
  if (!m) return;
  free(m->x); free(m->lp); free(m->l0); free(m->F); free(m->be);
  free(m->V0); free(m->mass); free(m->E); free(m->ys); free(m->v);
  o_tree_free(&m->t);
  o_nodes_release(&m->nd);
  free(m->nsup); free(m->sidx); free(m->S); free(m->dS);
  free(m->populated); free(m->betaK); free(m->bcmask);
  free(m->row_ptr); free(m->col); free(m->kg); free(m->gface);
  free(m);
}

int o_set_points(o_model* m, int n, const double* x, const double* lp, const double* l0,
                 const double* F, const double* be, const double* V0, const double* mass,
                 const double* E, const double* ys) {
  m->np = n;
  m->cap = n;
  m->x = (double*)realloc(m->x, sizeof(double) * 3 * (size_t)n);
  m->lp = (double*)realloc(m->lp, sizeof(double) * 3 * (size_t)n);
  m->l0 = (double*)realloc(m->l0, sizeof(double) * 3 * (size_t)n);
  m->F = (double*)realloc(m->F, sizeof(double) * 9 * (size_t)n);
  m->be = (double*)realloc(m->be, sizeof(double) * 6 * (size_t)n);
  m->V0 = (double*)realloc(m->V0, sizeof(double) * (size_t)n);
  m->mass = (double*)realloc(m->mass, sizeof(double) * (size_t)n);
  m->E = (double*)realloc(m->E, sizeof(double) * (size_t)n);
  m->ys = (double*)realloc(m->ys, sizeof(double) * (size_t)n);
  m->v = (double*)realloc(m->v, sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  for (size_t i = 0; i < 3 * (size_t)n; ++i) m->v[i] = 0.0;
  memcpy(m->x, x, sizeof(double) * 3 * (size_t)n);
  memcpy(m->lp, lp, sizeof(double) * 3 * (size_t)n);
  memcpy(m->l0, l0, sizeof(double) * 3 * (size_t)n);
  memcpy(m->F, F, sizeof(double) * 9 * (size_t)n);
  memcpy(m->be, be, sizeof(double) * 6 * (size_t)n);
  memcpy(m->V0, V0, sizeof(double) * (size_t)n);
  memcpy(m->mass, mass, sizeof(double) * (size_t)n);
  memcpy(m->E, E, sizeof(double) * (size_t)n);
  memcpy(m->ys, ys, sizeof(double) * (size_t)n);
  m->built = 0;
  return O_OK;
}

int o_get_points(const o_model* m, double* x, double* lp, double* l0, double* F, double* be,
                 double* V0, double* mass, double* E, double* ys) {
  int n = m->np;
  if (x) memcpy(x, m->x, sizeof(double) * 3 * (size_t)n);
  if (lp) memcpy(lp, m->lp, sizeof(double) * 3 * (size_t)n);
  if (l0) memcpy(l0, m->l0, sizeof(double) * 3 * (size_t)n);
  if (F) memcpy(F, m->F, sizeof(double) * 9 * (size_t)n);
  if (be) memcpy(be, m->be, sizeof(double) * 6 * (size_t)n);
  if (V0) memcpy(V0, m->V0, sizeof(double) * (size_t)n);
  if (mass) memcpy(mass, m->mass, sizeof(double) * (size_t)n);
  if (E) memcpy(E, m->E, sizeof(double) * (size_t)n);
  if (ys) memcpy(ys, m->ys, sizeof(double) * (size_t)n);
  return O_OK;
}

void o_set_body_z(o_model* m, double z) { m->p.body_z = z; }

int o_build(o_model* m, int nosplit) {
  int st = o_build_tree(m);
  if (st) return st;
  if (!nosplit) {
    st = o_split_points(m);
    if (st) return st;
  }
  st = o_build_nodes(m);
  if (st) return st;
  st = o_build_basis(m);
  if (st) return st;
  st = o_build_pattern_and_ghost(m);
  if (st) return st;
  m->built = 1;
  return O_OK;
}

void o_counts_get(const o_model* m, o_counts* c) {
  memset(c, 0, sizeof(*c));
  c->nleaf = m->t.n;
  c->nnode = m->nd.n;
  for (int n = 0; n < m->nd.n; ++n) c->nhang += m->nd.hang ? m->nd.hang[n] : 0;
  c->ndof = m->nd.ndof;
  c->nnzb = m->nnzb;
  c->nghost = m->nghost;
  c->npts = m->np;
  for (int p = 0; p < m->np && m->nsup; ++p)
    if (m->nsup[p] > c->maxs) c->maxs = m->nsup[p];
}

void o_export_tree(const o_model* m, int* lev, int* anchor) {
  memcpy(lev, m->t.lev, sizeof(int) * (size_t)m->t.n);
  memcpy(anchor, m->t.a, sizeof(int) * 3 * (size_t)m->t.n);
}

void o_export_nodes(const o_model* m, int* coord, int* hang, int* dof, int* cptr, int* cidx,
                    double* cw) {
  const o_nodes* nd = &m->nd;
  memcpy(coord, nd->c, sizeof(int) * 3 * (size_t)nd->n);
  memcpy(hang, nd->hang, sizeof(int) * (size_t)nd->n);
  memcpy(dof, nd->dof, sizeof(int) * (size_t)nd->n);
  memcpy(cptr, nd->cptr, sizeof(int) * (size_t)(nd->n + 1));
  memcpy(cidx, nd->cidx, sizeof(int) * (size_t)nd->cptr[nd->n]);
  memcpy(cw, nd->cw, sizeof(double) * (size_t)nd->cptr[nd->n]);
}

void o_export_support(const o_model* m, int* nsup, int* sidx, double* S, double* dS) {
  memcpy(nsup, m->nsup, sizeof(int) * (size_t)m->np);
  memcpy(sidx, m->sidx, sizeof(int) * O_MAXS * (size_t)m->np);
  memcpy(S, m->S, sizeof(double) * O_MAXS * (size_t)m->np);
  memcpy(dS, m->dS, sizeof(double) * 3 * O_MAXS * (size_t)m->np);
}

void o_export_pattern(const o_model* m, int* row_ptr, int* col) {
  memcpy(row_ptr, m->row_ptr, sizeof(int) * (size_t)(m->nd.ndof + 1));
  memcpy(col, m->col, sizeof(int) * (size_t)m->nnzb);
}

void o_export_ghost(const o_model* m, double* kg) {
  memcpy(kg, m->kg, sizeof(double) * (size_t)m->nnzb);
}

void o_export_ghost_faces(const o_model* m, int* faces, int* populated) {
  memcpy(faces, m->gface, sizeof(int) * 4 * (size_t)m->nghost);
  memcpy(populated, m->populated, sizeof(int) * (size_t)m->t.n);
}

void o_export_bcmask(const o_model* m, int* mask) {
  memcpy(mask, m->bcmask, sizeof(int) * (size_t)m->nd.ndof);
}

/* leaf holding the box corner, taken on the inside of the box */
static int corner_leaf(const o_model* m, const double* X, const int* side, double* xi) {
  int N = 1 << m->D, q[3];
  for (int d = 0; d < 3; ++d) {
    q[d] = side[d] > 0 ? (int)ceil(X[d]) - 1 : (int)floor(X[d]);
    if (q[d] < 0) q[d] = 0;
    if (q[d] > N - 1) q[d] = N - 1;
  }
  int K = o_locate(&m->t, q[0], q[1], q[2]);
  int s = 1 << (m->D - m->t.lev[K]);
  for (int d = 0; d < 3; ++d) xi[d] = (X[d] - (double)m->t.a[3 * K + d]) / (double)s;
  return K;
}

int o_eval_background(const o_model* m, const double* x, int* nent, int* idx, double* phi,
                      double* dphi) {
  double X[3], xi[3];
  int side[3] = {-1, -1, -1};
  for (int d = 0; d < 3; ++d) X[d] = x[d] * m->scale;
  int K = corner_leaf(m, X, side, xi);
  int st = o_leaf_basis(m, K, xi, nent, idx, phi, dphi);
  for (int i = 0; i < *nent; ++i) {
    idx[i] = m->nd.dof[idx[i]];
    for (int d = 0; d < 3; ++d) dphi[3 * i + d] *= m->scale;
  }
  return st;
}

/* point kinematics: dF = I + sum_v du_v (x) grad S_vp */
static void point_dF(const o_model* m, int p, const double* du, double* dF) {
  for (int i = 0; i < 9; ++i) dF[i] = (i % 4 == 0) ? 1.0 : 0.0;
  const int* si = m->sidx + O_MAXS * (size_t)p;
  const double* dS = m->dS + 3 * O_MAXS * (size_t)p;
  for (int k = 0; k < m->nsup[p]; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dF[3 * i + j] += du[3 * si[k] + i] * dS[3 * k + j];
}

int o_point_stress(o_model* m, const double* du, double* sigma) {
  for (int p = 0; p < m->np; ++p) {
    double dF[9], tau[9], ben[6], Ft[9];
    int pl;
    point_dF(m, p, du, dF);
    int st = o_constitutive(&m->p, m->E[p], m->ys[p], m->be + 6 * (size_t)p, dF, tau, ben, NULL, &pl);
    if (st) return st;
    o_mat33_mul(dF, m->F + 9 * (size_t)p, Ft);
    double J = o_det33(Ft);
    for (int i = 0; i < 9; ++i) sigma[9 * (size_t)p + i] = tau[i] / J;
  }
  return O_OK;
}

/* Coulomb friction at a contact node (Sec. 2.3: stick-slip regularised by the
 * tangential penalty eps_T = pt E_p (V0_p)^(2/3)).  Reading: the slip g is
 * the node's displacement relative to the body's surface over the current
 * step, projected on the tangent plane; no tangential force is carried from
 * one step to the next.  Trial force t = -eps_T (I - n n^T) g; stick if
 * |t| <= mu f_N, else slip with mu f_N t / |t|.  Adds the force to f and
 * writes its derivatives in d = y - X (through n, H and f_N) to Jd and in g to
 * Jg (row-major 3x3). */
static void friction(const o_params* p, double E, double V0, const double* g, const double* n,
                     const double* H, double fN, double epsN, double* f, double* Jd, double* Jg) {
  double epsT = p->pt * E * pow(V0, 2.0 / 3.0);
  double t[3], Hg[3];
  double ng = n[0] * g[0] + n[1] * g[1] + n[2] * g[2];
  for (int a = 0; a < 3; ++a) Hg[a] = H[3 * a] * g[0] + H[3 * a + 1] * g[1] + H[3 * a + 2] * g[2];
  for (int d = 0; d < 3; ++d) t[d] = -epsT * (g[d] - n[d] * ng);
  /* d t / d d = eps_T ((n.g) H + n (H g)^T) (dn/dd = H), d t / d g = -eps_T (I - n n^T) */
  double Td[9], Tg[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Td[3 * a + b] = epsT * (ng * H[3 * a + b] + n[a] * Hg[b]);
      Tg[3 * a + b] = -epsT * ((a == b ? 1.0 : 0.0) - n[a] * n[b]);
    }
  double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  if (tn <= p->mu * fN) {
    for (int d = 0; d < 3; ++d) f[d] += t[d];
    for (int q = 0; q < 9; ++q) {
      Jd[q] = Td[q];
      Jg[q] = Tg[q];
    }
    return;
  }
  double u[3] = {t[0] / tn, t[1] / tn, t[2] / tn};
  for (int d = 0; d < 3; ++d) f[d] += p->mu * fN * u[d];
  /* d(mu f_N u) = mu u (d f_N)^T + mu f_N (I - u u^T) d t / |t|, d f_N / d d = -eps_N n */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double sd = 0.0, sg = 0.0;
      for (int c = 0; c < 3; ++c) {
        double P = (a == c ? 1.0 : 0.0) - u[a] * u[c];
        sd += P * Td[3 * c + b];
        sg += P * Tg[3 * c + b];
      }
      Jd[3 * a + b] = p->mu * u[a] * (-epsN * n[b]) + p->mu * fN * sd / tn;
      Jg[3 * a + b] = p->mu * fN * sg / tn;
    }
}

/* [a]x, the matrix of b -> a x b (row-major) */
static void cross_mat(const double* a, double* C) {
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

static void mat33(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

int o_set_velocity(o_model* m, const double* v) {
  memcpy(m->v, v, sizeof(double) * 3 * (size_t)m->np);
  return O_OK;
}

int o_get_velocity(const o_model* m, double* v) {
  memcpy(v, m->v, sizeof(double) * 3 * (size_t)m->np);
  return O_OK;
}

void o_get_body(const o_model* m, double* pose, double* v, double* w, double* theta) {
  pose[0] = m->p.body_cx;
  pose[1] = m->p.body_cy;
  pose[2] = m->p.body_z;
  for (int d = 0; d < 3; ++d) {
    v[d] = m->p.body_v[d];
    w[d] = m->p.body_w[d];
    theta[d] = m->body_theta[d];
  }
}

int o_assemble_body(o_model* m, const double* du, const double* q, double load, double* R,
                    double* Kv, double* fint_all, double* reaction, double* Rb, double* Kbb,
                    double* Kgb, double* Kbg) {
  int ndof = m->nd.ndof;
  size_t n3 = 3 * (size_t)ndof;
  for (size_t i = 0; i < n3; ++i) R[i] = 0.0;
  if (fint_all)
    for (size_t i = 0; i < n3; ++i) fint_all[i] = 0.0;
  if (Kv)
    for (size_t i = 0; i < 9 * (size_t)m->nnzb; ++i) Kv[i] = 0.0;
  if (reaction) reaction[0] = reaction[1] = reaction[2] = 0.0;
  if (Rb)
    for (int i = 0; i < 6; ++i) Rb[i] = 0.0;
  if (Kbb)
    for (int i = 0; i < 36; ++i) Kbb[i] = 0.0;
  if (Kgb)
    for (size_t i = 0; i < 6 * n3; ++i) Kgb[i] = 0.0;
  if (Kbg)
    for (size_t i = 0; i < 6 * n3; ++i) Kbg[i] = 0.0;
  /* the body's increment over the step: translation qt, rotation qr; with
   * free components the given pose is the step-start one and the body sits
   * at pose + qt, else the given pose is the step-end one */
  const o_params* pp = &m->p;
  double qt[3], qr[3], shift[3];
  for (int d = 0; d < 3; ++d) {
    qt[d] = q ? q[d] : pp->body_d[d];
    qr[d] = q ? q[3 + d] : 0.0;
    shift[d] = pp->body_free ? qt[d] : 0.0;
  }
  const double X[3] = {pp->body_cx + shift[0], pp->body_cy + shift[1], pp->body_z + shift[2]};
  double dt = pp->dt, c2 = dt > 0.0 ? 2.0 / (dt * dt) : 0.0;
  double* fext_c = (double*)calloc(n3 > 0 ? n3 : 1, sizeof(double));
  double* finert = dt > 0.0 ? (double*)calloc(n3 > 0 ? n3 : 1, sizeof(double)) : NULL;
  double A[81];
  for (int p = 0; p < m->np; ++p) {
    const int* si = m->sidx + O_MAXS * (size_t)p;
    const double* S = m->S + O_MAXS * (size_t)p;
    const double* dS = m->dS + 3 * O_MAXS * (size_t)p;
    int ns = m->nsup[p];
    double dF[9], dFi[9], tau[9], ben[6];
    int pl;
    point_dF(m, p, du, dF);
    if (!(o_det33(dF) > 0.0)) {
      free(fext_c);
      free(finert);
      return O_ERR_NAN;
    }
    int st = o_constitutive(&m->p, m->E[p], m->ys[p], m->be + 6 * (size_t)p, dF, tau, ben,
                            Kv ? A : NULL, &pl);
    if (st) {
      free(fext_c);
      free(finert);
      return st;
    }
    o_inv33(dF, dFi);
    double V0 = m->V0[p];
    double gx[O_MAXS][3];
    for (int k = 0; k < ns; ++k)
      for (int mm = 0; mm < 3; ++mm) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += dS[3 * k + l] * dFi[3 * l + mm];
        gx[k][mm] = s;
      }
    /* Newmark acceleration of the point (time steps only) */
    double ap[3] = {0.0, 0.0, 0.0};
    if (dt > 0.0) {
      double dup[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < ns; ++k)
        for (int i = 0; i < 3; ++i) dup[i] += S[k] * du[3 * si[k] + i];
      for (int i = 0; i < 3; ++i) ap[i] = c2 * (dup[i] - dt * m->v[3 * p + i]);
    }
    /* f_int,v = V_p sigma grad_x S_v = V0 tau grad_x S_v; f_ext,v = S_v m g;
     * inertia S_v m a_p */
    for (int k = 0; k < ns; ++k)
      for (int i = 0; i < 3; ++i) {
        double f = 0.0;
        for (int j = 0; j < 3; ++j) f += tau[3 * i + j] * gx[k][j];
        f *= V0;
        R[3 * si[k] + i] += f;
        if (fint_all) fint_all[3 * si[k] + i] += f;
        double fe = load * m->mass[p] * S[k] * m->p.g[i];
        R[3 * si[k] + i] -= fe;
        fext_c[3 * si[k] + i] += fe;
        if (dt > 0.0) {
          R[3 * si[k] + i] += S[k] * m->mass[p] * ap[i];
          finert[3 * si[k] + i] += S[k] * m->mass[p] * ap[i];
        }
      }
    if (Kv) {
      /* K_{vi,wk} = V0 sum_{j,m} gx_vj (A_ijkm - tau_im delta_jk) gx_wm
       *           + (2 / dt^2) m_p S_v S_w delta_ik */
      for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; ++b) {
          int sl = o_find_slot(m, si[a], si[b]);
          double* blk = Kv + 9 * (size_t)sl;
          for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
              double s = 0.0;
              for (int j = 0; j < 3; ++j)
                for (int mm = 0; mm < 3; ++mm) {
                  double a4 = A[((i * 3 + j) * 3 + k) * 3 + mm] - (j == k ? tau[3 * i + mm] : 0.0);
                  s += gx[a][j] * a4 * gx[b][mm];
                }
              blk[3 * i + k] += V0 * s;
            }
          if (dt > 0.0) {
            double mk = c2 * m->mass[p] * S[a] * S[b];
            for (int i = 0; i < 3; ++i) blk[4 * i] += mk;
          }
        }
    }
  }
  /* ghost penalty on the step increment (Sec. 4, reading: K_G and K_G du) */
  for (int i = 0; i < ndof; ++i)
    for (int s = m->row_ptr[i]; s < m->row_ptr[i + 1]; ++s) {
      double kg = m->kg[s];
      if (kg == 0.0) continue;
      int j = m->col[s];
      for (int c = 0; c < 3; ++c) R[3 * i + c] += kg * du[3 * j + c];
      if (Kv)
        for (int c = 0; c < 3; ++c) Kv[9 * (size_t)s + 4 * c] += kg;
    }
  /* node-to-surface penalty contact at the GIMP domain corners (Sec. 2.3) */
  if (m->p.contact_on && m->p.body_kind != 0) {
    int idx[O_MAXS], nent;
    double ph[O_MAXS], dph[3 * O_MAXS];
    double Qr[9];
    cross_mat(qr, Qr);
    for (int p = 0; p < m->np; ++p) {
      double Lo[3], Hi[3];
      double N = (double)(1 << m->D);
      for (int d = 0; d < 3; ++d) {
        double lo = (m->x[3 * p + d] - m->lp[3 * p + d]) * m->scale;
        double hi = (m->x[3 * p + d] + m->lp[3 * p + d]) * m->scale;
        double rl = floor(lo + 0.5), rh = floor(hi + 0.5);
        lo = fabs(lo - rl) < 1e-9 ? rl : lo;
        hi = fabs(hi - rh) < 1e-9 ? rh : hi;
        Lo[d] = lo < 0.0 ? 0.0 : lo;
        Hi[d] = hi > N ? N : hi;
      }
      double epsN = m->p.pf * m->E[p] * pow(m->V0[p], 2.0 / 3.0);
      for (int c = 0; c < 8; ++c) {
        int side[3];
        double Xc[3], y[3], xi[3];
        for (int d = 0; d < 3; ++d) {
          side[d] = ((c >> d) & 1) ? 1 : -1;
          Xc[d] = side[d] > 0 ? Hi[d] : Lo[d];
          y[d] = m->x[3 * p + d] + side[d] * m->lp[3 * p + d];
        }
        int K = corner_leaf(m, Xc, side, xi);
        o_leaf_basis(m, K, xi, &nent, idx, ph, dph);
        double y0[3] = {y[0], y[1], y[2]};
        for (int i = 0; i < nent; ++i) {
          idx[i] = m->nd.dof[idx[i]];
          for (int d = 0; d < 3; ++d) y[d] += ph[i] * du[3 * idx[i] + d];
        }
        /* the body's signed distance at the node, in the frame of its given pose */
        double phi, n[3], H[9], yb[3];
        for (int d = 0; d < 3; ++d) yb[d] = y[d] - shift[d];
        o_body_sdf(&m->p, yb, &phi, n, H);
        if (!(phi < 0.0)) continue;
        /* normal force f_N n, f_N = -eps_N phi: d/dd = -eps_N (n n^T + phi H) */
        double fN = -epsN * phi, f[3], Fy[9], Ft[9], dv[3];
        for (int d = 0; d < 3; ++d) {
          f[d] = fN * n[d];
          dv[d] = y[d] - X[d];
        }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            Fy[3 * a + b] = -epsN * (n[a] * n[b] + phi * H[3 * a + b]);
            Ft[3 * a + b] = 0.0;
          }
        if (m->p.mu > 0.0) {
          /* slip against the body's displacement at the node, qt + qr x d:
           * dg/dy = I - [qr]x, dg/dqt = -(I - [qr]x), dg/dqr = [d]x */
          double g[3], Jd[9], Jg[9], IQ[9], Dx[9], T[9];
          for (int d = 0; d < 3; ++d) {
            double rot = qr[(d + 1) % 3] * dv[(d + 2) % 3] - qr[(d + 2) % 3] * dv[(d + 1) % 3];
            g[d] = (y[d] - y0[d]) - (qt[d] + rot);
          }
          friction(&m->p, m->E[p], m->V0[p], g, n, H, fN, epsN, f, Jd, Jg);
          for (int e = 0; e < 9; ++e) IQ[e] = (e % 4 == 0 ? 1.0 : 0.0) - Qr[e];
          mat33(Jg, IQ, T);
          for (int e = 0; e < 9; ++e) Fy[e] += Jd[e] + T[e];
          cross_mat(dv, Dx);
          mat33(Jg, Dx, Ft);
        }
        /* f acts on the material, -f on the body at the node (Sec. 2.3) */
        if (reaction)
          for (int d = 0; d < 3; ++d) reaction[d] -= f[d];
        for (int i = 0; i < nent; ++i)
          for (int d = 0; d < 3; ++d) {
            R[3 * idx[i] + d] -= ph[i] * f[d];
            fext_c[3 * idx[i] + d] += ph[i] * f[d];
          }
        if (Kv) {
          for (int a = 0; a < nent; ++a)
            for (int b = 0; b < nent; ++b) {
              int sl = o_find_slot(m, idx[a], idx[b]);
              for (int e = 0; e < 9; ++e) Kv[9 * (size_t)sl + e] -= ph[a] * ph[b] * Fy[e];
            }
        }
        /* the body's equations: + f and + d x f (their signs make the
         * body's residual m a - m g + sum f, J alpha + sum d x f) */
        double Dx[9], Fx[9], DF[9];
        cross_mat(dv, Dx);
        cross_mat(f, Fx);
        mat33(Dx, Fy, DF);
        if (Rb)
          for (int d = 0; d < 3; ++d) {
            Rb[d] += f[d];
            Rb[3 + d] += dv[(d + 1) % 3] * f[(d + 2) % 3] - dv[(d + 2) % 3] * f[(d + 1) % 3];
          }
        for (int i = 0; i < nent; ++i)
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              size_t r = 3 * (size_t)idx[i] + a, cl = 3 * (size_t)idx[i] + b;
              /* dR_g / dqt = -ph F_X = ph F_y, dR_g / dqr = -ph F_theta */
              if (Kgb) {
                Kgb[(size_t)b * n3 + r] += ph[i] * Fy[3 * a + b];
                Kgb[(size_t)(3 + b) * n3 + r] -= ph[i] * Ft[3 * a + b];
              }
              /* dRb_T / du = ph F_y, d(d x f) / du = ph ([d]x F_y - [f]x) */
              if (Kbg) {
                Kbg[(size_t)a * n3 + cl] += ph[i] * Fy[3 * a + b];
                Kbg[(size_t)(3 + a) * n3 + cl] += ph[i] * (DF[3 * a + b] - Fx[3 * a + b]);
              }
            }
        if (Kbb) {
          double DT[9];
          mat33(Dx, Ft, DT);
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              Kbb[6 * a + b] -= Fy[3 * a + b];
              Kbb[6 * a + 3 + b] += Ft[3 * a + b];
              Kbb[6 * (3 + a) + b] += Fx[3 * a + b] - DF[3 * a + b];
              Kbb[6 * (3 + a) + 3 + b] += DT[3 * a + b];
            }
        }
      }
    }
  }
  /* the body's Newmark inertia and weight (time steps only) */
  if (dt > 0.0) {
    for (int d = 0; d < 3; ++d) {
      if (Rb) {
        Rb[d] += pp->body_mass * (c2 * (qt[d] - dt * pp->body_v[d]) - load * pp->g[d]);
        Rb[3 + d] += pp->body_inertia * c2 * (qr[d] - dt * pp->body_w[d]);
      }
      if (Kbb) {
        Kbb[7 * d] += pp->body_mass * c2;
        Kbb[7 * (3 + d)] += pp->body_inertia * c2;
      }
    }
  }
  if (fint_all) {
    /* second half of the reference force: ||f_ext + f_c|| stored after f_int */
    double s = 0.0;
    for (size_t i = 0; i < n3; ++i) s += fext_c[i] * fext_c[i];
    fint_all[n3] = sqrt(s);
    /* time steps: ||f_inert|| after it (a free body's motion can be all
     * inertia, with no internal or external force to measure against) */
    if (finert) {
      s = 0.0;
      for (size_t i = 0; i < n3; ++i) s += finert[i] * finert[i];
      fint_all[n3 + 1] = sqrt(s);
    }
  }
  free(fext_c);
  free(finert);
  for (size_t i = 0; i < n3; ++i)
    if (!isfinite(R[i])) return O_ERR_NAN;
  return O_OK;
}

int o_assemble(o_model* m, const double* du, double load, double* R, double* Kv, double* fint_all,
               double* reaction) {
  return o_assemble_body(m, du, NULL, load, R, Kv, fint_all, reaction, NULL, NULL, NULL, NULL);
}

/* ---------------- linear solves on the free components ---------------- */

static int lu_solve(int n, double* A, double* b) {
  int* piv = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) {
    int pm = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)pm * n + k])) pm = i;
    if (A[(size_t)pm * n + k] == 0.0) {
      free(piv);
      return O_ERR_KRYLOV;
    }
    piv[k] = pm;
    if (pm != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)pm * n + j];
        A[(size_t)pm * n + j] = t;
      }
      double t = b[k];
      b[k] = b[pm];
      b[pm] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * b[j];
    b[i] = s / A[(size_t)i * n + i];
  }
  free(piv);
  return O_OK;
}

/* y = K x restricted to free components (fixed components of y are zero) */
static void free_matvec(const o_model* m, const double* Kv, const double* x, double* y) {
  int ndof = m->nd.ndof;
  for (int i = 0; i < ndof; ++i)
    for (int c = 0; c < 3; ++c) {
      if (m->bcmask[i] & (1 << c)) {
        y[3 * i + c] = 0.0;
        continue;
      }
      double s = 0.0;
      for (int q = m->row_ptr[i]; q < m->row_ptr[i + 1]; ++q) {
        int j = m->col[q];
        for (int e = 0; e < 3; ++e)
          if (!(m->bcmask[j] & (1 << e))) s += Kv[9 * (size_t)q + 3 * c + e] * x[3 * j + e];
      }
      y[3 * i + c] = s;
    }
}

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int o_solve(o_model* m, const double* Kv, const double* b, double* x, double tol, int maxit,
            int* its) {
  int ndof = m->nd.ndof, n3 = 3 * ndof;
  int* fid = (int*)malloc(sizeof(int) * (size_t)n3);
  int nf = 0;
  for (int i = 0; i < n3; ++i) {
    fid[i] = (m->bcmask[i / 3] & (1 << (i % 3))) ? -1 : nf++;
    x[i] = 0.0;
  }
  *its = 0;
  int st = O_OK;
  if (nf <= 1500) {
    double* A = (double*)calloc((size_t)nf * (size_t)nf, sizeof(double));
    double* r = (double*)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1));
    for (int i = 0; i < ndof; ++i)
      for (int q = m->row_ptr[i]; q < m->row_ptr[i + 1]; ++q) {
        int j = m->col[q];
        for (int c = 0; c < 3; ++c)
          for (int e = 0; e < 3; ++e) {
            int fi = fid[3 * i + c], fj = fid[3 * j + e];
            if (fi >= 0 && fj >= 0) A[(size_t)fi * nf + fj] += Kv[9 * (size_t)q + 3 * c + e];
          }
      }
    for (int i = 0; i < n3; ++i)
      if (fid[i] >= 0) r[fid[i]] = b[i];
    st = lu_solve(nf, A, r);
    for (int i = 0; i < n3; ++i)
      if (fid[i] >= 0) x[i] = r[fid[i]];
    free(A);
    free(r);
    *its = 1;
    free(fid);
    return st;
  }
  free(fid);
  /* point-Jacobi preconditioned CG (symmetric) or BiCGStab (Drucker-Prager
   * with psi != phi gives a non-symmetric tangent) */
  double* diag = (double*)malloc(sizeof(double) * (size_t)n3);
  for (int i = 0; i < ndof; ++i) {
    int q = o_find_slot(m, i, i);
    for (int c = 0; c < 3; ++c) {
      double dv = q >= 0 ? Kv[9 * (size_t)q + 4 * c] : 0.0;
      diag[3 * i + c] = (m->bcmask[i] & (1 << c)) || dv == 0.0 ? 0.0 : 1.0 / dv;
    }
  }
  double* r = (double*)malloc(sizeof(double) * (size_t)n3);
  double* z = (double*)malloc(sizeof(double) * (size_t)n3);
  double* pv = (double*)malloc(sizeof(double) * (size_t)n3);
  double* q = (double*)malloc(sizeof(double) * (size_t)n3);
  for (int i = 0; i < n3; ++i) r[i] = (m->bcmask[i / 3] & (1 << (i % 3))) ? 0.0 : b[i];
  double bn = sqrt(dot(n3, r, r));
  /* friction makes the contact stiffness non-symmetric */
  int nonsym = (m->p.model == 2 && m->p.psi != m->p.phi) || m->p.model == 3 ||
               (m->p.mu > 0.0 && m->p.contact_on && m->p.body_kind != 0);
  st = O_ERR_KRYLOV;
  if (bn == 0.0) {
    st = O_OK;
  } else if (!nonsym) {
    for (int i = 0; i < n3; ++i) {
      z[i] = diag[i] * r[i];
      pv[i] = z[i];
    }
    double rz = dot(n3, r, z);
    for (int k = 1; k <= maxit; ++k) {
      free_matvec(m, Kv, pv, q);
      double alpha = rz / dot(n3, pv, q);
      for (int i = 0; i < n3; ++i) {
        x[i] += alpha * pv[i];
        r[i] -= alpha * q[i];
      }
      *its = k;
      if (sqrt(dot(n3, r, r)) <= tol * bn) {
        st = O_OK;
        break;
      }
      for (int i = 0; i < n3; ++i) z[i] = diag[i] * r[i];
      double rz2 = dot(n3, r, z);
      double beta = rz2 / rz;
      rz = rz2;
      for (int i = 0; i < n3; ++i) pv[i] = z[i] + beta * pv[i];
    }
  } else {
    double* r0 = (double*)malloc(sizeof(double) * (size_t)n3);
    double* v = (double*)calloc((size_t)n3, sizeof(double));
    double* s = (double*)malloc(sizeof(double) * (size_t)n3);
    double* t = (double*)malloc(sizeof(double) * (size_t)n3);
    double* ph = (double*)malloc(sizeof(double) * (size_t)n3);
    double* sh = (double*)malloc(sizeof(double) * (size_t)n3);
    memcpy(r0, r, sizeof(double) * (size_t)n3);
    for (int i = 0; i < n3; ++i) pv[i] = 0.0;
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    for (int k = 1; k <= maxit; ++k) {
      double rho1 = dot(n3, r0, r);
      if (rho1 == 0.0) break;
      double beta = (rho1 / rho) * (alpha / omega);
      rho = rho1;
      for (int i = 0; i < n3; ++i) pv[i] = r[i] + beta * (pv[i] - omega * v[i]);
      for (int i = 0; i < n3; ++i) ph[i] = diag[i] * pv[i];
      free_matvec(m, Kv, ph, v);
      alpha = rho / dot(n3, r0, v);
      for (int i = 0; i < n3; ++i) s[i] = r[i] - alpha * v[i];
      *its = k;
      if (sqrt(dot(n3, s, s)) <= tol * bn) {
        for (int i = 0; i < n3; ++i) x[i] += alpha * ph[i];
        st = O_OK;
        break;
      }
      for (int i = 0; i < n3; ++i) sh[i] = diag[i] * s[i];
      free_matvec(m, Kv, sh, t);
      double tt = dot(n3, t, t);
      omega = tt > 0.0 ? dot(n3, t, s) / tt : 0.0;
      for (int i = 0; i < n3; ++i) {
        x[i] += alpha * ph[i] + omega * sh[i];
        r[i] = s[i] - omega * t[i];
      }
      if (sqrt(dot(n3, r, r)) <= tol * bn) {
        st = O_OK;
        break;
      }
      if (omega == 0.0) break;
    }
    free(r0); free(v); free(s); free(t); free(ph); free(sh);
  }
  free(diag); free(r); free(z); free(pv); free(q);
  return st;
}

/* ---------------- Newton load step (Sec. 2.4) and point update ---------------- */

static double norm_free(const o_model* m, const double* R) {
  double s = 0.0;
  for (int i = 0; i < 3 * m->nd.ndof; ++i)
    if (!(m->bcmask[i / 3] & (1 << (i % 3)))) s += R[i] * R[i];
  return sqrt(s);
}

static double norm2(int n, const double* a) { return sqrt(dot(n, a, a)); }

/* Newton-Raphson over the material increment du and the free components of
 * the body's increment q (Sec. 2.4).  The linearised system
 *   [K   Kgb] [dx]   [-R ]
 *   [Kbg Kbb] [dq] = [-Rb]
 * (restricted to free components) is solved by eliminating dx: with
 * w = K^-1 (-R) and Z = K^-1 Kgb, (Kbb - Kbg Z) dq = -Rb - Kbg w, dx = w - Z dq. */
int o_step(o_model* m, const o_step_params* sp, o_step_stats* stt) {
  memset(stt, 0, sizeof(*stt));
  const o_params* pp = &m->p;
  int fb[6], nb = 0;
  for (int j = 0; j < 6; ++j)
    if (pp->body_free & (1 << j)) fb[nb++] = j;
  if (nb && (!(pp->dt > 0.0) || pp->body_kind == 0 || !pp->contact_on ||
             ((pp->body_free & 0x38) && pp->body_kind != 4)))
    return stt->status = O_ERR_ARG;
  int st = o_build(m, 0);
  if (st) return stt->status = st;
  int n3 = 3 * m->nd.ndof;
  size_t N3 = (size_t)(n3 > 0 ? n3 : 1);
  double* du = (double*)calloc(N3, sizeof(double));
  double* R = (double*)malloc(sizeof(double) * N3);
  double* R1 = (double*)malloc(sizeof(double) * N3);
  double* fi = (double*)calloc(N3 + 2, sizeof(double));
  double* Kv = (double*)malloc(sizeof(double) * 9 * (size_t)(m->nnzb > 0 ? m->nnzb : 1));
  double* dx = (double*)malloc(sizeof(double) * N3);
  double* trial = (double*)malloc(sizeof(double) * N3);
  double *Kgb = NULL, *Kbg = NULL, *Z = NULL;
  if (nb) {
    Kgb = (double*)malloc(sizeof(double) * 6 * N3);
    Kbg = (double*)malloc(sizeof(double) * 6 * N3);
    Z = (double*)malloc(sizeof(double) * 6 * N3);
  }
  double q[6], qtr[6], dq[6] = {0, 0, 0, 0, 0, 0}, Rb[6], Rb1[6], Kbb[36];
  for (int d = 0; d < 3; ++d) {
    q[d] = (pp->body_free & (1 << d)) ? 0.0 : pp->body_d[d];
    q[3 + d] = 0.0;
  }
  double wref = 0.0;
  if (nb)
    for (int d = 0; d < 3; ++d) wref += pow(pp->body_mass * sp->load * pp->g[d], 2.0);
  wref = sqrt(wref);
  double reac[3];
  st = o_assemble_body(m, du, q, sp->load, R, Kv, fi, reac, Rb, Kbb, Kgb, Kbg);
  int conv = 0;
  for (int it = 0; st == O_OK && it <= sp->maxit; ++it) {
    double rn = norm_free(m, R);
    for (int j = 0; j < nb; ++j) rn = hypot(rn, Rb[fb[j]]);
    double fref = fmax(fmax(fmax(norm2(n3, fi), fi[n3]), fi[n3 + 1]), wref);
    if (it < 64) stt->res_hist[it] = fref > 0 ? rn / fref : rn;
    if (rn <= sp->tol * fref || fref == 0.0) {
      conv = 1;
      stt->newton_its = it;
      break;
    }
    if (it == sp->maxit) break;
    for (int i = 0; i < n3; ++i) trial[i] = -R[i];
    int lits = 0;
    st = o_solve(m, Kv, trial, dx, sp->lin_tol, sp->lin_maxit, &lits);
    stt->lin_its_total += lits;
    if (st) break;
    if (nb) {
      double Sm[36], rb[6];
      for (int l = 0; l < nb && !st; ++l) {
        st = o_solve(m, Kv, Kgb + (size_t)fb[l] * N3, Z + (size_t)l * N3, sp->lin_tol,
                     sp->lin_maxit, &lits);
        stt->lin_its_total += lits;
      }
      if (st) break;
      for (int j = 0; j < nb; ++j) {
        const double* kr = Kbg + (size_t)fb[j] * N3;
        rb[j] = -Rb[fb[j]] - dot(n3, kr, dx);
        for (int l = 0; l < nb; ++l) Sm[nb * j + l] = Kbb[6 * fb[j] + fb[l]] - dot(n3, kr, Z + (size_t)l * N3);
      }
      st = lu_solve(nb, Sm, rb);
      if (st) break;
      for (int j = 0; j < 6; ++j) dq[j] = 0.0;
      for (int l = 0; l < nb; ++l) {
        dq[fb[l]] = rb[l];
        const double* zl = Z + (size_t)l * N3;
        for (int i = 0; i < n3; ++i) dx[i] -= zl[i] * rb[l];
      }
    }
    /* line search (Sec. 2.4): eta = 1, else the lowest residual of {0.5,0.25,0.1} */
    const double etas[4] = {1.0, 0.5, 0.25, 0.1};
    double best = -1.0, besteta = 1.0;
    for (int e = 0; e < 4; ++e) {
      for (int i = 0; i < n3; ++i) trial[i] = du[i] + etas[e] * dx[i];
      for (int j = 0; j < 6; ++j) qtr[j] = q[j] + etas[e] * dq[j];
      int s2 = o_assemble_body(m, trial, qtr, sp->load, R1, NULL, NULL, NULL, Rb1, NULL, NULL, NULL);
      double r1 = s2 ? INFINITY : norm_free(m, R1);
      for (int j = 0; j < nb && !s2; ++j) r1 = hypot(r1, Rb1[fb[j]]);
      if (best < 0.0 || r1 < best) {
        best = r1;
        besteta = etas[e];
      }
      if (e == 0 && r1 < rn) break;
    }
    if (it < 64) stt->eta_hist[it] = besteta;
    for (int i = 0; i < n3; ++i) du[i] += besteta * dx[i];
    for (int j = 0; j < 6; ++j) q[j] += besteta * dq[j];
    st = o_assemble_body(m, du, q, sp->load, R, Kv, fi, reac, Rb, Kbb, Kgb, Kbg);
  }
  if (st == O_OK && !conv) st = O_ERR_NEWTON;
  if (st == O_OK) {
    for (int d = 0; d < 3; ++d) stt->reaction[d] = reac[d];
    for (int j = 0; j < 6; ++j) stt->body_q[j] = q[j];
    double dt = pp->dt, c2 = dt > 0.0 ? 2.0 / (dt * dt) : 0.0;
    /* point update: x += du_p with du_p = sum_v S_vp du_v; for a time step
     * v += dt a_p, a_p = 2 (du_p - dt v) / dt^2; F, b_e from the converged
     * state; domain half-lengths l = l0 diag(U), U = sqrt(F^T F) (reading) */
    for (int p = 0; p < m->np; ++p) {
      double dF[9], tau[9], ben[6], Fn[9];
      int pl;
      point_dF(m, p, du, dF);
      o_constitutive(&m->p, m->E[p], m->ys[p], m->be + 6 * (size_t)p, dF, tau, ben, NULL, &pl);
      o_mat33_mul(dF, m->F + 9 * (size_t)p, Fn);
      const int* si = m->sidx + O_MAXS * (size_t)p;
      const double* S = m->S + O_MAXS * (size_t)p;
      double dup[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < m->nsup[p]; ++k)
        for (int d = 0; d < 3; ++d) dup[d] += S[k] * du[3 * si[k] + d];
      for (int d = 0; d < 3; ++d) {
        m->x[3 * p + d] += dup[d];
        if (dt > 0.0) m->v[3 * p + d] += dt * c2 * (dup[d] - dt * m->v[3 * p + d]);
      }
      memcpy(m->F + 9 * (size_t)p, Fn, sizeof(Fn));
      memcpy(m->be + 6 * (size_t)p, ben, sizeof(ben));
      double C[9], Ft[9], lam[3], Q[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ft[3 * i + j] = Fn[3 * j + i];
      o_mat33_mul(Ft, Fn, C);
      o_eig_sym3(C, lam, Q);
      for (int d = 0; d < 3; ++d) {
        double u = 0.0;
        for (int a = 0; a < 3; ++a) u += sqrt(lam[a]) * Q[3 * d + a] * Q[3 * d + a];
        m->lp[3 * p + d] = m->l0[3 * p + d] * u;
      }
    }
    /* the free body's Newmark update: velocities, pose and rotation */
    if (nb) {
      o_params* pm = &m->p;
      for (int d = 0; d < 3; ++d) {
        pm->body_v[d] += dt * c2 * (q[d] - dt * pm->body_v[d]);
        pm->body_w[d] += dt * c2 * (q[3 + d] - dt * pm->body_w[d]);
        m->body_theta[d] += q[3 + d];
      }
      pm->body_cx += q[0];
      pm->body_cy += q[1];
      pm->body_z += q[2];
    }
  }
  free(du); free(R); free(R1); free(fi); free(Kv); free(dx); free(trial);
  free(Kgb); free(Kbg); free(Z);
  stt->status = st;
  return st;
}
