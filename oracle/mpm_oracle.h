/*
 * FP64 CPU oracle of the implicit octree GIMP MPM load step
 * (Bird, Coombs, Augarde, Pretti, O'Hare: "An implicit octree-based adaptive
 * Material Point Method").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow reference that the
 * GPU path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline and reference legs of the benchmark may load it; the product
 * path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Everything is double precision, single threaded, written as plain loops in
 * the order the paper states the method (Sec. 2-5).  Where the paper is silent
 * the oracle takes the readings listed in the design notes of the repository;
 * each is repeated at the point of use.
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H
#include <stdint.h>

#define O_MAXS 64   /* support entries per material point          */
#define O_MAXC 16   /* resolved hanging-node constraint entries      */
#define O_MAXK 64   /* overlapped leaves per GIMP domain             */

/* status codes (mirror the meaning of the product library's codes) */
#define O_OK 0
#define O_ERR_ARG 1
#define O_ERR_NEWTON 3
#define O_ERR_KRYLOV 4
#define O_ERR_NAN 5
#define O_ERR_SUPPORT 6
#define O_ERR_BALANCE 8
#define O_ERR_DOMAIN 9

typedef struct {
  /* domain: the closed cube [0,L]^3 (Sec. 3.1) */
  double L;
  int depth_min, depth_max;
  /* strong Dirichlet planes (Sec. 2.4): nodes on the plane x_axis = pos have
   * the components in mask (bit d = component d) fixed to zero increment */
  int nbc;
  int bc_axis[8];
  double bc_pos[8];
  int bc_mask[8];
  /* rigid body (Sec. 2.3): 0 none, 1 flat-ended cylinder, 2 cone + shaft,
   * 3 triangulated surface, 4 sphere */
  int body_kind;
  double body_cx, body_cy, body_z;   /* axis and bottom face / tip height */
  double body_r, body_alpha;         /* radius, cone half angle (rad)     */
  /* adaptivity (Sec. 5) */
  double dx_region, beta;
  /* material (Sec. 2.2): 0 Hencky elastic, 1 von Mises, 2 Drucker-Prager,
   * 3 Drucker-Prager cone with the Willam-Warnke deviatoric section (Sec. 6.4) */
  int model;
  double nu, phi, psi;
  double g[3];
  /* ghost (Sec. 4) and contact (Sec. 2.3) constants */
  double kappa, pf;
  int ghost_on, contact_on;
  /* Coulomb friction (Sec. 2.3): coefficient mu, tangential penalty factor pt
   * (eps_T = pt E_p (V0_p)^(2/3)), and the body's translation over the current
   * load step, against which the contact nodes' slip is measured */
  double mu, pt;
  double body_d[3];
  /* body_kind 3: a closed triangulated surface (Sec. 2.3 represents the rigid
   * bodies by closed triangular faceted meshes): nvert vertices (x, y, z,
   * relative to the body's reference point (body_cx, body_cy, body_z)) and
   * ntri triangles (three vertex indices each, counter-clockwise seen from
   * outside), host arrays */
  int ntri, nvert;
  const double* tri_v;
  const int* tri_t;
  /* body_kind 4: a sphere of radius body_r centred at (body_cx, body_cy,
   * body_z).
   * Dynamics (Sec. 2.4): dt > 0 makes the step a Newmark time step with
   * gamma = 1, beta = 1/2 (dt = 0: a quasi-static load step).  body_free
   * (bits 0-2 translation x, y, z, bits 3-5 rotation about x, y, z) lists
   * the rigid-body degrees of freedom that are unknowns of the Newton
   * iteration, coupled to the material by the contact forces; the others are
   * prescribed (translation body_d over the step, no rotation).  With free
   * components the body pose above is the one at the START of the step, and
   * body_mass, body_inertia (isotropic) and the body's velocity body_v and
   * angular velocity body_w at the step start enter its Newmark equations;
   * rotation may be free for the sphere only. */
  double dt;
  int body_free;
  double body_mass, body_inertia;
  double body_v[3], body_w[3];
} o_params;

typedef struct o_model o_model;

typedef struct {
  int nleaf, nnode, nhang, ndof, nnzb, nghost, npts, maxs;
} o_counts;

typedef struct {
  double load;         /* load factor applied to gravity                  */
  double tol;          /* Newton: ||R_free|| <= tol * f_ref               */
  int maxit;
  double lin_tol;      /* linear solve relative tolerance                  */
  int lin_maxit;
} o_step_params;

typedef struct {
  int newton_its, lin_its_total, status;
  double res_hist[64];
  double reaction[3];
  double eta_hist[64];
  double body_q[6];    /* the rigid body's converged increment over the step */
} o_step_stats;

o_model* o_create(const o_params* prm);
void o_free(o_model* m);
int o_set_points(o_model* m, int n, const double* x, const double* lp, const double* l0,
                 const double* F, const double* be, const double* V0, const double* mass,
                 const double* E, const double* ys);
int o_get_points(const o_model* m, double* x, double* lp, double* l0, double* F, double* be,
                 double* V0, double* mass, double* E, double* ys);
void o_set_body_z(o_model* m, double z);

/* Sec. 5 then Sec. 3: adapt the octree to the body, split GIMPs, build the nodes,
 * hanging constraints, the discrete GIMP basis, the block pattern and the ghost
 * faces.  `nosplit` disables the GIMP refinement step (used by pins). */
int o_build(o_model* m, int nosplit);
void o_counts_get(const o_model* m, o_counts* c);

/* exports (arrays sized from o_counts) */
void o_export_tree(const o_model* m, int* lev, int* anchor /*3*nleaf*/);
void o_export_nodes(const o_model* m, int* coord /*3*nnode*/, int* hang, int* dof,
                    int* cptr /*nnode+1*/, int* cidx, double* cw);
void o_export_support(const o_model* m, int* nsup /*P*/, int* sidx /*P*O_MAXS*/,
                      double* S /*P*O_MAXS*/, double* dS /*P*O_MAXS*3*/);
void o_export_pattern(const o_model* m, int* row_ptr, int* col);
void o_export_ghost(const o_model* m, double* kg /*nnzb scalar ghost coefficient*/);
void o_export_bcmask(const o_model* m, int* mask /*ndof*/);
void o_export_ghost_faces(const o_model* m, int* faces /*4*nghost: K,N,axis,sign*/,
                          int* populated /*nleaf*/);

/* evaluate the background basis of the mesh at arbitrary points (pins) */
int o_eval_background(const o_model* m, const double* x, int* nent, int* idx /*O_MAXS*/,
                      double* phi, double* dphi);

/* Eq. (MPMweak): residual and consistent tangent for a nodal increment du;
 * fint_all (optional) receives f_int over all dofs, then ||f_ext + f_c||, and
 * for time steps ||f_inert|| (3 ndof + 2 doubles) */
int o_assemble(o_model* m, const double* du, double load, double* R, double* Kvals,
               double* fint_all, double* reaction);
/* The same with the rigid body's increment q over the step (translation
 * q[0..2], rotation q[3..5]; prescribed components must hold their
 * prescribed values) and the body's equations: Rb[6] (host) its residual
 * (Newmark inertia, gravity and the contact forces and moments), Kbb[36] its
 * Jacobian in q (row-major), Kgb[6][3 ndof] the derivative of R in each
 * component of q, Kbg[6][3 ndof] the derivative of each component of Rb in
 * du.  Any of the body outputs may be NULL. */
int o_assemble_body(o_model* m, const double* du, const double* q, double load, double* R,
                    double* Kvals, double* fint_all, double* reaction, double* Rb, double* Kbb,
                    double* Kgb, double* Kbg);
/* material point velocities (3 per point, zero until set; children of a
 * GIMP split inherit their parent's) and the rigid body's state:
 * pose[3] (body_cx, body_cy, body_z), v[3], w[3], accumulated rotation
 * theta[3] */
int o_set_velocity(o_model* m, const double* v);
int o_get_velocity(const o_model* m, double* v);
void o_get_body(const o_model* m, double* pose, double* v, double* w, double* theta);
/* linear solve K x = b on the free components (dense LU when small, else PCG/BiCGStab) */
int o_solve(o_model* m, const double* Kvals, const double* b, double* x, double tol, int maxit,
            int* its);
/* one load step (Sec. 2.4, Sec. 5), updates the points */
int o_step(o_model* m, const o_step_params* sp, o_step_stats* st);

/* per-point constitutive update for a given dF (exposed for pins) */
int o_constitutive(const o_params* prm, double E, double ys, const double* be_n, const double* dF,
                   double* tau /*9*/, double* be_new /*6*/, double* A /*81*/, int* plastic);
void o_eig_sym3(const double* a /*9*/, double* lam /*3*/, double* Q /*9 col-major eigvecs*/);

/* signed distance of the rigid body (negative inside), outward normal n and
 * Hessian H (row-major) at x; returns 1 inside (exposed for pins) */
int o_body_sdf(const o_params* p, const double* x, double* phi, double* n /*3*/, double* H /*9*/);

/* point-wise state at the current increment (for parity of stresses) */
int o_point_stress(o_model* m, const double* du, double* sigma /*P*9*/);

#endif
