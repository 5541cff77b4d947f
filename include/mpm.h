/*
 * mpm.h -- C ABI of libmpm_gb300.so: the data-parallel hot path of one load step
 * of the implicit octree-based GIMP Material Point Method (Bird, Coombs,
 * Augarde, Pretti, O'Hare, "An implicit octree-based adaptive Material Point
 * Method").  Every computation behind these calls runs in hand-written CUDA
 * kernels for sm_103a on the stream given to mpm_create.
 *
 * Conventions
 *  - "device" pointers are CUDA global memory of the current device, owned by
 *    the caller unless stated otherwise; "host" pointers are ordinary memory.
 *  - Point arrays are structure-of-arrays in the caller's (canonical) order:
 *      x[3P] centre, lp[3P] current half-lengths, l0[3P] reference
 *      half-lengths, F[9P] row-major deformation gradient, be[6P] elastic left
 *      Cauchy-Green tensor (xx, yy, zz, xy, yz, xz), V0[P] reference volume,
 *      mass[P], E[P] Young's modulus, ys[P] yield stress (von Mises) or
 *      cohesion (Drucker-Prager).  All double precision.
 *  - Nodal vectors are [3*ndof] doubles, component-fastest, dofs numbered in
 *    Morton order of the active independent nodes of the mesh.
 *  - The stiffness is a 3x3 block matrix whose pattern is the sorted CSR
 *    (row_ptr, col) of mpm_mesh_export.  Its values are held in a sliced layout
 *    (slices of 32 block rows, each padded to a width that is a multiple of 4
 *    blocks) sized 9 * nslot entries (mpm_mesh_info.nslot); mpm_blocks_export
 *    reads them back as plain [nnzb][3][3] row-major blocks in CSR order.
 *  - Every call returns an mpm_status; on failure mpm_last_error(ctx) gives a
 *    message.  No call aborts, traps or spins without bound: device-side
 *    failures (support overflow, NaN, Krylov breakdown) come back as status
 *    codes and leave the context usable.
 *  - Calls are asynchronous on the context stream except where they return host
 *    values (counts, statistics, reaction), which synchronise that stream.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_MAXS 64 /* support entries per material point */

typedef enum {
  MPM_OK = 0,
  MPM_ERR_ARG = 1,       /* invalid argument                                  */
  MPM_ERR_CUDA = 2,      /* a CUDA runtime call failed                        */
  MPM_ERR_NEWTON = 3,    /* Newton iterations exhausted                       */
  MPM_ERR_KRYLOV = 4,    /* Krylov iteration cap reached or breakdown         */
  MPM_ERR_NAN = 5,       /* non-finite value or det F <= 0                    */
  MPM_ERR_SUPPORT = 6,   /* support / overlap / constraint list overflow      */
  MPM_ERR_CAPACITY = 7,  /* point capacity too small for the GIMP split       */
  MPM_ERR_BALANCE = 8,   /* octree balance or hanging-node layout failure     */
  MPM_ERR_DOMAIN = 9     /* a GIMP domain lies outside the cube               */
} mpm_status;

typedef enum { MPM_FP64 = 0, MPM_MIXED = 1 } mpm_precision;

/* Problem domain: the closed cube [0,L]^3 of Sec. 3.1, octree depths, and the
 * strong Dirichlet planes of Sec. 2.4 (nodes with coordinate bc_pos on axis
 * bc_axis have the components in bc_mask -- bit d = component d -- fixed). */
typedef struct {
  double L;
  int depth_min, depth_max;
  int nbc;
  int bc_axis[8];
  double bc_pos[8];
  int bc_mask[8];
} mpm_domain;

/* Rigid body of Sec. 2.3: kind 0 none, 1 flat-ended cylinder {z >= z, rho <=
 * r}, 2 cone of half angle alpha with tip at z and a cylindrical shaft of
 * radius r (axis through (cx, cy) for both), 3 a closed triangular faceted
 * mesh (Sec. 2.3's representation of the rigid bodies): nvert vertices tri_v
 * (device, 3 doubles each, relative to the reference point (cx, cy, z)) and
 * ntri triangles tri_t (device, 3 vertex indices each, counter-clockwise seen
 * from outside, every edge shared by two triangles); the arrays are the
 * caller's and must stay the same (up to the reference point) between
 * mpm_octree_build and the assemblies on its mesh.  Its signed distance is
 * that of the nearest surface point over all triangles, signed by the
 * angle-weighted pseudo-normal; Step 1 of Sec. 5 marks a leaf when the ball
 * around it meets the body.  step_d is the body's translation over the
 * current load step: the Coulomb friction of Sec. 2.3 measures the slip of
 * each contact node against it (unused when mu = 0).  Kind 4 is a sphere of
 * radius r centred at (cx, cy, z).
 *
 * A free body (Sec. 2.3 and 2.4: the contact forces "influence any
 * unconstrained degrees of freedom of the rigid body"), for time steps
 * (mpm_step_params.dt > 0) only: `free` lists the body's unknowns, bits 0-2
 * translation along x, y, z and bits 3-5 rotation about x, y, z (rotation
 * for the sphere only); the other components are prescribed (translation
 * step_d over the step, no rotation).  With free components (cx, cy, z) is
 * the pose at the START of the step, `mass` and the isotropic rotational
 * inertia `inertia` enter the body's Newmark equations, and v, w are its
 * velocity and angular velocity at the step start; mpm_step returns the
 * step's increment and the new velocities in mpm_step_stats, and the caller
 * moves the pose by the increment. */
typedef struct {
  int kind;
  double cx, cy, z, r, alpha;
  double step_d[3];
  int ntri, nvert;
  const double* tri_v;
  const int* tri_t;
  int free;
  double mass, inertia;
  double v[3], w[3];
} mpm_rigid;

/* Adaptivity of Sec. 5: refine leaves meeting the body or with a node within
 * dx_region of it (down to depth_max); split GIMPs with l_K < beta l_p. */
typedef struct {
  double dx_region, beta;
} mpm_adapt;

/* Material of Sec. 2.2 (model 0 Hencky elastic, 1 von Mises, 2 Drucker-Prager
 * with friction phi and dilation psi in radians, 3 the CPT material of Sec.
 * 6.4: the frictional cone with a Willam-Warnke deviatoric section, radius 1
 * on the compressive and (3 - sin phi)/(3 + sin phi) on the tensile meridian
 * relative to model 2's outer cone, with model 2's potential), gravity g (Eq. MPMweak body
 * force), ghost constant kappa (Sec. 4), contact penalty factors pf (normal,
 * eps_N = pf E_p (V0_p)^(2/3)) and pt (tangential, eps_T = pt E_p (V0_p)^(2/3))
 * and the Coulomb friction coefficient mu between body and material (Sec.
 * 2.3; mu > 0 makes the tangent non-symmetric, so the Krylov solve is
 * BiCGStab). */
typedef struct {
  int model;
  double nu, phi, psi;
  double g[3];
  double kappa, pf;
  int ghost_on, contact_on;
  double mu, pt;
} mpm_material;

/* Caller-owned device point arrays (layout above).  mpm_octree_build may grow
 * `count` up to `capacity` when it splits GIMPs (Sec. 5).  v[3P]: point
 * velocities, needed by time steps (Sec. 2.4) and updated by them; may be
 * NULL for quasi-static load steps.  Split children inherit their parent's
 * velocity. */
typedef struct {
  int count, capacity;
  double *x, *lp, *l0, *F, *be, *V0, *mass, *E, *ys;
  double* v;
} mpm_points;

typedef struct {
  int nleaf, nnode, nhang, ndof, nnzb, nghost, npts, maxs, ncontact, maxrow, nslot;
} mpm_mesh_info;

typedef struct {
  int method;      /* 0 auto (PCG if symmetric else BiCGStab), 1 PCG, 2 BiCGStab,
                      3 preconditioned by a geometric multigrid V-cycle:
                      PCG for symmetric tangents, BiCGStab (one V-cycle per
                      half-step) for the non-associated Drucker-Prager one,
                      4 restarted GMRES(30) with the block-Jacobi
                      preconditioner (Sec. 6.4 names GMRES with a Jacobi
                      preconditioner as the iterative route), any tangent */
  int precision;   /* mpm_precision of the stored matrix and the inner solve     */
  double tol;      /* relative residual target ||b - K x|| <= tol ||b||           */
  int maxit;       /* cap on Krylov iterations (all refinement rounds together)  */
  double inner_tol;/* MPM_MIXED: relative target of each FP32 inner solve        */
  int mg_reuse;    /* method 3: 0 builds the coarse Galerkin operators from this
                      K; 1 keeps those of the first method-3 solve since the
                      mesh was last built (the fine-level smoother is always
                      rebuilt from K), e.g. across the Newton iterations of one
                      load step: the V-cycle stays symmetric positive definite */
} mpm_solve_params;

typedef struct {
  int iterations, refinements, status;
  double relres;
} mpm_solve_stats;

typedef struct {
  double load;     /* load factor multiplying gravity                          */
  double tol;      /* Newton: ||R_free|| <= tol * max(||f_int||, ||f_ext+f_c||)  */
  int maxit;
  mpm_solve_params lin;
  double* du_out;  /* mpm_step, optional (device): receives the converged nodal
                      increment, 3*ndof doubles in the step's dof numbering, so
                      that mpm_adjoint need not solve the step again           */
  long long du_capacity; /* doubles du_out holds (MPM_ERR_CAPACITY if short) */
  double dt;       /* > 0: a Newmark time step of this length (Sec. 2.4, gamma = 1,
                      beta = 1/2: each point's acceleration at the step end is
                      2 (du_p - dt v_p) / dt^2, du_p = sum_v S_vp du_v, and its
                      velocity becomes v_p + dt a_p; the inertia term of Eq.
                      (MPMweak) joins the residual and the consistent mass
                      times 2 / dt^2 the tangent); 0: a quasi-static load step */
} mpm_step_params;

typedef struct {
  int newton_its, lin_its, status, npts, ndof, nnzb;
  double res_hist[64];
  double eta_hist[64];
  double reaction[3];
  double ms_build, ms_assemble, ms_solve, ms_update;
  /* sizes of the step's mesh, for the benchmark's byte counts: point-support
   * pairs plus ghost-face entries of the row source lists, padded block slots
   * of the sliced stiffness, and the rows and stencil size of the first
   * multigrid level (0 when no multigrid solve ran); npair: the sum over the
   * points of their squared support sizes (the point-pair blocks of the
   * tangent) */
  long long nsrc, nslot;
  int mg_rows1, mg_stencil1;
  long long npair;
  /* a free body's converged increment over the step (translation, rotation;
   * prescribed components at their values) and its velocity and angular
   * velocity at the step end */
  double body_q[6];
  double body_v[3], body_w[3];
} mpm_step_stats;

typedef struct mpm_ctx mpm_ctx;
typedef struct mpm_mesh mpm_mesh;

/* Create a context bound to the current CUDA device and to `stream` (a
 * cudaStream_t; NULL = legacy default stream).  The context owns scratch
 * memory and a device error word; release it with mpm_destroy. */
int mpm_create(mpm_ctx** ctx, void* stream);
int mpm_destroy(mpm_ctx* ctx);
const char* mpm_last_error(const mpm_ctx* ctx);

/* Sec. 5 (Steps 1-3, GIMP refinement) and Sec. 3 (octree, hanging nodes, Eq.
 * GIMP numerical) and Sec. 4 (ghost faces, Eq. ghost): rebuild the octree for
 * the body pose, split GIMPs (pts->count may grow; MPM_ERR_CAPACITY if it would
 * exceed pts->capacity), build nodes, hanging constraints, the discrete GIMP
 * basis, the 3x3 block pattern and the ghost matrix.  `flags` bit 0 disables
 * the GIMP split.  *mesh is created on first use and reused (its buffers grow)
 * when passed back non-NULL.  The mesh keeps a cell-sorted copy of the point
 * state: the points must not change until the mesh is rebuilt. */
int mpm_octree_build(mpm_ctx* ctx, const mpm_domain* dom, const mpm_rigid* body,
                     const mpm_adapt* ad, const mpm_material* mat, mpm_points* pts, int flags,
                     mpm_mesh** mesh);
/* Frees a mesh early.  Meshes still alive when their context is destroyed are
 * freed by mpm_destroy; a mesh must not be used or freed after that. */
int mpm_mesh_free(mpm_mesh* mesh);
/* counts of the mesh (host) */
int mpm_mesh_counts(const mpm_mesh* mesh, mpm_mesh_info* info);

/* Copies one mesh array to host memory for inspection (`what` selects it; see
 * MPM_EXPORT_*), `bytes` is the size of `dst` and must be large enough. */
enum {
  MPM_EXPORT_LEAF_LEVEL = 0,   /* int[nleaf]                                    */
  MPM_EXPORT_LEAF_ANCHOR = 1,  /* int[3*nleaf], finest-grid units               */
  MPM_EXPORT_NODE_COORD = 2,   /* int[3*nnode]                                  */
  MPM_EXPORT_NODE_HANG = 3,    /* int[nnode]                                    */
  MPM_EXPORT_NODE_DOF = 4,     /* int[nnode], -1 for inactive or hanging        */
  MPM_EXPORT_CPTR = 5,         /* int[nnode+1] resolved constraint lists         */
  MPM_EXPORT_CIDX = 6,         /* int[cptr[nnode]] independent node ids          */
  MPM_EXPORT_CW = 7,           /* double[cptr[nnode]] weights                    */
  MPM_EXPORT_NSUP = 8,         /* int[P] support size per point (caller order)   */
  MPM_EXPORT_SIDX = 9,         /* int[P*MPM_MAXS] support dofs, sorted          */
  MPM_EXPORT_S = 10,           /* double[P*MPM_MAXS] S_vp                        */
  MPM_EXPORT_DS = 11,          /* double[P*MPM_MAXS*3] grad S_vp                 */
  MPM_EXPORT_ROW_PTR = 12,     /* int[ndof+1]                                   */
  MPM_EXPORT_COL = 13,         /* int[nnzb]                                     */
  MPM_EXPORT_GHOST = 14,       /* double[nnzb] ghost coefficient per block      */
  MPM_EXPORT_BCMASK = 15,      /* int[ndof] fixed components                    */
  MPM_EXPORT_POPULATED = 16,   /* int[nleaf]                                    */
  MPM_EXPORT_GHOST_FACES = 17, /* int[4*nghost]: K, N, axis, sign              */
  MPM_EXPORT_MG_LEVELS = 18    /* int[32]: per multigrid coarse level (up to 8):
                                  depth, rows, stencil radius, stencil size;
                                  zeros until a method-3 solve on this mesh */
};
int mpm_mesh_export(const mpm_mesh* mesh, int what, void* dst, size_t bytes);

/* Eq. (MPMweak), static part, with the ghost term of Sec. 4 and the penalty
 * contact of Sec. 2.3: for the nodal increment du (device [3*ndof]) of the
 * current load step, R (device [3*ndof]) = f_int - load*f_ext - f_c + K_G du and,
 * if K_values (device [9*nslot], double for MPM_FP64, float for MPM_MIXED) is
 * non-NULL, the consistent tangent with the Dirichlet rows and columns
 * replaced by identity.  reaction (host [3], may be NULL) receives the force of
 * the material on the rigid body.  fint_norms (host [2], may be NULL) receives
 * ||f_int|| and ||f_ext + f_c||. */
int mpm_assemble(mpm_ctx* ctx, const mpm_mesh* mesh, const mpm_material* mat,
                 const mpm_rigid* body, const double* du, double load, int precision, double* R,
                 void* K_values, double* reaction, double* fint_norms);

/* Eq. (MPMweak) with its inertia term (Sec. 2.4) and the rigid body's
 * equations of a time step: mpm_assemble's R and K_values at the nodal
 * increment du for a Newmark step of length dt > 0 (the mesh must have been
 * built from points with velocities), with the body's increment q (host [6]:
 * translation, rotation over the step; prescribed components at their
 * values) and, for a free body, Rb (host [6]) its residual m a - m g +
 * sum f, J alpha + sum d x f (f the contact force on the material at a node,
 * d the node's offset from the body centre), Kbb (host [36], row-major) its
 * derivative in q, Kgb (device [6][3*ndof]) the derivative of R in each
 * component of q and Kbg (device [6][3*ndof]) the derivative of each
 * component of Rb in du.  Any of Rb, Kbb, Kgb, Kbg, K_values may be NULL.
 * fint_norms (host [3], may be NULL): ||f_int||, ||f_ext + f_c||,
 * ||f_inert||.  Synchronises the stream. */
int mpm_assemble_body(mpm_ctx* ctx, const mpm_mesh* mesh, const mpm_material* mat,
                      const mpm_rigid* body, const double* du, const double* q, double dt,
                      double load, int precision, double* R, void* K_values, double* reaction,
                      double* fint_norms, double* Rb, double* Kbb, double* Kgb, double* Kbg);

/* Copies stiffness values (as written by mpm_assemble with `precision`) to host
 * memory as [nnzb][3][3] row-major blocks in the CSR order of the pattern;
 * blocks_host must hold 9*nnzb doubles.  Synchronises the stream. */
int mpm_blocks_export(mpm_ctx* ctx, const mpm_mesh* mesh, const void* K_values, int precision,
                      double* blocks_host);

/* Preconditioned Krylov solve of K x = rhs on the free components (Sec. 1 names
 * Krylov solvers with a Jacobi-type preconditioner as the scalable option), 3x3
 * block-Jacobi preconditioner; MPM_MIXED runs FP32 inner solves inside FP64
 * iterative refinement.  K_values as produced by mpm_assemble with the same
 * precision; rhs, x device [3*ndof] doubles (x is overwritten). */
int mpm_solve(mpm_ctx* ctx, const mpm_mesh* mesh, const mpm_material* mat, const void* K_values,
              const double* rhs, double* x, const mpm_solve_params* prm, mpm_solve_stats* stats);

/* One load step (Sec. 2.4 Newton-Raphson with line search, Sec. 5
 * re-adaptation): rebuild the mesh for the body pose, iterate assemble/solve
 * until converged, then update the points (positions, F, b_e, domain sizes,
 * and for a time step their velocities).  A quasi-static load step when
 * prm->dt = 0, a Newmark time step when dt > 0 (then pts->v is required).
 * With a free body (mpm_rigid.free) each Newton iteration solves the linear
 * system of the material and body increments, the body's part by block
 * elimination: w = K^-1 (-R), Z = K^-1 dR/dq (one solve per free component),
 * (dRb/dq - dRb/du Z) dq = -Rb - dRb/du w, du = w - Z dq; the convergence test
 * takes the free components of the body's residual Rb into ||R_free|| and
 * the body's weight and the material's inertia force into the reference.
 * stats (host) receives the history.  The mesh is kept in the context. */
int mpm_step(mpm_ctx* ctx, const mpm_domain* dom, const mpm_rigid* body, const mpm_adapt* ad,
             const mpm_material* mat, mpm_points* pts, const mpm_step_params* prm,
             mpm_step_stats* stats);

/* Discrete adjoint of a sequence of load steps (the paper differentiates
 * nothing; this is the reverse mode of the Sec. 2.4 load step with the Sec. 5
 * re-adaptation, for inverse problems on the per-point material constants).
 *
 * ckpts[n] (n = 0..nsteps-1) is the point state at the START of load step n
 * (device SoA, before that step's GIMP splits) with the body position
 * `body_z` and the load factor `load` that the step used.  Only the first
 * `count` rows of each array are read; the largest `capacity` over the
 * checkpoints sizes the library's working copy and must hold every split of
 * every step (MPM_ERR_CAPACITY otherwise).  A rebuilt step whose point count
 * differs from the next checkpoint's is rejected with MPM_ERR_ARG.  The functional is J = w . reaction, the reaction
 * force on the body at the converged end of the last step, with w =
 * dJ_dreaction (host [3]).  Every discrete event (octree, splits, supports,
 * plastic/elastic branch of each point, contact candidates, ghost faces and
 * their beta) is frozen at its forward value, so J is differentiated where it
 * is smooth.  Per step, in reverse: rebuild the mesh from the checkpoint,
 * take the converged increment the forward stored in the checkpoint (`du`,
 * from mpm_step_params.du_out; the rebuild reproduces its dof numbering) or,
 * without one, re-solve Newton (prm: the forward's Newton and Krylov settings;
 * prm->load is ignored, each checkpoint carries its own), solve K mu = dJ/du with the
 * FP64 consistent tangent by PCG to prm->lin.tol within prm->lin.maxit
 * iterations (multigrid-preconditioned if prm->lin.method is 3, else block
 * Jacobi) (K is symmetric for material models 0 and 1;
 * model 2 is rejected with MPM_ERR_ARG), and run the backward kernels of the
 * residual, the point
 * update, the contact, the ghost term and the GIMP basis.
 * Outputs dJ_dE, dJ_dys: device [ckpts[0].pts.count] doubles (overwritten).
 * The checkpoint arrays are only read.  stats (host, optional) receives the
 * reaction of the last step, the adjoint Krylov iterations and the time of
 * the forward re-solves and of the backward work. */
typedef struct {
  mpm_points pts;
  double body_z;
  double load;
  const double* du;  /* optional (device): the step's converged increment   */
  long long du_len;  /* its length, 3*ndof (MPM_ERR_ARG if it does not match) */
} mpm_checkpoint;

typedef struct {
  int status, lin_its;
  double reaction[3];
  double ms_forward, ms_backward;
} mpm_adjoint_stats;

int mpm_adjoint(mpm_ctx* ctx, const mpm_domain* dom, const mpm_rigid* body, const mpm_adapt* ad,
                const mpm_material* mat, const mpm_checkpoint* ckpts, int nsteps,
                const mpm_step_params* prm, const double* dJ_dreaction, double* dJ_dE,
                double* dJ_dys, mpm_adjoint_stats* stats);

/* Allocation-free variant of mpm_solve (the paper has no counterpart).  For
 * callers that cannot allocate device memory while they solve -- for example
 * an application whose device memory is already handed out by its own pool,
 * so that a cudaMalloc would fail or fragment it, or a latency-bound loop that
 * cannot afford an allocation on its first call.  It runs the FP64 3x3
 * block-Jacobi PCG of mpm_solve (precision MPM_FP64, method PCG) with every
 * work vector, the preconditioner, the scalars and the partial sums of its
 * fixed-order reductions placed in one static device array of 32 MiB that the
 * library reserves on each device that loads it and keeps until the process
 * exits; the call itself allocates nothing.
 * Limit: 16,896 + 224 * 32 * ceil(ndof / 32) bytes must fit (vectors padded
 * to 4 components and to whole slices of 32 rows), i.e. at most 149,696 dofs
 * (449,088 unknowns); larger meshes are rejected with MPM_ERR_ARG and a
 * message.  The context's device must be the current device (MPM_ERR_ARG
 * otherwise).  The first call on a device looks up the array's device address,
 * so make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents (each call clears what must
 * start at zero): calls that overlap on the GPU, from any stream or context,
 * race with each other.  K_values (FP64, from mpm_assemble), rhs and x as in
 * mpm_solve; tol > 0 and maxit > 0. */
int mpm_solve_static(mpm_ctx* ctx, const mpm_mesh* mesh, const double* K_values, const double* rhs,
                     double* x, double tol, int maxit, mpm_solve_stats* stats);

/* Measurement hooks (no counterpart in the paper; they serve the benchmark):
 * CUDA events recorded on the context stream around every launch of the
 * tracked kernel classes below, and a count of all kernel launches made by
 * the library.  mpm_profile(ctx, 1) clears the totals and starts recording,
 * mpm_profile(ctx, 0) stops; mpm_profile_read synchronises the stream and
 * returns, per class, the launches and the summed milliseconds (host arrays
 * of MPM_PROF_NCLASS entries). */
enum {
  MPM_PROF_PCG_UPDATE = 0,   /* PCG vector update + preconditioner + dots       */
  MPM_PROF_PCG_SPMV = 1,     /* PCG SpMV fused with the direction update        */
  MPM_PROF_TANGENT = 2,      /* row-gather tangent assembly                     */
  MPM_PROF_CONSTITUTIVE = 3, /* per-point return map (+ spatial tangent)        */
  MPM_PROF_KINEMATICS = 4,   /* per-point dF                                     */
  MPM_PROF_FORCE = 5,        /* spatial basis gradients for the tangent          */
  MPM_PROF_BASIS = 6,        /* discrete GIMP basis                              */
  MPM_PROF_RESIDUAL = 7,     /* residual rows: internal force gather, ghost term */
  MPM_PROF_CONTACT = 8,      /* penalty contact                                  */
  MPM_PROF_BICG_SPMV = 9,    /* BiCGStab SpMV                                    */
  MPM_PROF_REFINE = 10,      /* FP64 refinement residual                         */
  MPM_PROF_PATTERN = 11,     /* block pattern rows                               */
  MPM_PROF_MG = 12,          /* V-cycle kernels below level 1 and the transfers  */
  MPM_PROF_MG_SETUP = 13,    /* multigrid smoother inverses and FP16 copy        */
  MPM_PROF_MG_FINE = 14,     /* V-cycle fine-level residual and smoothing        */
  MPM_PROF_MG_LEVEL1 = 15,   /* V-cycle level-1 residual and smoothing           */
  MPM_PROF_MG_RAP = 16,      /* multigrid Galerkin products                      */
  MPM_PROF_NCLASS = 17
};
int mpm_profile(mpm_ctx* ctx, int enable);
int mpm_profile_read(mpm_ctx* ctx, long long* launches, double* ms);
int mpm_launch_count(const mpm_ctx* ctx, long long* launches);

/* Measured FP64 fused multiply-add throughput of the context's GPU (no
 * counterpart in the paper; the roofline of the kernels that the precision
 * pattern keeps in FP64): independent FMA chains on every SM, timed with CUDA
 * events on the context stream for about `seconds` (0.05 to 10).
 * flops_per_s (host) receives 2 x FMAs / s, ms (host, may be NULL) the timed
 * duration.  Synchronises the stream. */
int mpm_fp64_peak(mpm_ctx* ctx, double seconds, double* flops_per_s, double* ms);

#ifdef __cplusplus
}
#endif
#endif
