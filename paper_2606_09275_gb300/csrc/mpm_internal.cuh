// Internal declarations of libmpm_gb300: context, mesh, device helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "mpm.h"

namespace mpm {

constexpr int MAXS = MPM_MAXS;   // support entries per point
constexpr int MAXC = 16;         // resolved constraint entries per node
constexpr int MAXK = 27;         // leaves overlapped by one GIMP domain (basis)
constexpr int SPLIT_STACK = 64;  // work list of the split test (overflow => split)
constexpr int MAXE = 512;        // (leaf corner, constraint) entries of one domain
constexpr int MAXCB = 32;        // background-basis entries at a contact corner
constexpr int MAXG = 64;         // dofs of one ghost face, I(K+) u I(K-)
constexpr int HASH = 2048;       // per-warp hash set of the pattern builder
constexpr int MAXROW = 1024;     // blocks in one row of the stiffness

// device error word bits
enum : int {
  EB_SUPPORT = 1,
  EB_NAN = 2,
  EB_BALANCE = 4,
  EB_DOMAIN = 8,
  EB_ROW = 16,
  EB_KRYLOV = 32
};

struct Geo {
  int D;        // finest level
  int N;        // 2^D finest cells per axis
  double L;     // cube side
  double unit;  // L / 2^D
  double scale; // 2^D / L
};

// the rigid body as the kernels see it: the caller's description and, for a
// triangulated body (kind 3), its pseudo-normals (computed with the mesh)
// and the bounding box of its vertices (body frame)
struct Body {
  mpm_rigid b;
  const double* fn;     // [ntri][3] unit face normals
  const double* en;     // [ntri][3][3] edge pseudo-normals (edges v0v1, v1v2, v2v0)
  const double* vn;     // [nvert][3] angle-weighted vertex pseudo-normals
  double lo[3], hi[3];  // vertex bounding box
};

struct CudaError : std::runtime_error {
  int code;
  CudaError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define MPM_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw ::mpm::CudaError(MPM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct ProfEv {
  int cls;
  cudaEvent_t a, b;
};

// one round of GIMP splitting (kept when the mesh records its splits)
struct SplitRound {
  int P = 0, cnt = 0;
  Buf flag, rank;
};

// device scalars of one Krylov solve: rotating slots k % 3 of r.z, p.q, r.r,
// ||b||^2 and the stopping threshold; the solve is over once `done` is set
struct Scal {
  double rz[3], pq[3], rr[3];
  double bb, thr;    // ||b||^2 and tol^2 ||b||^2
  double a[8];       // BiCGStab scalars
  int done, iters, breakdown, pad;
};

// storage of a fixed-order grid sum (grid_sum below)
struct GridRed {
  double* part;      // [NV][gridDim.x] partials
  unsigned* ticket;  // 0 before and after each launch
};

// one coarse level of the geometric multigrid: the active nodes of the uniform
// grid of depth d, a Galerkin operator stored per stencil offset (a cube of
// side 2R+1 around each node), the smoother's 3x3 inverses and level vectors
struct MGLevel {
  int d = 0, n1 = 0;           // depth, nodes per axis (2^d + 1)
  int nrow = 0, npad = 0;      // active nodes, padded to 32
  int R = 2, S = 125;          // stencil radius and size (2R+1)^3
  Buf gid, xyz, mask;          // grid node -> row (-1), row -> packed coords, fixed bits
  Buf A, Dinv, b, x, r;        // operator [S*9][npad], inverses [npad][12], vectors [npad][4]
};

// a V-cycle captured as a CUDA graph, replayed while its key (the pointers
// and sizes its launches take) is unchanged
struct VGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t key = 0;
  long long used = 0;          // last use (for replacement)
  int nkern = 0;
};

struct MGData {
  static constexpr int NVG = 8;
  VGraph vg[NVG];              // cached V-cycle graphs
  long long vg_clock = 0;
  bool graphs_off = false;     // a capture failed: plain launches
  long long gen = -1;          // mesh build the structure belongs to
  long long num_gen = -1;      // mesh build of the last coarse operators
  int prec = -1;               // value precision of the coarse operators
  int nlev = 0;                // coarse levels (the last one is solved densely)
  MGLevel lev[8];
  Buf p_idx, p_w;              // fine dof -> up to 8 level-1 rows and weights
  Buf t_ptr, t_idx, t_w;       // the transpose: level-1 row -> (fine dof, weight), by dof
  int t_max = 0;               // longest row of the transpose
  Buf acc;                     // 64-bit fixed-point accumulator of a Galerkin product
  Buf kp, kpc;                 // K P of every fine row over the 4^3 level-1 nodes around its cell, the cell
  Buf bound;                   // per level: largest l1 norm of an operator row (double bits)
  Buf fDinv, fx, fr;           // fine smoother inverses, fine V-cycle vectors
  Buf fKh;                     // FP16 copy of the fine matrix (mixed path)
  Buf cinv;                    // dense inverse of the coarsest operator
  int n3c = 0;
};

}  // namespace mpm

// every kernel launch of the library goes through these: the launch count is
// reported by mpm_launch_count; MPM_LAUNCH_P also brackets it with events
#define MPM_COUNT(ctx) (++(ctx)->nlaunch)
#define MPM_LAUNCH(...) \
  do {                  \
    __VA_ARGS__;        \
    MPM_COUNT(c);       \
  } while (0)
#define MPM_LAUNCH_P(cls, ...) \
  do {                         \
    ::mpm::prof_begin(c, cls); \
    __VA_ARGS__;               \
    MPM_COUNT(c);              \
    ::mpm::prof_end(c);        \
  } while (0)

struct mpm_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream on which CUDA graphs are captured
  int device = 0;
  int* d_err = nullptr;        // device error word
  double* d_red = nullptr;     // device reduction slots (64 doubles)
  // fixed-order grid sums (mpm::GridRed): per-block partials and the ticket
  // that elects the last block; the ticket is zero between launches
  mpm::Buf part;
  unsigned* d_ticket = nullptr;
  double* h_red = nullptr;     // pinned host mirror
  int* h_int = nullptr;        // pinned host ints (counts)
  mpm::Buf cub_tmp;            // CUB temporary storage
  mpm::Buf tmp[8];             // general scratch
  std::string err;
  mpm_mesh* step_mesh = nullptr;
  std::vector<mpm_mesh*> meshes;  // meshes made by mpm_octree_build, freed with the context
  // Newton / Krylov work vectors (grown on demand)
  mpm::Buf v[32];
  // measurement: launch count and optional per-class CUDA-event timing
  long long nlaunch = 0;
  bool prof_on = false;
  std::vector<mpm::ProfEv> prof;
  std::vector<cudaEvent_t> evpool;
  double prof_ms[MPM_PROF_NCLASS] = {};
  long long prof_n[MPM_PROF_NCLASS] = {};
};

struct mpm_mesh {
  mpm_ctx* ctx = nullptr;
  mpm::Geo g{};
  mpm_domain dom{};
  mpm_rigid body{};
  mpm_adapt ad{};
  mpm_material mat{};
  // octree leaves, Morton order of the anchor
  int nleaf = 0;
  mpm::Buf leaf_key, leaf_lev, leaf_tmp_key, leaf_tmp_lev, flag, scan;
  // nodes
  int nnode = 0, nhang = 0, ncon = 0;
  mpm::Buf node_key, corner, hang, owner, cptr, cidx, cw, node_dof;
  // dofs
  int ndof = 0;
  mpm::Buf dof_node, dof_mask;
  // points, in cell-sorted order (perm: sorted index -> caller index)
  int np = 0, maxs = 0;
  mpm::Buf perm, pcell, px, plp, pl0, pF, pbe, pV0, pmass, pE, pys;
  mpm::Buf nsup, sidx, S, dS;
  mpm::Buf populated, betaK, isB;
  // ghost faces
  int nghost = 0;
  mpm::Buf gface, gdof, gn;
  // pattern (sorted CSR over dofs) and its sliced storage: slices of 32 block
  // rows, each padded to a width that is a multiple of 4 blocks
  int nnzb = 0, maxrow = 0;
  mpm::Buf row_ptr, col, kg, rowcnt;
  int nslice = 0;
  long long nslot = 0;                  // padded block slots of the sliced storage
  mpm::Buf slice_w, slice_base, scol;   // width, first slot of each slice, slot columns
  mpm::Buf srow, spos;                  // storage row -> dof row, and back (npad each)
  // sources of each row: (sorted point or ghost face) << 6 | local index
  long long nsrc = 0;
  long long npair = 0;  // sum of squared support sizes (host copy, read after the build)
  mpm::Buf src_key, src_ptr;
  // gravity force at load 1
  mpm::Buf fext;
  // contact candidates (sorted point ids) and the basis at their 8 corners
  int ncand = 0;
  mpm::Buf cand, cb_n, cb_idx, cb_phi, cb_y0;
  // the transpose of the corner basis: nct rows, each with its (corner << 5 |
  // entry) list sorted; per-assembly corner forces, stiffness and flags
  int nct = 0;
  mpm::Buf ct_row, ct_ptr, ct_ent, cc_f, cc_k, cc_on;
  // ghost faces: jumps J at the 4 Gauss points (4 x MAXG) and the coefficient
  mpm::Buf gJ, gcoef;
  // triangulated body of the build: pseudo-normals and vertex bounding box
  mpm::Buf tri_fn, tri_en, tri_vn;
  double tri_lo[3] = {0, 0, 0}, tri_hi[3] = {0, 0, 0};
  // per-iteration point data (Mf: V0 tau dF^-T, 12 per point)
  mpm::Buf dF, dFinv, tau, Aalg, gx, Mf, V0t;
  mpm::Buf dS32;                        // FP32 copy of dS for the mixed tangent's grad_x S
  mpm::Buf pv;                          // sorted point velocities (time steps)
  bool has_v = false;                   // the points of this mesh build carried velocities
  mpm::Buf cc_t, cc_d;                  // per contact corner: d f / d(rotation), offset from the body centre
  mpm::Buf cc_b;                        // the body's contact sums (42 doubles)
  mpm::Buf pma;                         // per point m_p a_p of a time step
  long long dS32_gen = -1;              // build the copy belongs to
  mpm::Buf lawst;  // spectral state of the last residual-only evaluation (22 per point)
  int built = 0;
  long long gen = 0;                    // incremented by every build
  mpm::MGData* mg = nullptr;            // multigrid structure (built on first use)
  bool record_splits = false;
  std::vector<mpm::SplitRound> split_log;
};

namespace mpm {
// The sliced storage of the stiffness: slices of 32 storage rows, each as
// wide as its longest row rounded up to 4 blocks.  Storage row sr holds the
// dof row row[sr]: within each window of 256 storage rows (8 slices) the dof
// rows are ordered by decreasing length (ties by dof), so that the rows of a
// slice have nearly the same length and the slices carry little padding;
// pos[] is the inverse map.  Rows beyond ndof (the last slice's padding)
// are stored in place.  Vectors stay in dof order.
// sliced_slot: position of block idx of storage row sr (block slot index);
// entry e of that block lives at values[9*base + e*32*w + slot - base] where
// base/w are the slice's first slot and width
struct Sliced {
  const int* w;          // width (blocks) of each slice
  const long long* base; // first slot of each slice
  const int* scol;       // column of each slot (padding slots: the row itself)
  const int* row;        // dof row of each storage row
  const int* pos;        // storage row of each dof row
};
constexpr int SLICE_WINDOW = 256;  // storage rows over which the dof rows are sorted
__host__ __device__ inline long long sliced_slot(long long base, int sr, int idx) {
  return base + ((long long)(idx >> 2) * 32 + (sr & 31)) * 4 + (idx & 3);
}
__host__ __device__ inline long long sliced_entry(long long base, int w, long long slot, int e) {
  return 9 * base + (long long)e * 32 * w + (slot - base);
}
}  // namespace mpm

namespace mpm {

// ------------------------------------------------------------------ growable buffers

inline void* grow_bytes(mpm_ctx* c, Buf& b, size_t need) {
  if (need == 0) need = 16;
  if (need > b.bytes) {
    if (b.p) MPM_CUDA(cudaFreeAsync(b.p, c->stream));
    b.p = nullptr;
    size_t nb = need + need / 4 + 256;
    MPM_CUDA(cudaMallocAsync(&b.p, nb, c->stream));
    b.bytes = nb;
  }
  return b.p;
}

template <class T>
inline T* grow(mpm_ctx* c, Buf& b, size_t n) {
  return (T*)grow_bytes(c, b, n * sizeof(T));
}

template <class T>
inline T* ptr(const Buf& b) {
  return (T*)b.p;
}

// the kernels' view of a mesh's sliced storage
inline Sliced sliced_view(const mpm_mesh* m) {
  return Sliced{ptr<int>(m->slice_w), ptr<long long>(m->slice_base), ptr<int>(m->scol), ptr<int>(m->srow),
                ptr<int>(m->spos)};
}

inline void free_buf(mpm_ctx* c, Buf& b) {
  if (b.p) cudaFreeAsync(b.p, c->stream);
  b.p = nullptr;
  b.bytes = 0;
}

// partial-sum storage for a grid sum of nv values over `blocks` blocks
inline GridRed grid_red(mpm_ctx* c, int nv, long long blocks) {
  double* p = grow<double>(c, c->part, (size_t)nv * (size_t)(blocks < 1 ? 1 : blocks));
  return GridRed{p, c->d_ticket};
}

// at least one block: an empty grid is a launch error, and every kernel
// bounds-checks its index
inline int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ Morton codes

__host__ __device__ inline uint64_t spread3(uint64_t v) {
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

__host__ __device__ inline uint32_t compact3(uint64_t v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return (uint32_t)v;
}

__host__ __device__ inline uint64_t morton(int x, int y, int z) {
  return spread3((uint64_t)x) | (spread3((uint64_t)y) << 1) | (spread3((uint64_t)z) << 2);
}

__host__ __device__ inline void demorton(uint64_t k, int* a) {
  a[0] = (int)compact3(k);
  a[1] = (int)compact3(k >> 1);
  a[2] = (int)compact3(k >> 2);
}

// leaf holding finest cell (x,y,z): last anchor key <= key(cell)
__device__ inline int locate(const uint64_t* __restrict__ key, int n, int x, int y, int z) {
  uint64_t k = morton(x, y, z);
  int lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(key + mid) <= k)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// box bound in finest-grid units, moved onto a grid plane when within 1e-9
__device__ inline double snap_grid(double v) {
  double r = floor(v + 0.5);
  return fabs(v - r) < 1e-9 ? r : v;
}

// ------------------------------------------------------------------ rigid body geometry

__device__ inline double body_rxy(const mpm_rigid& b, const double* lo, const double* hi) {
  double dx = fmax(fmax(lo[0] - b.cx, 0.0), b.cx - hi[0]);
  double dy = fmax(fmax(lo[1] - b.cy, 0.0), b.cy - hi[1]);
  return sqrt(dx * dx + dy * dy);
}

// ---- triangulated body (kind 3): signed distance of the nearest surface
// point over all triangles (the first triangle attaining the smallest
// distance), signed by the pseudo-normal of the feature holding it (face,
// edge: sum of the two face normals, vertex: angle-weighted sum)

__device__ inline void tri_vertex(const Body& B, int v, double* o) {
  o[0] = B.b.tri_v[3 * (size_t)v] + B.b.cx;
  o[1] = B.b.tri_v[3 * (size_t)v + 1] + B.b.cy;
  o[2] = B.b.tri_v[3 * (size_t)v + 2] + B.b.z;
}

// Products and sums below are taken one rounding at a time (no fused
// multiply-add), in the order of the plain expressions: the nearest triangle
// and its feature are discrete decisions, taken the same way wherever this
// code is compiled.
__device__ inline double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ inline double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ inline double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ inline double rdot3(const double* a, const double* b) {
  return radd(radd(rmul(a[0], b[0]), rmul(a[1], b[1])), rmul(a[2], b[2]));
}

// nearest point q of triangle (a, b, c) to x by the Voronoi regions of its
// vertices, edges and face; feature 0 face, 1..3 edges ab, bc, ca, 4..6
// vertices a, b, c
__device__ inline int tri_nearest(const double* x, const double* a, const double* b,
                                  const double* c, double* q) {
  double ab[3], ac[3], ax[3], bx[3], cx[3];
  for (int d = 0; d < 3; ++d) {
    ab[d] = rsub(b[d], a[d]);
    ac[d] = rsub(c[d], a[d]);
    ax[d] = rsub(x[d], a[d]);
  }
  double d1 = rdot3(ab, ax), d2 = rdot3(ac, ax);
  if (d1 <= 0.0 && d2 <= 0.0) {
    for (int d = 0; d < 3; ++d) q[d] = a[d];
    return 4;
  }
  for (int d = 0; d < 3; ++d) bx[d] = rsub(x[d], b[d]);
  double d3 = rdot3(ab, bx), d4 = rdot3(ac, bx);
  if (d3 >= 0.0 && d4 <= d3) {
    for (int d = 0; d < 3; ++d) q[d] = b[d];
    return 5;
  }
  double vc = rsub(rmul(d1, d4), rmul(d3, d2));
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    double v = d1 / rsub(d1, d3);
    for (int d = 0; d < 3; ++d) q[d] = radd(a[d], rmul(v, ab[d]));
    return 1;
  }
  for (int d = 0; d < 3; ++d) cx[d] = rsub(x[d], c[d]);
  double d5 = rdot3(ab, cx), d6 = rdot3(ac, cx);
  if (d6 >= 0.0 && d5 <= d6) {
    for (int d = 0; d < 3; ++d) q[d] = c[d];
    return 6;
  }
  double vb = rsub(rmul(d5, d2), rmul(d1, d6));
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    double w = d2 / rsub(d2, d6);
    for (int d = 0; d < 3; ++d) q[d] = radd(a[d], rmul(w, ac[d]));
    return 3;
  }
  double va = rsub(rmul(d3, d6), rmul(d5, d4));
  double e43 = rsub(d4, d3), e56 = rsub(d5, d6);
  if (va <= 0.0 && e43 >= 0.0 && e56 >= 0.0) {
    double w = e43 / radd(e43, e56);
    for (int d = 0; d < 3; ++d) q[d] = radd(b[d], rmul(w, rsub(c[d], b[d])));
    return 2;
  }
  double den = 1.0 / radd(radd(va, vb), vc), v = rmul(vb, den), w = rmul(vc, den);
  for (int d = 0; d < 3; ++d) q[d] = radd(radd(a[d], rmul(v, ab[d])), rmul(w, ac[d]));
  return 0;
}

// distance from x to the vertex bounding box (a lower bound of the distance
// to the body)
__device__ inline double tri_box_distance(const Body& B, const double* x) {
  const double o[3] = {B.b.cx, B.b.cy, B.b.z};
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double e = fmax(fmax(B.lo[d] + o[d] - x[d], 0.0), x[d] - (B.hi[d] + o[d]));
    s += e * e;
  }
  return sqrt(s);
}

// signed distance at x with gradient n and Hessian H (n, H may be null):
// H is zero on a face, (I - e e^T - u u^T)/phi at an edge of direction e,
// (I - u u^T)/phi at a vertex, u = (x - q)/|x - q|
__device__ inline double tri_sdf(const Body& B, const double* x, double* n, double* H) {
  const int* T = B.b.tri_t;
  double best = 1e300, qb[3] = {0.0, 0.0, 0.0};
  int tb = -1, fb = 0;
  for (int t = 0; t < B.b.ntri; ++t) {
    double a[3], b[3], c[3], q[3];
    tri_vertex(B, T[3 * (size_t)t], a);
    tri_vertex(B, T[3 * (size_t)t + 1], b);
    tri_vertex(B, T[3 * (size_t)t + 2], c);
    int f = tri_nearest(x, a, b, c, q);
    double rr[3] = {rsub(x[0], q[0]), rsub(x[1], q[1]), rsub(x[2], q[2])};
    double d2 = rdot3(rr, rr);
    if (d2 < best) {
      best = d2;
      tb = t;
      fb = f;
      qb[0] = q[0];
      qb[1] = q[1];
      qb[2] = q[2];
    }
  }
  if (n) n[0] = n[1] = n[2] = 0.0;
  if (H)
    for (int i = 0; i < 9; ++i) H[i] = 0.0;
  if (tb < 0) return 1e300;
  double dist = sqrt(best);
  double r[3] = {rsub(x[0], qb[0]), rsub(x[1], qb[1]), rsub(x[2], qb[2])};
  const double* nt = B.fn + 3 * (size_t)tb;
  // x - q along the nearest triangle's normal: the surface is flat there
  double cr[3] = {rsub(rmul(r[1], nt[2]), rmul(r[2], nt[1])), rsub(rmul(r[2], nt[0]), rmul(r[0], nt[2])),
                  rsub(rmul(r[0], nt[1]), rmul(r[1], nt[0]))};
  if (fb != 0 && rdot3(cr, cr) <= 1e-24 * best) fb = 0;
  const double* N = fb == 0 ? nt
                            : (fb <= 3 ? B.en + 9 * (size_t)tb + 3 * (fb - 1)
                                       : B.vn + 3 * (size_t)T[3 * (size_t)tb + fb - 4]);
  double sg = rdot3(r, N) < 0.0 ? -1.0 : 1.0;
  if (!(dist > 0.0)) return 0.0;
  double phi = sg * dist;
  double u[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
  if (n) {
    for (int d = 0; d < 3; ++d) n[d] = fb == 0 ? nt[d] : sg * u[d];
  }
  if (H && fb != 0) {
    double e[3] = {0.0, 0.0, 0.0};
    if (fb <= 3) {
      double a[3], b[3];
      tri_vertex(B, T[3 * (size_t)tb + fb - 1], a);
      tri_vertex(B, T[3 * (size_t)tb + fb % 3], b);
      double l = sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) +
                      (b[2] - a[2]) * (b[2] - a[2]));
      for (int d = 0; d < 3; ++d) e[d] = (b[d] - a[d]) / l;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        H[3 * i + j] = ((i == j ? 1.0 : 0.0) - e[i] * e[j] - u[i] * u[j]) / phi;
  }
  return phi;
}

// does the closed box meet the solid body?  (triangulated body: when the
// ball around the box meets it)
__device__ inline bool body_meets_box(const Body& B, const double* lo, const double* hi) {
  const mpm_rigid& b = B.b;
  if (b.kind == 3) {
    double c[3], h2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      c[d] = 0.5 * (lo[d] + hi[d]);
      h2 += 0.25 * (hi[d] - lo[d]) * (hi[d] - lo[d]);
    }
    double hd = sqrt(h2);
    if (tri_box_distance(B, c) > hd) return false;  // (then the distance is > hd too)
    return tri_sdf(B, c, nullptr, nullptr) <= hd;
  }
  if (b.kind == 1) return hi[2] >= b.z && body_rxy(b, lo, hi) <= b.r;
  if (b.kind == 4) {
    // sphere: the box's nearest point to the centre is inside the ball
    const double c[3] = {b.cx, b.cy, b.z};
    double s2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      double e = fmax(fmax(lo[d] - c[d], 0.0), c[d] - hi[d]);
      s2 += e * e;
    }
    return sqrt(s2) <= b.r;
  }
  if (b.kind == 2) {
    if (hi[2] < b.z) return false;
    double rmax = fmin((hi[2] - b.z) * tan(b.alpha), b.r);
    return body_rxy(b, lo, hi) <= rmax;
  }
  return false;
}

__device__ inline double dist_to_segment(double px, double pz, double ax, double az, double bx,
                                         double bz) {
  double vx = bx - ax, vz = bz - az;
  double t = ((px - ax) * vx + (pz - az) * vz) / (vx * vx + vz * vz);
  t = fmin(fmax(t, 0.0), 1.0);
  double qx = ax + t * vx - px, qz = az + t * vz - pz;
  return sqrt(qx * qx + qz * qz);
}

// Euclidean distance from a point to the solid (0 inside); callers compare it
// with thr, and where it is surely above thr (triangulated body farther than
// thr from its bounding box) a lower bound above thr is returned instead
__device__ inline double body_distance(const Body& B, const double* x, double thr) {
  const mpm_rigid& b = B.b;
  if (b.kind == 3) {
    double lb = tri_box_distance(B, x);
    if (lb > thr) return lb;
    return fmax(tri_sdf(B, x, nullptr, nullptr), 0.0);
  }
  if (b.kind == 4) {
    double dx = x[0] - b.cx, dy = x[1] - b.cy, dz = x[2] - b.z;
    return fmax(sqrt(dx * dx + dy * dy + dz * dz) - b.r, 0.0);
  }
  double rx = x[0] - b.cx, ry = x[1] - b.cy;
  double rho = sqrt(rx * rx + ry * ry), z = x[2];
  if (b.kind == 1) {
    if (z >= b.z) return fmax(rho - b.r, 0.0);
    if (rho <= b.r) return b.z - z;
    return hypot(rho - b.r, b.z - z);
  }
  if (b.kind == 2) {
    double ta = tan(b.alpha), hc = b.r / ta;
    if (z >= b.z && rho <= fmin((z - b.z) * ta, b.r)) return 0.0;
    double d1 = dist_to_segment(rho, z, 0.0, b.z, b.r, b.z + hc);
    double d2 = (z >= b.z + hc) ? fabs(rho - b.r) : hypot(rho - b.r, b.z + hc - z);
    return fmin(d1, d2);
  }
  return 1e300;
}

// Signed distance (negative inside), outward normal n and Hessian H (row-major)
// of the body surface, for the penalty contact.  Returns true inside.
__device__ inline bool body_sdf(const Body& B, double L, const double* x, double* phi,
                                double* n, double* H) {
  const mpm_rigid& b = B.b;
  if (b.kind == 3) {
    *phi = tri_sdf(B, x, n, H);
    if (*phi < 0.0) return true;
    n[0] = n[1] = n[2] = 0.0;
    for (int i = 0; i < 9; ++i) H[i] = 0.0;
    return false;
  }
  if (b.kind == 4) {
    // sphere: phi = |x - c| - r, n = (x - c) / |x - c|, H = (I - n n^T) / |x - c|
    double d[3] = {x[0] - b.cx, x[1] - b.cy, x[2] - b.z};
    double rho = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int i = 0; i < 9; ++i) H[i] = 0.0;
    n[0] = n[1] = n[2] = 0.0;
    *phi = rho - b.r;
    if (!(*phi < 0.0)) return false;
    if (rho < 1e-12 * L) return true;  // at the centre: no direction is nearest
    for (int i = 0; i < 3; ++i) n[i] = d[i] / rho;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) H[3 * i + j] = ((i == j ? 1.0 : 0.0) - n[i] * n[j]) / rho;
    return true;
  }
  double rx = x[0] - b.cx, ry = x[1] - b.cy;
  double rho = sqrt(rx * rx + ry * ry), z = x[2];
#pragma unroll
  for (int i = 0; i < 9; ++i) H[i] = 0.0;
  n[0] = n[1] = n[2] = 0.0;
  bool axis = rho < 1e-12 * L;
  double ux = axis ? 1.0 : rx / rho, uy = axis ? 0.0 : ry / rho;
  double curv = 0.0;  // curvature factor of the lateral surface
  if (b.kind == 1) {
    if (!(z > b.z && rho < b.r)) {
      *phi = body_distance(B, x, 1e300);
      return false;
    }
    double fb = b.z - z, fs = rho - b.r;
    if (fb >= fs) {
      *phi = fb;
      n[2] = -1.0;
      return true;
    }
    *phi = fs;
    if (axis) return true;  // mean normal of the circle of wall points: zero
    n[0] = ux;
    n[1] = uy;
    curv = 1.0;
  } else if (b.kind == 2) {
    double ta = tan(b.alpha), hc = b.r / ta;
    if (!(z > b.z && rho < fmin((z - b.z) * ta, b.r))) {
      *phi = body_distance(B, x, 1e300);
      return false;
    }
    // nearest boundary point inside: the flank below the rim, the shaft wall
    // above it, except near the axis just above the rim where the flank is
    // nearer (its line's foot, moved along the flank normal, below the rim)
    double ca = cos(b.alpha), sa = sin(b.alpha);
    double pf = rho * ca - (z - b.z) * sa;
    bool flank = z <= b.z + hc || (pf > rho - b.r && (z - b.z) + pf * sa <= hc);
    if (flank) {
      *phi = pf;
      if (axis) {
        // on the axis: mean normal of the circle of closest points, no curvature
        n[2] = -sa;
        return true;
      }
      n[0] = ca * ux;
      n[1] = ca * uy;
      n[2] = -sa;
      curv = ca;
    } else {
      *phi = rho - b.r;
      if (axis) return true;  // mean normal of the circle of wall points: zero
      n[0] = ux;
      n[1] = uy;
      curv = 1.0;
    }
  } else {
    *phi = 1e300;
    return false;
  }
  if (!axis) {
    H[0] = curv * (1.0 - ux * ux) / rho;
    H[1] = -curv * ux * uy / rho;
    H[3] = H[1];
    H[4] = curv * (1.0 - uy * uy) / rho;
  }
  return true;
}

// ------------------------------------------------------------------ warp helpers

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum, result valid in thread 0; blockDim.x a multiple of 32, <= 1024
__device__ inline double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ fixed-order grid sums
//
// Sums over a whole grid without floating-point atomics.  Each block reduces
// its threads' values with the fixed shuffle tree of block_sum and stores the
// result in its own slot; the block that finishes last (elected by an integer
// ticket) adds the slots in block order.  For a given launch shape the result
// is the same bit for bit on every run, whatever order the blocks run in, so
// the Newton path (its residual norms, line search, Krylov scalars) is
// reproducible.  Every block of the grid must reach grid_sum (or none: a
// kernel may return early only where all of its blocks do).
template <int NV>
__device__ inline void grid_sum(const double* v, double* const* out, GridRed g) {
  __shared__ double gsh[32];
  __shared__ int glast;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = block_sum(v[i], gsh);
    if (threadIdx.x == 0) g.part[(size_t)i * gridDim.x + blockIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    glast = atomicAdd(g.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!glast) return;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s += __ldcg(g.part + (size_t)i * gridDim.x + b);
    s = block_sum(s, gsh);
    if (threadIdx.x == 0 && out[i]) *out[i] += s;
  }
  if (threadIdx.x == 0) *g.ticket = 0u;
}

__device__ inline void grid_sum1(double v, double* out, GridRed g) {
  double* o[1] = {out};
  grid_sum<1>(&v, o, g);
}

__device__ inline void grid_sum2(double a, double b, double* oa, double* ob, GridRed g) {
  double v[2] = {a, b};
  double* o[2] = {oa, ob};
  grid_sum<2>(v, o, g);
}

// ------------------------------------------------------------------ event timing

void prof_flush(mpm_ctx* c);

inline cudaEvent_t prof_event(mpm_ctx* c) {
  if (c->evpool.empty()) {
    cudaEvent_t e;
    MPM_CUDA(cudaEventCreate(&e));
    return e;
  }
  cudaEvent_t e = c->evpool.back();
  c->evpool.pop_back();
  return e;
}

// bracket one launch of class `cls` with events on the context stream
inline void prof_begin(mpm_ctx* c, int cls) {
  if (!c->prof_on) return;
  if (c->prof.size() >= 2048) prof_flush(c);
  ProfEv e{cls, prof_event(c), prof_event(c)};
  MPM_CUDA(cudaEventRecord(e.a, c->stream));
  c->prof.push_back(e);
}

inline void prof_end(mpm_ctx* c) {
  if (!c->prof_on || c->prof.empty()) return;
  MPM_CUDA(cudaEventRecord(c->prof.back().b, c->stream));
}

// ------------------------------------------------------------------ host entry helpers

void set_error(mpm_ctx* c, const std::string& m);
int check_device_error(mpm_ctx* c, const char* where);
void sync(mpm_ctx* c);

// the kernels' view of the body for this mesh (mpm_build.cu)
Body body_view(const mpm_mesh* m, const mpm_rigid& b);

// build phase (mpm_build.cu); cand_extra widens the contact candidates' band
// beyond 4 finest cells (a free body's possible motion over a time step)
void build_mesh(mpm_ctx* c, mpm_mesh* m, const mpm_domain& dom, const mpm_rigid& body,
                const mpm_adapt& ad, const mpm_material& mat, mpm_points* pts, int flags,
                double cand_extra = 0.0);

// the rigid body's increment as the contact kernels see it: translation qt
// and rotation qr over the step (the friction's reference displacement at a
// node is qt + qr x d) and the shift of the body from its given pose (qt for
// a free body, whose given pose is the step-start one; zero otherwise)
struct BodyInc {
  double qt[3], qr[3], shift[3];
};

// assembly (mpm_assemble.cu)
struct AsmOut {
  double reaction[3];
  double fint_norm, fextc_norm, finert_norm;
  double Rb[6], Kbb[36];  // a free body's residual and its derivative in q
};
// a time step's inertia and a free body's equations: dt > 0 adds the Newmark
// inertia (needs the build's point velocities); q is the body's increment;
// with `body` the assembly forms the body's residual (AsmOut.Rb, with its
// residual) and, with the tangent, AsmOut.Kbb and the coupling blocks Kgb,
// Kbg (device [6][3 nd] each, when non-null)
struct Dyn {
  double dt = 0.0;
  double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  bool body = false;
  double* Kgb = nullptr;
  double* Kbg = nullptr;
};
// reuse: with K, only the tangent, from the state the last residual-only call
// left at the same increment (dF, tau and the spectral state); R untouched
void assemble(mpm_ctx* c, const mpm_mesh* m, const mpm_material& mat, const mpm_rigid& body,
              const double* du, double load, int precision, double* R, void* K, AsmOut* out,
              bool want_norms, bool reuse = false, const Dyn* dyn = nullptr);
double norm_free(mpm_ctx* c, const mpm_mesh* m, const double* R);
void blocks_export(mpm_ctx* c, const mpm_mesh* m, const void* K, int precision, double* out);

// solve (mpm_solve.cu)
void solve(mpm_ctx* c, const mpm_mesh* m, const mpm_material& mat, const void* K, const double* b,
           double* x, const mpm_solve_params& prm, mpm_solve_stats* st);

// geometric multigrid preconditioner (mpm_mg.cu): structure for the current
// mesh build and Galerkin operators for the stiffness K (T = float or double);
// mg_apply computes z = B r (one V-cycle).  `sk`/`k` let a PCG loop skip the
// work once its residual has converged (slot (k+1) % 3 of rr); with k < 0
// only sk->done is looked at.  rz (device, may be null) receives += r.z.
template <class T>
void mg_setup(mpm_ctx* c, mpm_mesh* m, const T* K, bool reuse);
template <class T>
void mg_apply(mpm_ctx* c, const mpm_mesh* m, const T* K, const T* r, T* z, const Scal* sk, int k,
              double* rz);
void mg_release(mpm_ctx* c, mpm_mesh* m);

// release every buffer of a mesh (mpm_ctx.cu)
void mesh_release(mpm_mesh* m);

// Newton-Raphson of one load step on a built mesh (mpm_step.cu); *du_out is
// the converged increment (context scratch)
void newton(mpm_ctx* c, mpm_mesh* m, const mpm_material* mat, const mpm_rigid& bd,
            const mpm_step_params* prm, mpm_step_stats& st, double** du_out);

// point update (mpm_step.cu)
void point_update(mpm_ctx* c, const mpm_mesh* m, const mpm_material& mat, const double* du,
                  mpm_points* pts, double dt = 0.0);

// CUB wrappers (mpm_cub.cu)
void cub_exclusive_sum_int(mpm_ctx* c, const int* in, int* out, int n);
void cub_sort_u64(mpm_ctx* c, uint64_t* keys, uint64_t* tmp, int n, int end_bit);
void cub_sort_pairs_int(mpm_ctx* c, const int* kin, int* kout, const int* vin, int* vout, int n,
                        int end_bit);
int cub_unique_u64(mpm_ctx* c, const uint64_t* in, uint64_t* out, int n);

}  // namespace mpm
