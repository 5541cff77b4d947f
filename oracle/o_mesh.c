/*
 * Oracle: octree background mesh (Sec. 3.1), adaptive refinement (Sec. 5),
 * rigid-body geometry (Sec. 2.3) and hanging-node constraints (Sec. 3.1).
 * TEST INFRASTRUCTURE ONLY: plain loops, no tuning.
 */
#include "o_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Morton key: bit b of x,y,z goes to bits 3b, 3b+1, 3b+2. */
uint64_t o_morton(int x, int y, int z) {
  uint64_t k = 0;
  for (int b = 0; b < 21; ++b) {
    k |= (uint64_t)((x >> b) & 1) << (3 * b);
    k |= (uint64_t)((y >> b) & 1) << (3 * b + 1);
    k |= (uint64_t)((z >> b) & 1) << (3 * b + 2);
  }
  return k;
}

typedef struct {
  uint64_t key;
  int lev, a[3];
} leafrec;

static int cmp_leafrec(const void* A, const void* B) {
  const leafrec* a = (const leafrec*)A;
  const leafrec* b = (const leafrec*)B;
  return (a->key > b->key) - (a->key < b->key);
}

void o_tree_free(o_tree* t) {
  free(t->lev);
  free(t->a);
  free(t->key);
  memset(t, 0, sizeof(*t));
}

static void tree_from_recs(o_tree* t, leafrec* r, int n) {
  qsort(r, (size_t)n, sizeof(leafrec), cmp_leafrec);
  o_tree_free(t);
  t->n = n;
  t->lev = (int*)malloc(sizeof(int) * (size_t)n);
  t->a = (int*)malloc(sizeof(int) * 3 * (size_t)n);
  t->key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    t->lev[i] = r[i].lev;
    for (int d = 0; d < 3; ++d) t->a[3 * i + d] = r[i].a[d];
    t->key[i] = r[i].key;
  }
}

/* A complete linear octree sorted by anchor key: the leaf that holds finest
 * cell q is the last leaf whose anchor key is <= key(q). */
int o_locate(const o_tree* t, int x, int y, int z) {
  uint64_t k = o_morton(x, y, z);
  int lo = 0, hi = t->n - 1, ans = 0;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (t->key[mid] <= k) {
      ans = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  return ans;
}

static void tree_uniform(o_tree* t, int D, int depth) {
  int nside = 1 << depth, s = 1 << (D - depth);
  int n = nside * nside * nside;
  leafrec* r = (leafrec*)malloc(sizeof(leafrec) * (size_t)n);
  int c = 0;
  for (int k = 0; k < nside; ++k)
    for (int j = 0; j < nside; ++j)
      for (int i = 0; i < nside; ++i) {
        r[c].lev = depth;
        r[c].a[0] = i * s;
        r[c].a[1] = j * s;
        r[c].a[2] = k * s;
        r[c].key = o_morton(r[c].a[0], r[c].a[1], r[c].a[2]);
        ++c;
      }
  tree_from_recs(t, r, n);
  free(r);
}

/* split every marked leaf into its 8 children */
static void tree_refine(o_tree* t, int D, const int* mark) {
  int n = 0;
  for (int i = 0; i < t->n; ++i) n += (mark[i] && t->lev[i] < D) ? 8 : 1;
  leafrec* r = (leafrec*)malloc(sizeof(leafrec) * (size_t)n);
  int c = 0;
  for (int i = 0; i < t->n; ++i) {
    int* a = t->a + 3 * i;
    if (mark[i] && t->lev[i] < D) {
      int h = 1 << (D - t->lev[i] - 1);
      for (int ch = 0; ch < 8; ++ch) {
        r[c].lev = t->lev[i] + 1;
        r[c].a[0] = a[0] + ((ch >> 0) & 1) * h;
        r[c].a[1] = a[1] + ((ch >> 1) & 1) * h;
        r[c].a[2] = a[2] + ((ch >> 2) & 1) * h;
        r[c].key = o_morton(r[c].a[0], r[c].a[1], r[c].a[2]);
        ++c;
      }
    } else {
      r[c].lev = t->lev[i];
      for (int d = 0; d < 3; ++d) r[c].a[d] = a[d];
      r[c].key = t->key[i];
      ++c;
    }
  }
  tree_from_recs(t, r, n);
  free(r);
}

/* Sec. 5: at most one hanging node per edge or face, read as 2:1 balance
 * across faces and edges.  A leaf coarser than its face/edge neighbour by more
 * than one level is refined, until nothing changes. */
static int tree_balance(o_tree* t, int D) {
  int N = 1 << D;
  for (int iter = 0; iter < 4 * D + 8; ++iter) {
    int* mark = (int*)calloc((size_t)t->n, sizeof(int));
    int any = 0;
    for (int K = 0; K < t->n; ++K) {
      int s = 1 << (D - t->lev[K]);
      const int* a = t->a + 3 * K;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int nz = (dx != 0) + (dy != 0) + (dz != 0);
            if (nz == 0 || nz == 3) continue; /* faces and edges only */
            int dd[3] = {dx, dy, dz}, q[3];
            int ok = 1;
            for (int d = 0; d < 3; ++d) {
              q[d] = dd[d] == 1 ? a[d] + s : (dd[d] == -1 ? a[d] - 1 : a[d]);
              if (q[d] < 0 || q[d] >= N) ok = 0;
            }
            if (!ok) continue;
            int nb = o_locate(t, q[0], q[1], q[2]);
            if (t->lev[nb] < t->lev[K] - 1) {
              mark[nb] = 1;
              any = 1;
            }
          }
    }
    if (!any) {
      free(mark);
      return O_OK;
    }
    tree_refine(t, D, mark);
    free(mark);
  }
  return O_ERR_BALANCE;
}

/* ---------------- rigid body geometry (Sec. 2.3; analytic surfaces) ---------------- */

/* ---- closed triangulated body (kind 3) ----
 * The signed distance is taken from the nearest point q of the surface over
 * all triangles (the first triangle attaining the smallest distance); the
 * sign is that of (x - q) . N with N the pseudo-normal of the feature that
 * holds q: the face normal, the sum of the two face normals at an edge, or
 * the angle-weighted sum of the face normals at a vertex (Baerentzen and
 * Aanaes, signed distance by angle-weighted pseudo-normals). */

static void tvert(const o_params* p, int v, double* o) {
  o[0] = p->tri_v[3 * v] + p->body_cx;
  o[1] = p->tri_v[3 * v + 1] + p->body_cy;
  o[2] = p->tri_v[3 * v + 2] + p->body_z;
}

static void sub3(const double* a, const double* b, double* o) {
  for (int d = 0; d < 3; ++d) o[d] = a[d] - b[d];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* unit normal of triangle t */
static void tri_normal(const o_params* p, int t, double* n) {
  double a[3], b[3], c[3], u[3], v[3];
  tvert(p, p->tri_t[3 * t], a);
  tvert(p, p->tri_t[3 * t + 1], b);
  tvert(p, p->tri_t[3 * t + 2], c);
  sub3(b, a, u);
  sub3(c, a, v);
  cross3(u, v, n);
  double l = sqrt(dot3(n, n));
  for (int d = 0; d < 3; ++d) n[d] /= l;
}

/* nearest point q of triangle (a, b, c) to x by the Voronoi regions of its
 * vertices, edges and face; feat: 0 face, 1 edge ab, 2 edge bc, 3 edge ca,
 * 4 vertex a, 5 vertex b, 6 vertex c */
static void tri_nearest(const double* x, const double* a, const double* b, const double* c,
                        double* q, int* feat) {
  double ab[3], ac[3], ax[3], bx[3], cx[3];
  sub3(b, a, ab);
  sub3(c, a, ac);
  sub3(x, a, ax);
  double d1 = dot3(ab, ax), d2 = dot3(ac, ax);
  if (d1 <= 0.0 && d2 <= 0.0) {
    for (int d = 0; d < 3; ++d) q[d] = a[d];
    *feat = 4;
    return;
  }
  sub3(x, b, bx);
  double d3 = dot3(ab, bx), d4 = dot3(ac, bx);
  if (d3 >= 0.0 && d4 <= d3) {
    for (int d = 0; d < 3; ++d) q[d] = b[d];
    *feat = 5;
    return;
  }
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    double v = d1 / (d1 - d3);
    for (int d = 0; d < 3; ++d) q[d] = a[d] + v * ab[d];
    *feat = 1;
    return;
  }
  sub3(x, c, cx);
  double d5 = dot3(ab, cx), d6 = dot3(ac, cx);
  if (d6 >= 0.0 && d5 <= d6) {
    for (int d = 0; d < 3; ++d) q[d] = c[d];
    *feat = 6;
    return;
  }
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    double w = d2 / (d2 - d6);
    for (int d = 0; d < 3; ++d) q[d] = a[d] + w * ac[d];
    *feat = 3;
    return;
  }
  double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
    double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    for (int d = 0; d < 3; ++d) q[d] = b[d] + w * (c[d] - b[d]);
    *feat = 2;
    return;
  }
  double den = 1.0 / (va + vb + vc), v = vb * den, w = vc * den;
  for (int d = 0; d < 3; ++d) q[d] = a[d] + v * ab[d] + w * ac[d];
  *feat = 0;
}

/* pseudo-normal of feature `feat` of triangle t (any length; its sign matters) */
static void tri_pseudo_normal(const o_params* p, int t, int feat, double* N) {
  const int* T = p->tri_t;
  tri_normal(p, t, N);
  if (feat == 0) return;
  if (feat <= 3) {
    int i = T[3 * t + feat - 1], j = T[3 * t + feat % 3];
    for (int u = 0; u < p->ntri; ++u) {
      if (u == t) continue;
      int has_i = 0, has_j = 0;
      for (int k = 0; k < 3; ++k) {
        has_i |= T[3 * u + k] == i;
        has_j |= T[3 * u + k] == j;
      }
      if (has_i && has_j) {
        double n2[3];
        tri_normal(p, u, n2);
        for (int d = 0; d < 3; ++d) N[d] += n2[d];
        return;
      }
    }
    return;
  }
  int v = T[3 * t + feat - 4];
  for (int d = 0; d < 3; ++d) N[d] = 0.0;
  for (int u = 0; u < p->ntri; ++u)
    for (int k = 0; k < 3; ++k) {
      if (T[3 * u + k] != v) continue;
      double a[3], b[3], c[3], e1[3], e2[3], n2[3];
      tvert(p, v, a);
      tvert(p, T[3 * u + (k + 1) % 3], b);
      tvert(p, T[3 * u + (k + 2) % 3], c);
      sub3(b, a, e1);
      sub3(c, a, e2);
      double cs = dot3(e1, e2) / sqrt(dot3(e1, e1) * dot3(e2, e2));
      double ang = acos(cs < -1.0 ? -1.0 : (cs > 1.0 ? 1.0 : cs));
      tri_normal(p, u, n2);
      for (int d = 0; d < 3; ++d) N[d] += ang * n2[d];
    }
}

/* signed distance of the triangulated body at x, with its gradient n and
 * Hessian H (zero on a face; (I - e e^T - u u^T)/phi at an edge of direction
 * e and (I - u u^T)/phi at a vertex, u = (x - q)/|x - q|) */
static double tri_sdf(const o_params* p, const double* x, double* n, double* H) {
  double best = INFINITY, qb[3] = {0, 0, 0};
  int tb = -1, fb = 0;
  for (int t = 0; t < p->ntri; ++t) {
    double a[3], b[3], c[3], q[3];
    int f;
    tvert(p, p->tri_t[3 * t], a);
    tvert(p, p->tri_t[3 * t + 1], b);
    tvert(p, p->tri_t[3 * t + 2], c);
    tri_nearest(x, a, b, c, q, &f);
    double r[3];
    sub3(x, q, r);
    double d2 = dot3(r, r);
    if (d2 < best) {
      best = d2;
      tb = t;
      fb = f;
      for (int d = 0; d < 3; ++d) qb[d] = q[d];
    }
  }
  if (n) n[0] = n[1] = n[2] = 0.0;
  if (H)
    for (int i = 0; i < 9; ++i) H[i] = 0.0;
  if (tb < 0) return INFINITY;
  double dist = sqrt(best), N[3], r[3], nt[3], cr[3];
  sub3(x, qb, r);
  /* x - q along the nearest triangle's normal: q lies on that face's plane
   * (its edge or vertex only bounds it), so the surface is flat there: face */
  tri_normal(p, tb, nt);
  cross3(r, nt, cr);
  if (fb != 0 && dot3(cr, cr) <= 1e-24 * best) fb = 0;
  tri_pseudo_normal(p, tb, fb, N);
  double sg = dot3(r, N) < 0.0 ? -1.0 : 1.0;
  double phi = sg * dist;
  if (!(dist > 0.0)) return 0.0;
  double u[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
  if (n) {
    if (fb == 0) {
      tri_normal(p, tb, n);
    } else {
      for (int d = 0; d < 3; ++d) n[d] = sg * u[d];
    }
  }
  if (H && fb != 0) {
    double e[3] = {0, 0, 0};
    if (fb <= 3) {
      double a[3], b[3];
      tvert(p, p->tri_t[3 * tb + fb - 1], a);
      tvert(p, p->tri_t[3 * tb + fb % 3], b);
      sub3(b, a, e);
      double l = sqrt(dot3(e, e));
      for (int d = 0; d < 3; ++d) e[d] /= l;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        H[3 * i + j] = ((i == j ? 1.0 : 0.0) - e[i] * e[j] - u[i] * u[j]) / phi;
  }
  return phi;
}

static double dist_xy_rect(const o_params* p, const double* lo, const double* hi) {
  double dx = fmax(fmax(lo[0] - p->body_cx, 0.0), p->body_cx - hi[0]);
  double dy = fmax(fmax(lo[1] - p->body_cy, 0.0), p->body_cy - hi[1]);
  return sqrt(dx * dx + dy * dy);
}

/* Step 1 of Sec. 5: does the closed box meet the solid body?  For the
 * triangulated body (reading): when the ball around the box (centre, half
 * diagonal) meets it, i.e. the signed distance at the centre is at most the
 * half diagonal. */
static int body_box_intersect(const o_params* p, const double* lo, const double* hi) {
  if (p->body_kind == 3) {
    double c[3], h2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      c[d] = 0.5 * (lo[d] + hi[d]);
      h2 += 0.25 * (hi[d] - lo[d]) * (hi[d] - lo[d]);
    }
    return tri_sdf(p, c, NULL, NULL) <= sqrt(h2);
  }
  if (p->body_kind == 1) {
    return hi[2] >= p->body_z && dist_xy_rect(p, lo, hi) <= p->body_r;
  }
  if (p->body_kind == 4) {
    /* the closed box meets the ball when its nearest point to the centre does */
    const double c[3] = {p->body_cx, p->body_cy, p->body_z};
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      double e = fmax(fmax(lo[d] - c[d], 0.0), c[d] - hi[d]);
      s += e * e;
    }
    return sqrt(s) <= p->body_r;
  }
  if (p->body_kind == 2) {
    if (hi[2] < p->body_z) return 0;
    double rmax = fmin((hi[2] - p->body_z) * tan(p->body_alpha), p->body_r);
    return dist_xy_rect(p, lo, hi) <= rmax;
  }
  return 0;
}

static double seg_dist(double px, double pz, double ax, double az, double bx, double bz) {
  double vx = bx - ax, vz = bz - az;
  double t = ((px - ax) * vx + (pz - az) * vz) / (vx * vx + vz * vz);
  if (t < 0) t = 0;
  if (t > 1) t = 1;
  double qx = ax + t * vx - px, qz = az + t * vz - pz;
  return sqrt(qx * qx + qz * qz);
}

/* Step 2 of Sec. 5: Euclidean distance from a node to the solid (0 inside) */
static double body_dist(const o_params* p, const double* x) {
  if (p->body_kind == 3) return fmax(tri_sdf(p, x, NULL, NULL), 0.0);
  if (p->body_kind == 4) {
    double dx = x[0] - p->body_cx, dy = x[1] - p->body_cy, dz = x[2] - p->body_z;
    return fmax(sqrt(dx * dx + dy * dy + dz * dz) - p->body_r, 0.0);
  }
  double rx = x[0] - p->body_cx, ry = x[1] - p->body_cy;
  double rho = sqrt(rx * rx + ry * ry), z = x[2];
  if (p->body_kind == 1) {
    if (z >= p->body_z) return fmax(rho - p->body_r, 0.0);
    if (rho <= p->body_r) return p->body_z - z;
    return hypot(rho - p->body_r, p->body_z - z);
  }
  if (p->body_kind == 2) {
    double ta = tan(p->body_alpha), hc = p->body_r / ta;
    if (z >= p->body_z && rho <= fmin((z - p->body_z) * ta, p->body_r)) return 0.0;
    double d1 = seg_dist(rho, z, 0.0, p->body_z, p->body_r, p->body_z + hc);
    double d2;
    if (z >= p->body_z + hc)
      d2 = fabs(rho - p->body_r);
    else
      d2 = hypot(rho - p->body_r, p->body_z + hc - z);
    return fmin(d1, d2);
  }
  return 1e300;
}

/* Signed distance used by the penalty contact (negative inside the body),
 * its gradient n (unit outward normal) and Hessian H. */
int o_body_sdf(const o_params* p, const double* x, double* phi, double* n, double* H) {
  if (p->body_kind == 3) {
    *phi = tri_sdf(p, x, n, H);
    if (*phi < 0.0) return 1;
    for (int i = 0; i < 3; ++i) n[i] = 0.0;
    for (int i = 0; i < 9; ++i) H[i] = 0.0;
    return 0;
  }
  if (p->body_kind == 4) {
    /* sphere: phi = |x - c| - r, n = (x - c) / |x - c|, H = (I - n n^T) / |x - c| */
    double d[3] = {x[0] - p->body_cx, x[1] - p->body_cy, x[2] - p->body_z};
    double rho = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 9; ++i) H[i] = 0.0;
    n[0] = n[1] = n[2] = 0.0;
    *phi = rho - p->body_r;
    if (!(*phi < 0.0)) return 0;
    if (rho < 1e-12 * p->L) return 1; /* at the centre every direction is nearest (reading: n = 0) */
    for (int i = 0; i < 3; ++i) n[i] = d[i] / rho;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) H[3 * i + j] = ((i == j ? 1.0 : 0.0) - n[i] * n[j]) / rho;
    return 1;
  }
  double rx = x[0] - p->body_cx, ry = x[1] - p->body_cy;
  double rho = sqrt(rx * rx + ry * ry), z = x[2];
  for (int i = 0; i < 9; ++i) H[i] = 0.0;
  n[0] = n[1] = n[2] = 0.0;
  double ux = 1.0, uy = 0.0;
  int axis = rho < 1e-12 * p->L;
  if (!axis) {
    ux = rx / rho;
    uy = ry / rho;
  }
  if (p->body_kind == 1) {
    int inside = z > p->body_z && rho < p->body_r;
    if (!inside) {
      *phi = body_dist(p, x);
      return 0;
    }
    double fb = p->body_z - z, fs = rho - p->body_r;
    if (fb >= fs) {
      *phi = fb;
      n[2] = -1.0;
    } else {
      *phi = fs;
      if (axis) return 1; /* the mean normal of the circle of wall points is zero (reading) */
      n[0] = ux;
      n[1] = uy;
      H[0] = (1.0 - ux * ux) / rho;
      H[1] = -ux * uy / rho;
      H[3] = -ux * uy / rho;
      H[4] = (1.0 - uy * uy) / rho;
    }
    return 1;
  }
  if (p->body_kind == 2) {
    double ta = tan(p->body_alpha), hc = p->body_r / ta;
    int inside = z > p->body_z && rho < fmin((z - p->body_z) * ta, p->body_r);
    if (!inside) {
      *phi = body_dist(p, x);
      return 0;
    }
    double ca = cos(p->body_alpha), sa = sin(p->body_alpha), f;
    /* inside, the nearest boundary point is on the flank below the rim, or
     * on the shaft wall above it; just above the rim near the axis the flank
     * is the nearer of the two.  phi_f: signed distance to the flank's line,
     * whose foot (moved along the flank normal) must lie below the rim. */
    double phi_f = rho * ca - (z - p->body_z) * sa;
    double zfoot = (z - p->body_z) + phi_f * sa;
    int flank = z <= p->body_z + hc || (phi_f > rho - p->body_r && zfoot <= hc);
    if (flank) {
      *phi = phi_f;
      if (axis) {
        /* on the axis the closest points form a circle: take the mean of their
         * normals, (0, 0, -sin alpha), and no curvature term (reading) */
        n[2] = -sa;
        return 1;
      }
      n[0] = ca * ux;
      n[1] = ca * uy;
      n[2] = -sa;
      f = ca;
    } else {
      *phi = rho - p->body_r;
      if (axis) return 1; /* the mean normal of the circle of wall points is zero (reading) */
      n[0] = ux;
      n[1] = uy;
      f = 1.0;
    }
    if (!axis) {
      H[0] = f * (1.0 - ux * ux) / rho;
      H[1] = -f * ux * uy / rho;
      H[3] = -f * ux * uy / rho;
      H[4] = f * (1.0 - uy * uy) / rho;
    }
    return 1;
  }
  *phi = 1e300;
  return 0;
}

/* Sec. 5, Steps 1-3 repeated until the cells at the body reach depth_max;
 * each refinement is followed by the 2:1 balance. */
int o_build_tree(o_model* m) {
  const o_params* p = &m->p;
  int D = m->D;
  tree_uniform(&m->t, D, p->depth_min);
  if (p->body_kind == 0 || p->depth_max <= p->depth_min) return O_OK;
  for (int iter = 0; iter < 4 * D + 8; ++iter) {
    o_tree* t = &m->t;
    int* mark = (int*)calloc((size_t)t->n, sizeof(int));
    int any = 0;
    for (int K = 0; K < t->n; ++K) {
      if (t->lev[K] >= p->depth_max) continue;
      int s = 1 << (D - t->lev[K]);
      double lo[3], hi[3];
      for (int d = 0; d < 3; ++d) {
        lo[d] = (double)t->a[3 * K + d] * m->unit;
        hi[d] = (double)(t->a[3 * K + d] + s) * m->unit;
      }
      if (body_box_intersect(p, lo, hi)) {
        mark[K] = 1;
      } else {
        for (int c = 0; c < 8 && !mark[K]; ++c) {
          double xc[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1],
                          (c & 4) ? hi[2] : lo[2]};
          if (body_dist(p, xc) <= p->dx_region) mark[K] = 1;
        }
      }
      any |= mark[K];
    }
    if (!any) {
      free(mark);
      return O_OK;
    }
    tree_refine(&m->t, D, mark);
    free(mark);
    int st = tree_balance(&m->t, D);
    if (st) return st;
  }
  return O_ERR_BALANCE;
}

/* ---------------- nodes, hanging classification, constraints (Sec. 3.1) ---------------- */

typedef struct {
  uint64_t key;
  int c[3];
} noderec;

static int cmp_noderec(const void* A, const void* B) {
  const noderec* a = (const noderec*)A;
  const noderec* b = (const noderec*)B;
  return (a->key > b->key) - (a->key < b->key);
}

static int node_find(const o_nodes* nd, uint64_t k) {
  int lo = 0, hi = nd->n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (nd->key[mid] == k) return mid;
    if (nd->key[mid] < k)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

typedef struct {
  int n;
  int id[O_MAXC];
  double w[O_MAXC];
} clist;

static int clist_add(clist* l, int id, double w) {
  for (int i = 0; i < l->n; ++i)
    if (l->id[i] == id) {
      l->w[i] += w;
      return 0;
    }
  if (l->n >= O_MAXC) return O_ERR_SUPPORT;
  l->id[l->n] = id;
  l->w[l->n] = w;
  l->n++;
  return 0;
}

/* direct constraint of hanging node n: u_n = sum_{i in S(n)} phi_{i,K_n}(x_n) u_i */
static int direct_constraint(const o_model* m, int n, clist* out) {
  const o_tree* t = &m->t;
  const o_nodes* nd = &m->nd;
  int K = nd->owner[n];
  int s = 1 << (m->D - t->lev[K]);
  out->n = 0;
  int twice[3];
  for (int d = 0; d < 3; ++d) {
    twice[d] = 2 * (nd->c[3 * n + d] - t->a[3 * K + d]);
    if (twice[d] != 0 && twice[d] != s && twice[d] != 2 * s) return O_ERR_BALANCE;
  }
  for (int c = 0; c < 8; ++c) {
    double w = 1.0;
    for (int d = 0; d < 3; ++d) {
      double xi = (double)twice[d] / (2.0 * s);
      w *= ((c >> d) & 1) ? xi : 1.0 - xi;
    }
    if (w != 0.0) {
      if (out->n >= O_MAXC) return O_ERR_SUPPORT;
      out->id[out->n] = nd->corner[8 * K + c];
      out->w[out->n] = w;
      out->n++;
    }
  }
  return 0;
}

/* supports that are themselves hanging are substituted until only
 * independent nodes remain (chains resolved transitively) */
static int resolve(const o_model* m, int n, double w, int depth, clist* out) {
  if (!m->nd.hang[n]) return clist_add(out, n, w);
  if (depth > 64) return O_ERR_BALANCE;
  clist dir;
  int st = direct_constraint(m, n, &dir);
  if (st) return st;
  for (int i = 0; i < dir.n; ++i) {
    st = resolve(m, dir.id[i], w * dir.w[i], depth + 1, out);
    if (st) return st;
  }
  return 0;
}

static void nodes_free(o_nodes* nd) {
  free(nd->c);
  free(nd->key);
  free(nd->corner);
  free(nd->hang);
  free(nd->owner);
  free(nd->cptr);
  free(nd->cidx);
  free(nd->cw);
  free(nd->dof);
  memset(nd, 0, sizeof(*nd));
}

int o_build_nodes(o_model* m) {
  const o_tree* t = &m->t;
  o_nodes* nd = &m->nd;
  int D = m->D, N = 1 << D;
  nodes_free(nd);
  int n8 = 8 * t->n;
  noderec* r = (noderec*)malloc(sizeof(noderec) * (size_t)n8);
  for (int K = 0; K < t->n; ++K) {
    int s = 1 << (D - t->lev[K]);
    for (int c = 0; c < 8; ++c) {
      noderec* q = r + 8 * K + c;
      for (int d = 0; d < 3; ++d) q->c[d] = t->a[3 * K + d] + ((c >> d) & 1) * s;
      q->key = o_morton(q->c[0], q->c[1], q->c[2]);
    }
  }
  qsort(r, (size_t)n8, sizeof(noderec), cmp_noderec);
  int nu = 0;
  for (int i = 0; i < n8; ++i)
    if (i == 0 || r[i].key != r[i - 1].key) r[nu++] = r[i];
  nd->n = nu;
  nd->c = (int*)malloc(sizeof(int) * 3 * (size_t)nu);
  nd->key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nu);
  for (int i = 0; i < nu; ++i) {
    nd->key[i] = r[i].key;
    for (int d = 0; d < 3; ++d) nd->c[3 * i + d] = r[i].c[d];
  }
  free(r);
  nd->corner = (int*)malloc(sizeof(int) * (size_t)n8);
  for (int K = 0; K < t->n; ++K) {
    int s = 1 << (D - t->lev[K]);
    for (int c = 0; c < 8; ++c) {
      int q[3];
      for (int d = 0; d < 3; ++d) q[d] = t->a[3 * K + d] + ((c >> d) & 1) * s;
      nd->corner[8 * K + c] = node_find(nd, o_morton(q[0], q[1], q[2]));
    }
  }
  /* Eq. (hanging node): n hangs if it lies on the boundary of a leaf K without
   * being one of K's vertices.  Such K hold one of the 8 finest cells around
   * x_n; the owner K_n is the largest of them (ties: lowest Morton key). */
  nd->hang = (int*)calloc((size_t)nu, sizeof(int));
  nd->owner = (int*)malloc(sizeof(int) * (size_t)nu);
  for (int n = 0; n < nu; ++n) {
    int best = -1;
    const int* X = nd->c + 3 * n;
    for (int sc = 0; sc < 8; ++sc) {
      int q[3], ok = 1;
      for (int d = 0; d < 3; ++d) {
        q[d] = X[d] - 1 + ((sc >> d) & 1);
        if (q[d] < 0 || q[d] >= N) ok = 0;
      }
      if (!ok) continue;
      int K = o_locate(t, q[0], q[1], q[2]);
      int s = 1 << (D - t->lev[K]);
      int corner = 1;
      for (int d = 0; d < 3; ++d) {
        int r0 = X[d] - t->a[3 * K + d];
        if (r0 != 0 && r0 != s) corner = 0;
      }
      if (corner) continue;
      if (best < 0 || t->lev[K] < t->lev[best] ||
          (t->lev[K] == t->lev[best] && t->key[K] < t->key[best]))
        best = K;
    }
    nd->hang[n] = best >= 0;
    nd->owner[n] = best;
  }
  /* Eq. (constraint equation reduced), resolved transitively */
  nd->cptr = (int*)malloc(sizeof(int) * (size_t)(nu + 1));
  clist* all = (clist*)malloc(sizeof(clist) * (size_t)nu);
  int tot = 0;
  for (int n = 0; n < nu; ++n) {
    all[n].n = 0;
    int st = resolve(m, n, 1.0, 0, &all[n]);
    if (st) {
      free(all);
      return st;
    }
    /* sort by node id */
    for (int i = 1; i < all[n].n; ++i)
      for (int j = i; j > 0 && all[n].id[j - 1] > all[n].id[j]; --j) {
        int ti = all[n].id[j];
        all[n].id[j] = all[n].id[j - 1];
        all[n].id[j - 1] = ti;
        double tw = all[n].w[j];
        all[n].w[j] = all[n].w[j - 1];
        all[n].w[j - 1] = tw;
      }
    nd->cptr[n] = tot;
    tot += all[n].n;
  }
  nd->cptr[nu] = tot;
  nd->cidx = (int*)malloc(sizeof(int) * (size_t)(tot > 0 ? tot : 1));
  nd->cw = (double*)malloc(sizeof(double) * (size_t)(tot > 0 ? tot : 1));
  for (int n = 0; n < nu; ++n)
    for (int i = 0; i < all[n].n; ++i) {
      nd->cidx[nd->cptr[n] + i] = all[n].id[i];
      nd->cw[nd->cptr[n] + i] = all[n].w[i];
    }
  free(all);
  nd->dof = (int*)malloc(sizeof(int) * (size_t)nu);
  for (int n = 0; n < nu; ++n) nd->dof[n] = -1;
  nd->ndof = 0;
  return O_OK;
}

void o_nodes_release(o_nodes* nd) { nodes_free(nd); }
