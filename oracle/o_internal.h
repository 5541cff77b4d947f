/* Internal state of the CPU oracle.  TEST INFRASTRUCTURE ONLY (see mpm_oracle.h). */
#ifndef O_INTERNAL_H
#define O_INTERNAL_H
#include "mpm_oracle.h"
#include <stddef.h>

typedef struct {
  int n;
  int *lev;          /* refinement level of each leaf                 */
  int *a;            /* anchors, 3 ints per leaf, finest-grid units    */
  uint64_t *key;     /* Morton key of the anchor                       */
} o_tree;

typedef struct {
  int n;
  int *c;            /* integer coordinates, 3 per node (0..2^D)       */
  uint64_t *key;
  int *corner;       /* 8 node ids per leaf, corner c = cx + 2cy + 4cz */
  int *hang;         /* 1 if hanging (Sec. 3.1 definition)             */
  int *owner;        /* K_n for hanging nodes                          */
  int *cptr, *cidx;  /* resolved constraint lists (independent nodes)  */
  double *cw;
  int *dof;          /* dof index of active independent nodes, else -1 */
  int ndof;
} o_nodes;

struct o_model {
  o_params p;
  int D;             /* finest level = depth_max                      */
  double unit;       /* L / 2^D                                        */
  double scale;      /* 2^D / L                                        */
  /* points */
  int np, cap;
  double *x, *lp, *l0, *F, *be, *V0, *mass, *E, *ys;
  double *v;         /* velocities (dynamic steps), 3 per point        */
  double body_theta[3];
  /* mesh */
  o_tree t;
  o_nodes nd;
  int *nsup, *sidx;  /* support: dof ids after numbering              */
  double *S, *dS;
  int *populated;    /* per leaf                                       */
  double *betaK;     /* per leaf: max E of overlapping points          */
  int *bcmask;       /* per dof: fixed components                      */
  /* block pattern (3x3 blocks) over dofs */
  int nnzb;
  int *row_ptr, *col;
  /* ghost: scalar coefficient per block */
  int nghost;
  int *gface;        /* per ghost face: K, N, axis, sign                */
  double *kg;
  int built;
};

/* o_mesh.c */
uint64_t o_morton(int x, int y, int z);
void o_tree_free(o_tree* t);
int o_locate(const o_tree* t, int x, int y, int z);
int o_build_tree(o_model* m);
int o_build_nodes(o_model* m);
int o_body_sdf(const o_params* p, const double* x, double* phi, double* n, double* H);
/* o_basis.c */
int o_split_points(o_model* m);
int o_build_basis(o_model* m);
int o_build_pattern_and_ghost(o_model* m);
int o_leaf_basis(const o_model* m, int K, const double* xi, int* nent, int* idx, double* phi,
                 double* dphi);
int o_find_slot(const o_model* m, int i, int j);
/* o_material.c */
void o_mat33_mul(const double* a, const double* b, double* c);
double o_det33(const double* a);
void o_inv33(const double* a, double* ai);

#endif
