/* fco_internal.h -- oracle internals (TEST INFRASTRUCTURE; see fco.h). */
#ifndef FCO_INTERNAL_H
#define FCO_INTERNAL_H
#include "fco.h"
#include <stddef.h>

typedef struct { int32_t tree, level, x, y; } fco_leaf;

struct fco_sim {
    fco_params p;
    int F;                 /* fields per cell                             */
    int n;                 /* leaves                                      */
    fco_leaf *leaves;      /* SFC order                                   */
    int tree_first[FCO_MAX_TREES + 1];  /* first leaf of each tree, [ntrees] = n */
    int ntab;              /* trees of a table connectivity                */
    int32_t *table;        /* [ntab][4][3] (FCO_CONN_TABLE), else NULL     */
    double *q;             /* [n][F][m][m] current state                  */
    double t;
    double dt_next;        /* 0 until known                               */
    int    dt_from_cells;  /* next CFL dt comes from cell speeds (R10)    */
    double last_courant;
    int64_t cell_updates;
    fco_substep_hook hook; /* test hook before each (sub)step's ghost fill */
    void  *hook_ctx;
};

/* forest */
uint64_t fco_morton(uint32_t X, uint32_t Y);
uint64_t fco_leaf_key(const fco_leaf *l);
void fco_sort_leaves(fco_leaf *l, int n);
int  fco_num_trees(int conn);
int  fco_map_point(int conn, int t, long long X, long long Y, long long *Xo, long long *Yo);
int  fco_orientation(int conn, int t, long long X, long long Y);
/* the simulation's connectivity (built-in or its table) */
int  fco_sim_num_trees(const fco_sim *s);
int  fco_sim_map_point(const fco_sim *s, int t, long long X, long long Y, long long *Xo, long long *Yo);
int  fco_sim_orientation(const fco_sim *s, int t, long long X, long long Y);
int  fco_find_leaf(const fco_sim *s, int t, long long X, long long Y);
void fco_index_trees(fco_sim *s);
int  fco_build_neighbors(fco_sim *s, int32_t *tab);
int  fco_balance_topology(fco_sim *s);
void fco_set_topology(fco_sim *s, fco_leaf *leaves, int n);
int  fco_forest_uniform_topology(fco_sim *s, int level);
int  fco_forest_set_leaves_topology(fco_sim *s, int n, const int32_t *tree, const int32_t *level,
                                    const int32_t *x, const int32_t *y);
int  fco_adapt(fco_sim *s, const int8_t *flags, int32_t **origin_out);

/* numerics: one Riemann problem at an edge, in the edge's normal direction.
 * dir 0: x-edge (normal momentum hu), dir 1: y-edge (normal momentum hv). */
typedef struct {
    int    nw;             /* number of waves                             */
    double W[3][3];        /* W[p][k]                                     */
    double s[3];
    double amdq[3], apdq[3];
    double un, ut, c;      /* Roe averages: normal, transverse velocity, celerity */
} fco_edge;

void fco_riemann_swe(int dir, const double *qL, const double *qR, double g, fco_edge *e);
/* replace the fluctuations of a shallow-water edge by the Harten-Hyman
 * entropy-fixed ones (qL, qR: the edge's states) */
void fco_entropy_fix_swe(int dir, const double *qL, const double *qR, double g, fco_edge *e);
void fco_riemann_adv(double vel, const double *qL, const double *qR, fco_edge *e);
/* split a fluctuation at an edge into the two transverse directions */
void fco_transverse_swe(int dir, const fco_edge *e, const double *asdq, double *bm, double *bp);
double fco_mc_limiter(double theta);

/* analytic flux of the state in direction dir (shallow water) */
void fco_flux_swe(int dir, const double *q, double g, double *f);

#define FCO_PAD(m) ((m) + 4)
#define FCO_IDX(m, i, j) (((j) + 2) * FCO_PAD(m) + ((i) + 2))

#endif
