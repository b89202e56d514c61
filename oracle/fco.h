/*
 * fco.h -- plain FP64 CPU oracle for the forest-of-quadtrees patch method
 * (Burstedde, Calhoun, Mandli & Terrel, "ForestClaw: hybrid forest-of-octrees
 * AMR for hyperbolic conservation laws", arXiv:1308.1472).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the CUDA library, and it never reads
 * anything the CUDA library produced.
 *
 * Everything is FP64 unless a function name says f32.  Loops run one patch at
 * a time, one cell or edge at a time, in the order the method states them.
 *
 * Paper passages followed (section / equation of the paper):
 *   Sec. 2   forest of quadtrees, leaf = patch, 2:1 balance, per-patch flags
 *   Sec. 3   wave propagation on an m x m patch with two ghost layers; ghost
 *            fill by same-level copy, fine-to-coarse averaging and limited
 *            conservative coarse-to-fine interpolation; regrid transfer
 *   Sec. 4   SFC leaf order, global dt vs. per-level dt (sub-cycling),
 *            fine-to-coarse correction after the fine levels
 *   Sec. 5   Eq. (1) scalar advection; max-min tagging and family coarsening
 * The Riemann solver, limiter and transverse terms are delegated by the paper
 * to the wave-propagation literature it cites (LeVeque 1997; Roe 1981); the
 * oracle writes them out from that mathematics.
 *
 * Pins (the test suite's oracle tests) hold it to closed forms, invariants,
 * brute force on small inputs and measured accuracy.  Parity unpinned beyond
 * those invariants: the exact values of the transverse split of the normal
 * fluctuations, the level-by-level order of the ghost fill, the limited
 * coarse-to-fine interpolation and the coarse-fine flux correction have no
 * published numbers; they are held only by what fixes them partly (linear
 * exactness of the ghost fill, the transverse split against the Roe
 * y-Jacobian, conservation to roundoff, the lake at rest, accuracy against
 * exact and uniform-fine solutions).
 */
#ifndef FCO_H
#define FCO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FCO_MAXLEVEL 30     /* coordinate bits per axis at the finest resolution */

/* return codes */
#define FCO_OK              0
#define FCO_ERR_ARG        -1
#define FCO_ERR_CAPACITY   -2
#define FCO_ERR_UNBALANCED -3
#define FCO_ERR_DRY        -4
#define FCO_ERR_CFL        -5
#define FCO_ERR_NONFINITE  -6

/* connectivity */
#define FCO_CONN_SQUARE   0   /* unit square, reflecting walls            */
#define FCO_CONN_PERIODIC 1   /* unit square, doubly periodic             */
#define FCO_CONN_SPHERE   2   /* six-tree cubed sphere (scalar advection) */
#define FCO_CONN_PILLOW   3   /* two-tree sphere, one tree per hemisphere (scalar advection) */
#define FCO_CONN_TABLE    4   /* trees joined by a connectivity table (fco_set_connectivity);
                                 forest only: no fields, no stepping */
#define FCO_MAX_TREES    16   /* trees of a table connectivity (4 tree bits in the leaf key) */

/* equations */
#define FCO_EQ_SWE 0          /* q = (h, hu, hv)                          */
#define FCO_EQ_ADV 1          /* q scalar, q_t + u.grad q = 0 (Eq. 1)     */

/* tagging criteria */
#define FCO_TAG_GRAD   0      /* max undivided centred |grad h|           */
#define FCO_TAG_MAXMIN 1      /* max - min over the patch (Sec. 5)        */

/* neighbour kinds in the neighbour table */
#define FCO_NB_NONE    0      /* domain boundary (or cube corner)         */
#define FCO_NB_SAME    1
#define FCO_NB_COARSER 2
#define FCO_NB_FINER   3

/* initial conditions */
#define FCO_INIT_DAMBREAK 0   /* p = {x0, y0, r2, h_in, h_out}            */
#define FCO_INIT_HUMPS    1   /* p = {base, A_0, w_0, cx_0, cy_0, ...}    */
#define FCO_INIT_ADV_BOX  2   /* p = {x0, x1, y0, y1, q_in, q_out}        */
#define FCO_INIT_ADV_SINE 3   /* p = {a, b, kx, ky}: q = a + b sin(2pi(kx x + ky y)) */
#define FCO_INIT_HILL     4   /* sphere: p = {lon0, lat0, width}          */
#define FCO_INIT_HALF     5   /* sphere: p = {lon, lat}: q = 1 where the point's
                                 dot product with the unit vector of (lon, lat)
                                 is positive, else 0 (Sec. 5, Example 2) */

typedef struct fco_params {
    int32_t conn;
    int32_t m;            /* cells per patch side; even, >= 4           */
    int32_t min_level;
    int32_t max_level;
    int32_t equation;
    int32_t subcycle;     /* 0: one global dt; 1: dt halves per level   */
    int32_t tag_crit;
    int32_t refluxing;    /* coarse-fine flux correction on/off         */
    double  g;            /* gravity (shallow water)                    */
    double  cfl;          /* target Courant number                      */
    double  tag_threshold;
    double  adv_u;        /* constant advection velocity on the square  */
    double  adv_v;
    double  omega_axis_tilt; /* sphere: rotation axis tilt (radians)    */
    double  omega;        /* sphere: angular speed                      */
    int32_t transverse;   /* 0 or 1: the normal fluctuations are split
                             transversely (T1); 2: the limited second-order
                             corrections are split with them (T2, square only) */
    int32_t entropy_fix;  /* 1: Harten-Hyman entropy fix of transonic
                             rarefactions in the shallow-water fluctuations   */
    int32_t velocity;     /* advection on the square: 0 constant (adv_u,
                             adv_v); 1 swirl, stream function
                             adv_u sin^2(pi x) sin^2(pi y) / pi             */
} fco_params;

#define FCO_VEL_CONSTANT 0
#define FCO_VEL_SWIRL    1

typedef struct fco_sim fco_sim;

fco_sim *fco_create(const fco_params *p);
void     fco_destroy(fco_sim *s);
const char *fco_last_error(void);

/* ---- forest (integer) -------------------------------------------------- */
/* Table connectivity (Sec. 2: every tree is a reference square, the trees'
 * connectivity comes from outside): ntrees (1..FCO_MAX_TREES) trees and
 * table[ntrees][4][3], per tree and side (0 -x, 1 +x, 2 -y, 3 +y) the
 * neighbour tree (-1: domain boundary), the neighbour's side facing it and 1
 * if the coordinate along the shared side runs the other way (the table of
 * fco_table_map_point).  Copies the table and resets the forest to uniform
 * min_level over the ntrees trees.  Only for conn = FCO_CONN_TABLE. */
int fco_set_connectivity(fco_sim *s, int ntrees, const int32_t *table);
int fco_forest_uniform(fco_sim *s, int level);
int fco_forest_set_leaves(fco_sim *s, int n, const int32_t *tree, const int32_t *level,
                          const int32_t *x, const int32_t *y);
int fco_num_leaves(const fco_sim *s);
int fco_get_leaves(const fco_sim *s, int32_t *tree, int32_t *level, int32_t *x, int32_t *y);
/* table[n][8][4] = {kind, id0, id1, orient}; directions -x,+x,-y,+y,
 * (-x,-y),(+x,-y),(-x,+y),(+x,+y). */
int fco_get_neighbors(const fco_sim *s, int32_t *table);
int fco_is_balanced(const fco_sim *s);
int fco_balance(fco_sim *s);               /* topology only, fields dropped */
/* Apply flags (-1 coarsen, 0 keep, +1 refine) to the topology only and report
 * the new leaves; fields are not touched.  Used by the integer tests. */
int fco_adapt_topology(fco_sim *s, const int8_t *flags);

/* ---- fields ------------------------------------------------------------ */
int fco_num_fields(const fco_sim *s);
int fco_init_fields(fco_sim *s, int kind, const double *p, int np);
int fco_init_refine(fco_sim *s, int kind, const double *p, int np);
int fco_get_fields(const fco_sim *s, double *out);      /* [n][F][m][m] */
int fco_set_fields(fco_sim *s, const double *in);
int fco_conservation_sums(const fco_sim *s, double *sums);
/* padded ghost-filled arrays of every patch at the current time:
 * out[n][F][m+4][m+4] */
int fco_fill_ghosts(fco_sim *s, double *out);
/* table-driven connectivity: tab[(t * 4 + side) * 3 + {0, 1, 2}] = {neighbour
 * tree or -1, its side facing t, 1 if the along coordinate is reversed};
 * sides 0 -x, 1 +x, 2 -y, 3 +y; finest-level coordinates as fco_map_point's */
int fco_table_map_point(const int32_t *tab, int t, long long X, long long Y, long long *Xo, long long *Yo);

/* test hook for partitioned runs: called before the ghost fill of every
 * (sub)step with the level about to step (-1: every level, global dt), the
 * current state q and, under sub-cycling, the state at the start of each
 * level's current substep qold (q again with a global dt), both
 * [n][F][m][m]; the hook may overwrite both (say, with values received from
 * other ranks).  A non-zero return ends the step with FCO_ERR_ARG.  It adds
 * no arithmetic: a NULL hook leaves every result as it was. */
typedef int (*fco_substep_hook)(void *ctx, int level, double *q, double *qold, int n);
void fco_set_substep_hook(fco_sim *s, fco_substep_hook hook, void *ctx);

/* ---- tagging and regrid ------------------------------------------------ */
int fco_tag(fco_sim *s, int8_t *flags);
int fco_regrid(fco_sim *s, const int8_t *flags);

/* ---- time stepping ----------------------------------------------------- */
/* dt_fixed > 0: use it for every (coarse) step; 0: CFL-driven.
 * t_out, dt_out may be NULL. */
int fco_advance(fco_sim *s, double dt_fixed, int nsteps, double *t_out, double *dt_out);
double fco_time(const fco_sim *s);
double fco_next_dt(const fco_sim *s);
/* largest Courant number seen in the last step */
double fco_last_courant(const fco_sim *s);
/* cell-updates performed so far (one interior cell advanced by one substep) */
int64_t fco_cell_updates(const fco_sim *s);

/* ---- single-patch and 1D kernels used by the pins ---------------------- */
/* Roe solve in x for shallow water: waves[3][3] (wave p, component k), s[3],
 * amdq[3], apdq[3]. */
int fco_roe_x(const double *qL, const double *qR, double g,
              double *waves, double *s, double *amdq, double *apdq);
/* the fluctuations with the Harten-Hyman entropy fix (same waves/speeds) */
int fco_roe_x_efix(const double *qL, const double *qR, double g, double *amdq, double *apdq);
/* transverse split of a fluctuation at an x-edge into y-going parts */
int fco_roe_transverse_x(const double *qL, const double *qR, double g,
                         const double *asdq, double *bmasdq, double *bpasdq);
/* MC limiter phi(theta) */
double fco_mc(double theta);
/* one wave-propagation step on a single padded patch (periodic or prefilled
 * ghosts supplied by the caller): qpad[F][m+4][m+4] in, qout[F][m][m] out.
 * Returns max wave speed in *smax. */
int fco_patch_step(int equation, int m, double g, double dx, double dy, double dt,
                   double adv_u, double adv_v,
                   const double *qpad, double *qout, double *smax);
/* 1D wave propagation (Roe + MC), periodic=0 uses transmissive ends, for the
 * convergence pin against the exact Riemann solution. q[3][n] with hv = 0. */
int fco_swe1d(int n, double dx, double dt, int nsteps, double g, double *h, double *hu);
/* the same with the Harten-Hyman entropy fix on (efix = 1) or off (0) */
int fco_swe1d_efix(int n, double dx, double dt, int nsteps, double g, int efix, double *h, double *hu);
/* exact 1D shallow-water Riemann solution sampled at xi = x/t */
int fco_swe_exact(double hL, double uL, double hR, double uR, double g,
                  int n, const double *xi, double *h, double *u);

/* FP32 twin of the tagging criterion (decisions taken in single precision,
 * the precision of the FP32 kernels): padded h in, 1 if refine. */
int fco_tag_patch_f32(int crit, int m, float threshold, const float *hpad);

/* Cubed-sphere geometry (Fig. 1 right; Sec. 4 coordinate transformations).
 * Doubled centred coordinates: a point of tree t is the cube point
 * N n_t + U a_t + V b_t with N = 2^30 and -N <= U, V <= N.
 * fco_sphere_fold: the tree holding a point beyond tree t's border and its
 *   coordinates there (border points stay in t; -1 beyond a cube corner).
 * fco_sphere_point: the unit-sphere point of (U, V) under the equiangular
 *   gnomonic map.
 * fco_sphere_cell_area: spherical area of the cell [U0, U1] x [V0, V1].
 * fco_sphere_psi: streamfunction of solid-body rotation (angular speed omega
 *   about the axis tilted by omega_axis_tilt from +z toward +x). */
int fco_sphere_fold(int t, long long U, long long V, long long *Uo, long long *Vo);
int fco_sphere_point(int t, long long U, long long V, double p[3]);
double fco_sphere_cell_area(int t, long long U0, long long U1, long long V0, long long V1);
double fco_sphere_psi(const fco_params *pr, const double p[3]);

/* Two-tree sphere geometry (Sec. 5, Example 2), same doubled centred
 * coordinates.  fco_pillow_fold: the tree holding a point beyond tree t's
 * border and its coordinates there (x border: the other tree, x continued;
 * y border: the other tree with a half turn; both: tree t, reflected
 * through the corner).  fco_pillow_point: the unit-sphere point of (U, V)
 * (tree 0 north, tree 1 south with x mirrored; concentric squares to
 * circles of colatitude pi r / 2).  fco_pillow_cell_area: the integral of
 * the map's area element over the cell.  The streamfunction is
 * fco_sphere_psi's. */
int fco_pillow_fold(int t, long long U, long long V, long long *Uo, long long *Vo);
int fco_pillow_point(int t, long long U, long long V, double p[3]);
double fco_pillow_cell_area(int t, long long U0, long long U1, long long V0, long long V1);

/* Learned tagger network (3x3 valid convs 3->16->16->2, ReLU, global max pool).
 * Weights layout: w1[16][3][3][3], b1[16], w2[16][16][3][3], b2[16],
 * w3[2][16][3][3], b3[2] (3058 values in this order). x[N][3][S][S].
 * Forward writes logits[N][2]; backward (given dlogits) writes grads in the
 * same layout and returns the loss when targets are supplied. */
#define FCO_CNN_NPARAM 3058
int fco_cnn_forward(int N, int S, const double *w, const double *x, double *logits);
double fco_cnn_loss_grad(int N, int S, const double *w, const double *x,
                         const double *targets, double *grad);

#ifdef __cplusplus
}
#endif
#endif
