/*
 * fco3.h -- plain FP64 CPU oracle for the three-dimensional form of the
 * patch method (octree of m x m x m patches; Burstedde, Calhoun, Mandli &
 * Terrel, arXiv:1308.1472, Sec. 1-2: the method is stated for d = 2 and 3,
 * every result of the paper is two-dimensional).
 *
 * TEST INFRASTRUCTURE ONLY.  The slow, obviously-correct reference that the
 * CUDA path is checked against; only the test suite, the smoke check and the
 * CPU-baseline legs may load it.  It shares no code, header, table or helper
 * with the CUDA library and never reads anything the CUDA library produced.
 *
 * Scope: one tree (the unit cube, periodic in x, y and z), scalar advection
 * q_t + u.grad q = 0 with a constant velocity (Sec. 5, Eq. (1) in three
 * dimensions), one global time step for every level or sub-cycling by level
 * (Sec. 4), coarse-fine correction of the coarse cells next to finer
 * patches (Sec. 4), max - min tagging and regrid by family coarsening /
 * refinement + 2:1 balance (Sec. 2, Sec. 5).
 *
 * Readings of what the paper leaves to the wave-propagation literature (the
 * paper gives no three-dimensional scheme):
 *   * waves and fluctuations per face as in two dimensions; MC-limited
 *     second-order corrections per face direction;
 *   * transverse terms: a fluctuation entering a cell is split by the speeds
 *     of the two other directions into that cell's faces of those directions
 *     with coefficient dt / (2 dx);
 *   * double-transverse (corner) terms: each transverse part is split again
 *     by the speed of the third direction, onto the third-direction faces of
 *     the cell it moved into with coefficient -dt^2 / (6 dx^2) and onto those
 *     of the cell it came from with +dt^2 / (6 dx^2), so that with the
 *     limiter off the update equals the tensor-product upwind step
 *     prod_d (1 - nu_d D_d) exactly (pinned in tests);
 *   * ghost cells: same-level copy, 2x2x2 average of finer cells, limited
 *     linear interpolation (minmod slopes in x, y, z, offsets +-1/4) from the
 *     complete tile of a coarser patch; complete tiles are filled level by
 *     level from the coarsest;
 *   * 2:1 balance across faces, edges and corners (26 directions);
 *   * coarse-fine correction: the flux of a coarse face cell is replaced by
 *     the mean of the four fine face fluxes across it (under sub-cycling:
 *     dt times the flux, summed over the fine substeps);
 *   * sub-cycling as in two dimensions: level l takes 2^(l - lmin) substeps
 *     of dt / 2^(l - lmin), coarse levels first; ghost values of another
 *     level are its old and new states blended linearly in time.
 */
#ifndef FCO3_H
#define FCO3_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FCO3_L 20          /* coordinate bits per axis at the finest resolution */

#define FCO3_OK              0
#define FCO3_ERR_ARG        -1
#define FCO3_ERR_UNBALANCED -3
#define FCO3_ERR_CFL        -5

#define FCO3_INIT_BOX    0   /* q = a inside [x0,x1)x[y0,y1)x[z0,z1), b outside: {x0,x1,y0,y1,z0,z1,a,b} */
#define FCO3_INIT_SINE   1   /* q = a + b sin(2 pi (kx x + ky y + kz z)): {a, b, kx, ky, kz}               */
#define FCO3_INIT_GAUSS  2   /* q = a + b exp(-|x - c|^2 / r^2): {a, b, cx, cy, cz, r}                   */

typedef struct {
    int32_t m;            /* cells per patch edge (even, >= 4)                    */
    int32_t min_level, max_level;
    int32_t limiter;      /* 0: none (first order), 1: MC                          */
    int32_t transverse;   /* 0: none, 1: transverse, 2: transverse + corner terms  */
    int32_t refluxing;    /* coarse-fine correction on (1) / off (0)               */
    int32_t subcycle;     /* 0: one global dt; 1: level l takes 2^(l-lmin) substeps */
    double cfl;
    double u, v, w;       /* constant velocity                                     */
    double tag_threshold; /* max - min over a patch                                */
} fco3_params;

typedef struct fco3 fco3;

const char *fco3_last_error(void);
fco3 *fco3_create(const fco3_params *p);
void fco3_destroy(fco3 *s);

/* forest: leaves in Morton order of (x, y, z) with x the lowest bit */
int fco3_num_leaves(const fco3 *s);
int fco3_forest_uniform(fco3 *s, int level);
int fco3_set_leaves(fco3 *s, int n, const int8_t *level, const int32_t *x, const int32_t *y, const int32_t *z);
int fco3_get_leaves(const fco3 *s, int8_t *level, int32_t *x, int32_t *y, int32_t *z);
/* refine (only) until every pair of leaves touching by a face, edge or
   corner differs by at most one level */
int fco3_balance(fco3 *s);
int fco3_is_balanced(const fco3 *s);

/* fields: [leaf][k][j][i], m^3 per leaf */
int fco3_set_fields(fco3 *s, const double *q);
int fco3_get_fields(const fco3 *s, double *q);
int fco3_init(fco3 *s, int kind, const double *prm, int np);
int fco3_init_refine(fco3 *s, int kind, const double *prm, int np);

/* complete (m+4)^3 tile of every leaf ([leaf][k][j][i], index -2..m+1) */
int fco3_fill_tiles(fco3 *s, double *tiles);

int fco3_tag(fco3 *s, int8_t *flags);               /* -1 coarsen, 0 keep, 1 refine */
int fco3_regrid(fco3 *s, const int8_t *flags);
/* nsteps steps of dt (dt <= 0: the CFL step cfl * dx_finest / max |u_d|) */
int fco3_advance(fco3 *s, int nsteps, double dt, double *t_out, double *dt_out);
double fco3_next_dt(const fco3 *s);
double fco3_time(const fco3 *s);
int fco3_sum(const fco3 *s, double *sum);             /* sum of q dx^3 */

#ifdef __cplusplus
}
#endif
#endif
