/*
 * fc3.h -- C ABI of the three-dimensional patch solver: an octree of
 * m x m x m patches on the periodic unit cube, scalar advection
 * q_t + u.grad q = 0 with a constant velocity (Burstedde, Calhoun, Mandli &
 * Terrel, arXiv:1308.1472: the method of Sec. 2-4 for d = 3, Eq. (1) of
 * Sec. 5 in three dimensions).
 *
 * Every call returns FC_OK (0) or a negative FC_ERR_* code of fc.h;
 * fc_last_error() gives a thread-local message.  No exception crosses the
 * ABI.  The library owns all device memory; the caller owns every host
 * buffer it passes.  Arrays of leaves are in Morton order of (x, y, z)
 * with x in the lowest bit.
 *
 * The method per step (one global dt for every level, or sub-cycled):
 *   ghost cells (two layers): same-level copy, mean of the 2x2x2 finer
 *     cells, or limited linear interpolation (minmod slopes in x, y, z,
 *     offsets +-1/4) from the complete tile of a coarser patch (Sec. 3);
 *   per face: wave, fluctuations and the MC-limited second-order
 *     correction; each fluctuation entering a cell is split by the two
 *     perpendicular speeds into that cell's faces of those directions
 *     (coefficient dt / (2 dx)) and again by the third speed (corner terms,
 *     -dt^2 / (6 dx^2) on the cell the part moved into, +dt^2 / (6 dx^2) on
 *     the cell it left), so that with the limiter off the step is the
 *     tensor-product upwind step (the paper gives no 3D scheme: this is the
 *     reading taken);
 *   conservative update, then the coarse-fine correction (Sec. 4): a coarse
 *     face cell next to finer patches takes the mean of the four fine face
 *     fluxes in place of its own (dt times the flux, summed over the fine
 *     substeps under sub-cycling).
 */
#ifndef FC3_H
#define FC3_H
#include <stdint.h>

#include "fc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FC3_INIT_BOX   0   /* q = a inside [x0,x1)x[y0,y1)x[z0,z1), b outside: {x0,x1,y0,y1,z0,z1,a,b} */
#define FC3_INIT_SINE  1   /* q = a + b sin(2 pi (kx x + ky y + kz z)): {a, b, kx, ky, kz}               */
#define FC3_INIT_GAUSS 2   /* q = a + b exp(-|x - c|^2 / r^2): {a, b, cx, cy, cz, r}                   */

typedef struct {
    int32_t m;            /* cells per patch edge: 4 or 8                          */
    int32_t min_level;    /* 0 .. max_level                                        */
    int32_t max_level;    /* <= 10                                                 */
    int32_t precision;    /* FC_FP64 or FC_FP32                                    */
    int32_t limiter;      /* 0: none (first order), 1: MC                          */
    int32_t transverse;   /* 0: none, 1: transverse, 2: transverse + corner terms  */
    int32_t refluxing;    /* coarse-fine correction on (1) / off (0)               */
    int32_t subcycle;     /* 0: one global dt; 1: level l takes 2^(l-lmin) substeps
                             of dt / 2^(l-lmin) (Sec. 4), other levels' ghost values
                             blended linearly in time                               */
    int32_t device;       /* CUDA device ordinal, -1: current                      */
    double cfl;           /* (0, 1]: dt = cfl * dx_finest / max |u_d|              */
    double u, v, w;       /* constant velocity                                     */
    double tag_threshold; /* max - min over a patch (Sec. 5)                       */
    void *stream;         /* cudaStream_t to run on, or NULL for the library's own */
} fc3_params;

typedef struct fc3_ctx fc3_ctx;

/* Context with a uniform forest at min_level and q = 0.  Errors:
   INVALID_ARG for a parameter out of range, CUDA. */
int fc3_create(const fc3_params *p, fc3_ctx **out);
void fc3_destroy(fc3_ctx *ctx);

/* Forest.  fc3_forest_uniform: every leaf at `level` (fields set to 0).
   fc3_forest_set_leaves: n leaves (host arrays, caller-owned) that must
   tile the cube in Morton order and be 2:1 balanced across faces, edges and
   corners (UNBALANCED otherwise; INVALID_ARG for out-of-range, unsorted or
   overlapping leaves); fields set to 0.  fc3_forest_get_leaves copies at
   most cap leaves (CAPACITY if n > cap). */
int fc3_forest_uniform(fc3_ctx *ctx, int level);
int fc3_forest_set_leaves(fc3_ctx *ctx, int64_t n, const int8_t *level, const int32_t *x, const int32_t *y,
                          const int32_t *z);
int fc3_forest_num_leaves(const fc3_ctx *ctx, int64_t *n);
int fc3_forest_get_leaves(const fc3_ctx *ctx, int8_t *level, int32_t *x, int32_t *y, int32_t *z, int64_t cap);

/* Fields, host buffers of n * m^3 values of the context's precision
   (float or double), layout [leaf][k][j][i].  count is the buffer length
   in values (CAPACITY if too small). */
int fc3_write_fields(fc3_ctx *ctx, const void *src, int64_t count);
int fc3_read_fields(fc3_ctx *ctx, void *dst, int64_t count);
/* point samples at cell centres of an FC3_INIT_* field (np parameters) */
int fc3_set_initial(fc3_ctx *ctx, int kind, const double *prm, int np);
/* uniform at min_level, then (max_level - min_level) rounds of {initial
   field, tag, refine the tagged leaves, balance}, then the initial field */
int fc3_init_refine(fc3_ctx *ctx, int kind, const double *prm, int np);

/* Tagging (Sec. 5): flags[n] (caller-owned): 1 refine (max - min of the
   patch above the threshold and level < max_level), -1 coarsen (a family of
   eight sibling leaves above min_level whose averaged parent is at or below
   the threshold, and no sibling above it), 0 keep. */
int fc3_tag(fc3_ctx *ctx, int8_t *flags);
/* Regrid by flags[n]: refinement wins, a family coarsens when all eight are
   flagged -1, then 2:1 balance; new leaves take the old values (copy,
   limited linear interpolation from the parent, mean of the children). */
int fc3_regrid(fc3_ctx *ctx, const int8_t *flags);

/* nsteps (coarse) steps of dt (dt <= 0: cfl * dx / max |u_d|, dx of the
   finest level, or of the coarsest under sub-cycling); CFL_VIOLATION if dt
   gives a Courant number above 1.  t_out, dt_out may be NULL. */
int fc3_advance(fc3_ctx *ctx, int nsteps, double dt, double *t_out, double *dt_out);
/* sum over cells of q dx^3, FP64 (per-patch sums, then a compensated sum
   over the patches) */
int fc3_conservation_sum(fc3_ctx *ctx, double *sum);
/* time, next CFL step and interior cell-updates since creation */
int fc3_stats(fc3_ctx *ctx, double *time, double *next_dt, double *cell_updates);
/* wait for the context's stream */
int fc3_sync(fc3_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
