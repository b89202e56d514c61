/*
 * fc.h -- C ABI of the GB300 forest-of-quadtrees patch library (libfc.so).
 *
 * Method: Burstedde, Calhoun, Mandli & Terrel, "ForestClaw: hybrid
 * forest-of-octrees AMR for hyperbolic conservation laws" (arXiv:1308.1472).
 * Every leaf of a 2:1-balanced forest of quadtrees carries one m x m
 * finite-volume patch (Sec. 2); patches are advanced by the second-order wave
 * propagation method with two ghost layers filled by same-level copy,
 * fine-to-coarse averaging and limited coarse-to-fine interpolation (Sec. 3);
 * time stepping uses one global dt or per-level dt with coarse-fine correction
 * (Sec. 4); tagging is per patch (Sec. 5).
 *
 * Conventions for every entry point:
 *  - return 0 on success or a negative FC_ERR_* code; fc_last_error() gives a
 *    message for the calling thread; no C++ exception crosses this boundary;
 *  - the library owns all device memory of a context (allocated on the
 *    context's device and stream); caller buffers are owned by the caller and
 *    are only read or written during the call;
 *  - arrays of leaves are in space-filling-curve order: (tree, Morton key of
 *    the leaf's lower-left corner at 30 bits per axis, x in the lower bit);
 *  - fields are stored structure-of-arrays, [field][leaf][j][i] inside the
 *    library; the read/write calls use [leaf][field][j][i] (i fastest);
 *  - floating-point buffers use the context precision (double for FC_FP64,
 *    float for FC_FP32) unless the name says otherwise.
 * All GPU work of a context is issued on the stream given in fc_params (NULL:
 * a non-blocking stream the context creates); calls return after that work
 * completed unless stated otherwise.
 */
#ifndef FC_H
#define FC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define FC_OK                  0
#define FC_ERR_INVALID_ARG    -1   /* bad argument or parameter            */
#define FC_ERR_CAPACITY       -2   /* caller buffer too small              */
#define FC_ERR_UNBALANCED     -3   /* forest violates 2:1 balance          */
#define FC_ERR_DRY_STATE      -4   /* depth h <= 0 met by the solver       */
#define FC_ERR_CFL_VIOLATION  -5   /* Courant number > 1 after 3 retries   */
#define FC_ERR_NONFINITE      -6   /* NaN or Inf in the state              */
#define FC_ERR_TIMEOUT        -7   /* a bounded device wait gave up (the
                                       * tensor-core forward of fc_cnn_forward) */
#define FC_ERR_CUDA           -8   /* CUDA runtime error                   */
#define FC_ERR_UNIMPLEMENTED  -9   /* feature not available                */

/* ---- enumerations ------------------------------------------------------ */
#define FC_CONN_SQUARE    0   /* unit square, one tree, reflecting walls   */
#define FC_CONN_PERIODIC  1   /* unit square, one tree, periodic           */
#define FC_CONN_SPHERE    2   /* six trees on the cube faces               */
#define FC_CONN_PILLOW    3   /* two trees, one per hemisphere (Sec. 5, Example 2):
                                 tree 0 north, tree 1 south with x mirrored; the
                                 two trees side by side form a strip periodic in
                                 x, y borders meet with a half turn; a point at
                                 (x, y) in [-1,1]^2 lies at colatitude
                                 (pi/2) max(|x|, |y|) from its tree's pole */
#define FC_CONN_TABLE     4   /* trees joined by a connectivity table given
                                 with fc_set_connectivity (forest only) */
#define FC_MAX_TREES     16   /* trees of a table connectivity */

#define FC_EQ_SWE 0           /* shallow water, q = (h, hu, hv), Roe solver */
#define FC_EQ_ADV 1           /* scalar advection, Sec. 5 Eq. (1)          */

#define FC_FP64 0
#define FC_FP32 1

#define FC_TAG_GRAD   0       /* max centred undivided |grad q0| > thr     */
#define FC_TAG_MAXMIN 1       /* max - min of q0 over the patch > thr (Sec. 5) */

#define FC_TAGGER_PLAIN   0
#define FC_TAGGER_LEARNED 1

#define FC_INIT_DAMBREAK 0    /* p = {x0, y0, r2, h_in, h_out}             */
#define FC_INIT_HUMPS    1    /* p = {base, (A, w, cx, cy) per hump}       */
#define FC_INIT_ADV_BOX  2    /* p = {x0, x1, y0, y1, q_in, q_out}         */
#define FC_INIT_ADV_SINE 3    /* p = {a, b, kx, ky}: a + b sin(2pi(kx x + ky y)) */
#define FC_INIT_HILL     4    /* sphere: p = {lon0, lat0, width}:
                                 exp(-(d / width)^2), d = great-circle distance
                                 of the mapped cell centre to (lon0, lat0) */
#define FC_INIT_HALF     5    /* sphere: p = {lon, lat}: 1 where the mapped cell
                                 centre lies in the half facing (lon, lat),
                                 else 0 (Sec. 5, Example 2) */

#define FC_NB_NONE    0
#define FC_NB_SAME    1
#define FC_NB_COARSER 2
#define FC_NB_FINER   3

typedef struct fc_params {
    int32_t conn;           /* FC_CONN_*                                   */
    int32_t m;              /* cells per patch side: 8, 16 or 32           */
    int32_t min_level;      /* coarsest level allowed (>= 0)               */
    int32_t max_level;      /* finest level allowed (<= 14)                */
    int32_t equation;       /* FC_EQ_*                                     */
    int32_t precision;      /* FC_FP64 or FC_FP32 patch arithmetic         */
    int32_t subcycle;       /* 0: one global dt; 1: dt halves per level    */
    int32_t tag_crit;       /* FC_TAG_*                                    */
    int32_t refluxing;      /* coarse-fine flux correction on (1) / off (0) */
    int32_t device;         /* CUDA device ordinal, -1 = current device    */
    double  g;              /* gravity                                     */
    double  cfl;            /* target Courant number, e.g. 0.9             */
    double  tag_threshold;
    double  adv_u, adv_v;   /* constant advection velocity (square)        */
    void   *stream;         /* cudaStream_t to issue work on, may be NULL  */
    double  omega;          /* spheres: angular speed of the rotation      */
    double  omega_axis_tilt;/* spheres: rotation axis tilted from +z
                               toward +x by this angle (radians)            */
    int32_t transverse;     /* 0 or 1: the normal fluctuations are split
                               transversely (T1, the default); 2: the
                               limited second-order corrections are split
                               with them (T2: A-dQ + cq and A+dQ - cq, cq the
                               edge's summed limited correction; LeVeque 1997;
                               square and periodic square only)             */
    int32_t entropy_fix;    /* 1: Harten-Hyman entropy fix of transonic 1-
                               and 3-waves in the shallow-water fluctuations
                               (a transonic wave is split between its end
                               speeds); 0: none.  With T2 or the fix only
                               launch variants 0 and 1 are available.       */
    int32_t velocity;       /* advection on the square: FC_VEL_CONSTANT
                               (adv_u, adv_v) or FC_VEL_SWIRL, the
                               divergence-free swirl with stream function
                               adv_u sin^2(pi x) sin^2(pi y) / pi (the paper's
                               Example 1 flow, which it does not give; edge
                               speeds are stream-function differences over
                               the edge length); swirl: launch variants 0, 1 */
} fc_params;

#define FC_VEL_CONSTANT 0
#define FC_VEL_SWIRL    1

typedef struct fc_stats_t {
    int64_t num_leaves;
    int64_t leaves_per_level[16];
    int64_t cell_updates;       /* interior cells advanced by one (sub)step */
    int64_t steps;              /* accepted (coarse) steps                  */
    int64_t retries;            /* steps retaken after a Courant number > 1 */
    int64_t regrids;
    double  time;
    double  last_dt;
    double  last_courant;
    double  next_dt;
} fc_stats_t;

typedef struct fc_ctx fc_ctx;

/* ---- context -----------------------------------------------------------
 * fc_create: validate params, bind the device, create a forest of uniform
 * level min_level with zero fields.  *out receives an opaque context that the
 * caller releases with fc_destroy.  Sec. 2 (forest of quadtrees, leaf =
 * patch of m x m cells). */
int  fc_create(const fc_params *params, fc_ctx **out);
void fc_destroy(fc_ctx *ctx);
const char *fc_last_error(void);

/* ---- forest (integer work, bit-exact) ----------------------------------
 * Sec. 2 and Sec. 4: forest of quadtrees in space-filling-curve order.
 * fc_forest_uniform: every tree refined uniformly to `level`; fields zeroed.
 * fc_forest_set_leaves: replace the forest by n caller leaves (host arrays,
 *   any order; they must tile the domain); fields zeroed.
 * fc_forest_num_leaves / fc_forest_get_leaves: host copies of the leaves in
 *   SFC order; cap = capacity of each array (FC_ERR_CAPACITY if < n).
 * fc_forest_get_neighbors: host copy of the neighbour table, int32
 *   [n][8][4] = {kind, id0, id1, orient}; directions -x, +x, -y, +y, then
 *   corners (-x,-y), (+x,-y), (-x,+y), (+x,+y).  kind FC_NB_*; for a finer
 *   face neighbour id0/id1 are the two leaves in increasing coordinate along
 *   the face, otherwise id1 = -1; orient = 0 inside a tree.  cap counts int32.
 *   Cubed sphere (Fig. 1 right, Sec. 4): tree t lies on the cube face with
 *   outward normal n_t and axes a_t (x), b_t (y), a_t x b_t = n_t, trees
 *   0..5 = +x, +y, -x, -y, +z, -z with (a, b) = (+y, +z), (-x, +z), (-y, +z),
 *   (+x, +z), (+y, -x), (+y, +x).  Across a tree border orient encodes the
 *   map of index offsets into the neighbour's tree as 1 + 4 swap + 2 (image
 *   of +x negative) + (image of +y negative); corners where three trees meet
 *   have kind FC_NB_NONE in the diagonal direction.
 *   Two-tree sphere (Sec. 5, Example 2): across an x border the other tree
 *   with x continued (orient 0 is not used there: the code of the identity
 *   map is 1); across a y border the other tree with a half turn; beyond
 *   both borders at a tree corner the patch's own corner reflected through
 *   the corner point (the corners are points of the equator where two cells
 *   meet), so a corner leaf is its own diagonal neighbour.
 * fc_forest_balance: refine until face and corner neighbours differ by at most
 *   one level (Sec. 2, 2:1 balance); fields zeroed. */
int fc_forest_uniform(fc_ctx *ctx, int level);
/* fc_set_connectivity (ctx created with conn = FC_CONN_TABLE): the trees and
 *   their connectivity from outside (Sec. 2: every tree is a reference square,
 *   the forest's connectivity may come from a mesh generator).  table: host
 *   int32 [ntrees][4][3], 1 <= ntrees <= FC_MAX_TREES; per tree and side (0 -x,
 *   1 +x, 2 -y, 3 +y) the neighbour tree (-1: domain boundary), the
 *   neighbour's side facing this tree and 1 if the coordinate along the
 *   shared side runs the other way, 0 if not.  A point beyond one side is
 *   carried across it (depth beyond the side = depth inside the neighbour); a
 *   point beyond two sides is carried across both in either order, and if
 *   the two orders disagree (three trees meet at the corner) it has no image.
 *   The table is copied to the device; the forest becomes uniform at
 *   min_level over the ntrees trees.  On such a context the forest calls work
 *   (uniform, set_leaves, balance, leaves, neighbour table with the
 *   orientation code of every crossing of a tree side: 1 + 4 swap + 2 (image
 *   of +x negative) + (image of +y negative), the identity being 1); the calls
 *   that need fields (initial data, writes, stepping, tagging, regridding,
 *   tiles) return FC_ERR_UNIMPLEMENTED.  FC_ERR_INVALID_ARG for a bad table
 *   (an entry naming a tree, side or flag out of range). */
int fc_set_connectivity(fc_ctx *ctx, int ntrees, const int32_t *table);
int fc_forest_set_leaves(fc_ctx *ctx, int64_t n, const int32_t *tree, const int32_t *level,
                         const int32_t *x, const int32_t *y);
int fc_forest_num_leaves(const fc_ctx *ctx, int64_t *n);
int fc_forest_get_leaves(const fc_ctx *ctx, int32_t *tree, int32_t *level, int32_t *x, int32_t *y,
                         int64_t cap);
int fc_forest_get_neighbors(const fc_ctx *ctx, int32_t *table, int64_t cap);
int fc_forest_balance(fc_ctx *ctx);

/* ---- fields -------------------------------------------------------------
 * fc_set_initial: point samples of an initial condition (FC_INIT_*, np
 *   parameters, host array) at every cell centre of the current forest.
 * fc_init_refine: uniform forest at min_level, then (max_level - min_level)
 *   rounds of {initialise, tag, refine flagged leaves, balance}, then a final
 *   initialisation (Sec. 5 tagging drives the refinement).
 * fc_read_fields: copy the state to dst, [leaf][field][j][i] in the context
 *   precision; dst is device memory if dst_is_device, else host memory;
 *   cap_bytes = size of dst.  field = -1 copies all fields, otherwise one
 *   field ([leaf][j][i]).  Host buffers go through a device staging buffer
 *   (the layout kernel in device memory, the copy engines over the host link;
 *   page-locked buffers -- cudaHostAlloc, cudaHostRegister, a pinned torch
 *   tensor -- at the link's rate).
 * fc_write_fields: the inverse of fc_read_fields for all fields.
 * fc_conservation_sums: sums[f] = sum over cells of (cell area) * q_f, FP64,
 *   deterministic order (host array of F doubles). */
int fc_set_initial(fc_ctx *ctx, int kind, const double *p, int np);
int fc_init_refine(fc_ctx *ctx, int kind, const double *p, int np);
int fc_num_fields(const fc_ctx *ctx);
int fc_read_fields(const fc_ctx *ctx, int field, void *dst, int64_t cap_bytes, int dst_is_device);
int fc_write_fields(fc_ctx *ctx, const void *src, int64_t bytes, int src_is_device);
/* fc_read_fields_async / fc_write_fields_async: the same transfers, enqueued
 *   on the context stream after the work already enqueued there, without
 *   waiting for them.  Host buffers must be page-locked (FC_ERR_INVALID_ARG
 *   for pageable memory) and stay untouched until fc_sync or another call
 *   that waits for the stream.  Contexts on different streams run
 *   concurrently, so with two contexts one can step while the other's state
 *   moves over the host link (double buffering). */
int fc_read_fields_async(const fc_ctx *ctx, int field, void *dst, int64_t cap_bytes, int dst_is_device);
int fc_write_fields_async(fc_ctx *ctx, const void *src, int64_t bytes, int src_is_device);
int fc_conservation_sums(const fc_ctx *ctx, double *sums);

/* ---- tagging and regrid -------------------------------------------------
 * fc_tag: per-leaf flags into the caller's host array (n int8): +1 refine if
 *   the criterion holds on the patch (ghost cells included); -1 for all four
 *   members of a sibling family above min_level whose averaged parent does not
 *   meet the criterion and that are not flagged +1; else 0 (Sec. 5).
 *   tagger = FC_TAGGER_PLAIN, or FC_TAGGER_LEARNED after fc_set_tagger.
 * fc_regrid: apply flags (host array, n int8): refine wins over coarsen; a
 *   family coarsens iff all four are -1 above min_level; +1 leaves below
 *   max_level split; then 2:1 balance by refinement.  New fine patches get the
 *   limited linear interpolation of their old ancestor, new coarse patches
 *   the average of their four children (Sec. 3, last paragraph). */
int fc_tag(fc_ctx *ctx, int8_t *flags_out, int tagger);
int fc_regrid(fc_ctx *ctx, const int8_t *flags);

/* ---- time stepping ------------------------------------------------------
 * fc_advance: nsteps (coarse) steps of the wave propagation method (Sec. 3)
 *   on every leaf patch: ghost fill, Roe / advection Riemann solves, MC-limited
 *   corrections with transverse propagation, conservative update, CFL
 *   reduction and (if enabled) coarse-fine flux correction (Sec. 4).
 *   dt_fixed > 0 fixes the (coarse) step; dt_fixed = 0 chooses it from the
 *   Courant condition: cfl / (largest wave speed / dx) of the previous step,
 *   or of the cell speeds after initialisation or regrid; a step whose
 *   Courant number exceeds 1 is retaken with dt <- 0.9 dt cfl / nu up to three
 *   times (FC_ERR_CFL_VIOLATION if it still exceeds 1).  With subcycle = 1
 *   level l takes 2^(l - lmin) steps of dt / 2^(l - lmin) per coarse step.
 *   On the spheres the update is in capacity form: kappa = cell area /
 *   (reference cell width)^2 of the map (equiangular on the cube; on the
 *   two trees the square of half-width r goes to colatitude pi r / 2 and
 *   areas are integrals of the map's area element), edge speeds = difference
 *   of the rotation's streamfunction over the edge / reference width, and
 *   the Courant number uses |speed| / (smaller adjacent kappa); conservation
 *   sums there are sums of cell area x q.
 *   t_out, dt_out (host, may be NULL): time after the call, last dt.
 * fc_advance_async: the same without waiting for completion and without
 *   retry bookkeeping on the host; the device retakes a step by itself and
 *   fc_sync reports the outcome. */
int fc_advance(fc_ctx *ctx, double dt_fixed, int nsteps, double *t_out, double *dt_out);
int fc_advance_async(fc_ctx *ctx, double dt_fixed, int nsteps);
int fc_sync(fc_ctx *ctx);
int fc_stats(const fc_ctx *ctx, fc_stats_t *stats);
/* fc_autotune: time the launch-shape variants of the fused patch update on
 *   each level's patches of this context's forest and state, and keep the
 *   fastest per level for later steps (a launch over all levels, under one
 *   global dt, takes the choice of the level with the most patches).
 *   Variants 0..3, one patch per CTA: bit 0 threads per CTA (128/192 for
 *   m = 8, 352/384 for m = 16, 512/1024 for m = 32); bit 1 one CTA per patch
 *   (0) or persistent CTAs that walk the patch list and copy each next patch
 *   into shared memory asynchronously while the current one is computed (1;
 *   square and periodic square only).  Variants 4..6, shallow water on the
 *   square and periodic square only: the row sweep, in which one warp fills
 *   and then sweeps the padded tiles of several patches row by row with the
 *   edge records in registers.  4: one tile column per lane (two for
 *   m = 32); 5: two columns per lane, in FP32 as one packed pair (paired
 *   FP32 instructions); 6: in FP32 the persistent form of 5, in which each
 *   warp walks the patch list and copies the next patches' interiors and
 *   same-level ghost cells into the tile rows the sweep has finished with,
 *   in FP64 four columns per lane.  The trial launches write a scratch state buffer only; the
 *   simulation state is unchanged.  variant_out (0..FC_UPDATE_VARIANTS-1, the
 *   choice for the level with the most patches) and ms_by_variant
 *   (FC_UPDATE_VARIANTS doubles, ms per launch on that level, -1 for a
 *   variant not available) may be NULL. */
#define FC_UPDATE_VARIANTS 7
int fc_autotune(fc_ctx *ctx, int *variant_out, double *ms_by_variant);
/* fc_set_variant: use launch-shape variant `variant` (as for fc_autotune) on
 *   every level for later steps, e.g. to repeat a run exactly; FC_ERR_INVALID_ARG if it is not
 *   available for this context. */
int fc_set_variant(fc_ctx *ctx, int variant);
/* fc_set_step_streams: spread the launches of a step over at most nstreams
 *   streams (1..FC_MAX_STEP_STREAMS; default 2) for later steps.  Sec. 4's
 *   sub-cycled step orders its launches by data only: level l's substep
 *   k reads its own state after substep k-1, the finer level's state at the
 *   same time and the coarser level's tiles filled for that time, and writes
 *   its new state and its flux registers; a tile fill reads the states of
 *   the filled level and its finer neighbour level at its time (blended
 *   between two substeps where the time falls inside one) and the coarser
 *   level's tiles; a coarse-fine correction reads both sides' registers and
 *   corrects the coarse level's newest state.  Launches that neither write
 *   what the other reads or writes may run at the same time (a coarse
 *   level's substep beside the finer level's substeps it does not feed), and
 *   the step graph runs them on different streams; the step control that
 *   ends the step follows all of them.  1 runs the launches one after another in plan order;
 *   results are the same bits either way.  FC_ERR_INVALID_ARG outside
 *   1..FC_MAX_STEP_STREAMS. */
#define FC_MAX_STEP_STREAMS 4
int fc_set_step_streams(fc_ctx *ctx, int nstreams);
/* fc_step_schedule: the current step graph's shape: launches per step (step
 *   control included), streams used, and the launches on its longest chain of
 *   data dependences (all launches when the step runs on one stream). */
int fc_step_schedule(fc_ctx *ctx, int *launches, int *streams, int *chain);
/* fc_profile_steps: run nsteps steps eagerly (no graph), launch after launch
 *   in plan order, with a CUDA event pair around every kernel launch on the
 *   context stream; per launch kind
 *   (0 ghost-tile fill, 1 fused update, 2 coarse-fine correction, 3 step
 *   control) write the summed device time in ms, the number of launches and
 *   the number of interior cells the launches updated (host arrays of 4).
 *   Step results are the same as fc_advance's. */
int fc_profile_steps(fc_ctx *ctx, double dt_fixed, int nsteps, double *ms_by_kind, int64_t *launches_by_kind,
                     int64_t *cells_by_kind);

/* ---- conservation sums without device allocation ---------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * must not allocate device memory, such as a process that reserves its whole
 * device-memory budget up front and only hands out fixed buffers, or code
 * where an allocation could stall the device or fail under memory pressure.
 * It sums every field times the cell area of the unit square, 1 / (2^level m)^2
 * (per-patch partials, then a fixed-order reduction): on the square and the
 * periodic square these are the sums of fc_conservation_sums.  It knows no
 * mapping, so on the two spheres, whose sums weight cells by their mapped
 * areas, its results differ from fc_conservation_sums'.  Its scratch is an
 * array compiled into the library: 131,072 patches x 3 fields of FP64
 * (3 MiB), held on every GPU that loads the library until the process exits.
 * It calls no allocating routine.
 *   q      device fields [leaf][field][j][i] in `precision` (FC_FP64 or
 *          FC_FP32), e.g. as written by fc_read_fields with dst_is_device = 1;
 *   level  device int32[n], level of each leaf (cell size 1 / (2^level m));
 *   n <= 131072 leaves, 1 <= nfields <= 3, m in {8, 16, 32}, otherwise
 *          FC_ERR_CAPACITY / FC_ERR_INVALID_ARG before any GPU work;
 *   sums   device double[nfields], written; stream: cudaStream_t or NULL.
 * The work is issued on `stream`, and the call waits for that stream to
 * finish it before returning.
 * The first call on a device looks up the scratch array's device address once,
 * with that device current; make that first call before any stream capture
 * begins.  Every call shares the one scratch array, so calls whose GPU work
 * overlaps in time (other streams or threads on the same device) race. */
int fc_conservation_sums_noalloc(const void *q, const int32_t *level, int64_t n, int m, int nfields,
                                 int precision, double *sums, void *stream);

/* ---- checkpoint -----------------------------------------------------------
 * fc_save / fc_load: forest, fields, time and step size as a little-endian
 * binary file; a resumed run continues bit for bit. */
int fc_save(const fc_ctx *ctx, const char *path);
int fc_load(fc_ctx *ctx, const char *path);

/* ---- learned tagger (no counterpart in the paper) ------------------------
 * The network stands in for the Sec. 5 criterion and predicts its flags some
 * steps ahead: 3x3 valid convolutions 3->16->16->2 with ReLU after the first
 * two, global max pool per output channel -> logits (refine, coarsen).
 * Parameters (3058 floats) in the order w1[16][3][3][3], b1[16],
 * w2[16][16][3][3], b2[16], w3[2][16][3][3], b3[2].  With bf16 = 1 weights,
 * input and hidden activations are rounded to BF16 before every product and all
 * sums accumulate in FP32; with bf16 = 0 the same kernels use FP32 values.
 * All array arguments are device memory; work runs on `stream` and the calls
 * return after it completed.
 * fc_cnn_forward: x [n][3][S][S] -> logits [n][2], 7 <= S <= 36.  With
 *   bf16 = 1 the convolutions run on the tensor cores (tcgen05 MMAs of BF16
 *   operands with FP32 accumulators in tensor memory; each 3x3 tap of a layer
 *   is one MMA over 128 output positions), the same products and FP32 sums in
 *   another order than the FP32-mode kernel; a tile whose MMAs do not
 *   complete within the wait limit (fc_cnn_set_wait_limit) makes the call
 *   return FC_ERR_TIMEOUT, with the logits of the unfinished samples
 *   undefined.
 * fc_cnn_set_wait_limit: the number of polls of a tile's completion barrier
 *   after which the tensor-core forward gives up (default 2^24; 0 makes every
 *   tile report a timeout, for testing the error path: the kernel still waits
 *   a bounded time for its MMAs before freeing their tensor memory).  Host
 *   setting, process-wide; FC_ERR_INVALID_ARG for a negative limit.
 * fc_cnn_loss_grad: mean over the n samples of the summed binary cross-entropy
 *   of the two logits against targets [n][2] in {0, 1}; gradient into grad
 *   [3058] (deterministic order), loss into *loss (host).
 * fc_cnn_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected
 *   with step >= 1) on the FP32 master weights w with moments m1, m2. */
int fc_cnn_forward(int n, int S, const float *w, const float *x, float *logits, int bf16, void *stream);
int fc_cnn_loss_grad(int n, int S, const float *w, const float *x, const float *targets, float *grad,
                     float *loss, int bf16, void *stream);
int fc_cnn_adam(float *w, const float *grad, float *m1, float *m2, int step, float lr, void *stream);
int fc_cnn_set_wait_limit(long long polls);
/* fc_cnn_input_stats: mean and standard deviation of each channel of network
 *   inputs x [n][3][S][S] (device), over all n S^2 values of the channel, in
 *   FP64 with a fixed order of summation (deterministic); stats: host
 *   double[6] = (mean h, mean hu, mean hv, sd h, sd hu, sd hv), the standard
 *   deviations about the means (two passes).  The training data's input
 *   transform is xform = (mean h, 1 / sd h, 1 / sd hu, 1 / sd hv).
 * fc_cnn_normalize: apply that transform in place, (h - xform[0]) * xform[1],
 *   hu * xform[2], hv * xform[3], evaluated in FP64 and rounded to float as
 *   fc_export_tiles does, so that raw tiles normalised here equal tiles
 *   exported with the same xform.  Both return after the work completed. */
int fc_cnn_input_stats(int n, int S, const float *x, double *stats, void *stream);
int fc_cnn_normalize(int n, int S, float *x, const double *xform, void *stream);
/* fc_export_tiles: the ghost-filled tile of every leaf at the current time
 *   (shallow water only) as network input, float [n][3][m+4][m+4] with
 *   channels (h - xform[0]) * xform[1], hu * xform[2], hv * xform[3]; dst is
 *   device memory if dst_is_device, cap = capacity in floats. */
int fc_export_tiles(fc_ctx *ctx, float *dst, int64_t cap, const double *xform, int dst_is_device);
/* fc_set_tagger: give the context network weights (host float[3058]), the
 *   input transform xform[4] of fc_export_tiles and the BF16 mode used by
 *   fc_tag(..., FC_TAGGER_LEARNED).  Learned flags combine with the plain
 *   criterion: where the network's refine probability lies in [0.4, 0.6] the
 *   plain flag is kept; otherwise a leaf is refined if the plain criterion or
 *   the network (p > 0.5) says refine, and coarsened only if both the plain
 *   flag and the network (p > 0.5) say coarsen. */
int fc_set_tagger(fc_ctx *ctx, const float *w, const double *xform, int bf16);

#ifdef __cplusplus
}
#endif
#endif
