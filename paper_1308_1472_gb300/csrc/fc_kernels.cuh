// fc_kernels.cuh -- launch interface of the patch kernels (fc_kernels.cu).
#pragma once
#include "fc_internal.cuh"

namespace fc {

// everything a field kernel needs to know about one launch
template <typename T>
struct Env {
    ForestDev f;
    T *q[3];                 // state buffers, each [F][n][m*m]
    int n, m, F;
    int eq, conn, subcycle;
    int t2;                  // corrections split transversely with the fluctuations
    int efix;                // Harten-Hyman entropy fix (shallow water)
    T g, adv_u, adv_v;
    T *gr;                   // coarse-source tiles [slot][F][(m+4)^2]
    const int *grslot;       // [n] tile slot of a patch, -1 if none
    const int *cfslot;       // [n][4] flux-register slot of a side, -1 if none
    double *reg;             // [slot][m][F]
    StepCtl *ctl;
    int lmin;                // coarsest level present
    int kdone[kMaxLevels];   // substeps finished by each level at this launch
    T alpha[kMaxLevels];     // weight of a level's newest buffer at this time
    const T *geo;            // cubed sphere: [n][geo_size(m)] patch geometry
    const int *nbrec;        // [n][kRecInts] static neighbour records
};

// static neighbour record of a patch: 9 entries of 6 ints (8 directions and
// the patch itself), padded to a whole number of 16-byte pieces
constexpr int kRecInts = 56;
int launch_nbrec(const ForestDev &f, const int *grslot, int *rec, cudaStream_t s);

// internal equation code of the fused update: scalar advection on the cubed
// sphere in capacity form (variable edge speeds, cell capacities)
constexpr int kEqSphere = 2;

// Cubed-sphere geometry of one patch, constant between regrids: inverse
// capacities 1/kappa of cells (i, j) in -1..m, speeds (flux / reference edge
// length) of x-edges (i in -1..m+1, rows -1..m) and of y-edges (i in -1..m,
// rows -1..m+1), row-major with i fastest.
__host__ __device__ constexpr int geo_ncap(int m) { return (m + 2) * (m + 2); }
__host__ __device__ constexpr int geo_nedge(int m) { return (m + 2) * (m + 3); }
__host__ __device__ constexpr int geo_size(int m) { return geo_ncap(m) + 2 * geo_nedge(m); }
__host__ __device__ constexpr int geo_cap(int m, int i, int j) { return (j + 1) * (m + 2) + (i + 1); }
__host__ __device__ constexpr int geo_sx(int m, int i, int j) { return geo_ncap(m) + (j + 1) * (m + 3) + (i + 1); }
__host__ __device__ constexpr int geo_sy(int m, int i, int j)
{
    return geo_ncap(m) + geo_nedge(m) + (j + 1) * (m + 2) + (i + 1);
}

// patch-list launch description
struct List {
    const int *idx;          // patch indices (device), or nullptr for 0..count-1
    int count;
};

template <typename T> int launch_fill_tiles(const Env<T> &e, List l, cudaStream_t s);
// one substep of the listed patches; ksub: substep index of the updated
// level; fine_acc: sides facing a coarser level add to their register
// variant 0..3: one CTA per patch (bit 0: threads per CTA; bit 1: the
// persistent pipelined kernel, not on the cubed sphere); 4..6: the row sweep
// (fc_sweep.cuh), shallow water only: 4 one column per lane (two for m = 32),
// 5 two columns per lane (packed FP32 pairs), 6 FP32: persistent form of 5
// with the next patches copied during the sweep, FP64: four columns per lane
constexpr int kUpdateVariants = 7;
// number of variants (0 .. n-1) available for an equation and connectivity
inline int update_variant_count(int eq, int conn, bool t2, bool efix)
{
    if (conn == FC_CONN_SPHERE || t2 || efix) return 2;
    return eq == FC_EQ_SWE ? 7 : 4;
}
template <typename T> int launch_update(const Env<T> &e, List l, int ksub, int fine_acc, int variant, cudaStream_t s);
// the fused update with T2 and / or the entropy fix (fc_update_ext.cu):
// variants 0 and 1 (threads per CTA) of the one-CTA-per-patch kernel
template <typename T> int launch_update_ext(const Env<T> &e, List l, int ksub, int fine_acc, int variant,
                                            cudaStream_t s);
// row-sweep update (fc_sweep.cuh), k = 0..2 selects the columns per lane
template <typename T> int launch_sweep(const Env<T> &e, List l, int fine_acc, int k, cudaStream_t s);
int launch_level_dt(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, cudaStream_t s);
// patches: coarse patches with a finer face neighbour; the coarse level's
// newest buffer (after kdone substeps) is corrected
template <typename T> int launch_reflux(const Env<T> &e, List patches, cudaStream_t s);
int launch_step_ctl(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, const int *nsub,
                    cudaStream_t s);
template <typename T> int launch_cell_rate(const Env<T> &e, cudaStream_t s);
int launch_dt_from_next(StepCtl *ctl, cudaStream_t s);
int launch_dt_from_cells(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, cudaStream_t s);
template <typename T> int launch_init(const Env<T> &e, int kind, const double *d_p, int np, cudaStream_t s);
template <typename T> int launch_sums(const Env<T> &e, double *d_part, double *d_out, cudaStream_t s);
template <typename T> int launch_tag(const Env<T> &e, int crit, double thr, int min_level, int8_t *d_flags,
                                     cudaStream_t s);
// regrid transfer into enew.q[0] from the old state, origin records
// {kind, old index, level difference} and complete tiles of the old leaves
template <typename T> int launch_transfer(const Env<T> &eold, const Env<T> &enew, const int *origin,
                                          const T *tiles_old, const int *old_x, const int *old_y,
                                          cudaStream_t s);
// cubed sphere: geometry of every patch into geo (FP64 evaluation, stored in T)
template <typename T> int launch_geometry(const Env<T> &e, double omega, double tilt, T *geo, cudaStream_t s);
template <typename T> int launch_read(const Env<T> &e, int field, T *dst, cudaStream_t s);
template <typename T> int launch_write(const Env<T> &e, const T *src, cudaStream_t s);
// write with the cell-speed maxima of the new state folded in (shallow water)
template <typename T> int launch_write_speed(const Env<T> &e, const T *src, cudaStream_t s);

}  // namespace fc
