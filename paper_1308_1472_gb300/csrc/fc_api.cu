// fc_api.cu -- the C ABI (include/fc.h): context, forest preparation, the
// static launch plan of one (coarse) step captured as a CUDA graph, regrid,
// tagging, field I/O and checkpoints.
//
// Sec. 4 of the paper: one exchange and update per step with a global dt, or,
// with sub-cycling, a coarse-to-fine recursion (level l takes two steps per
// step of level l-1, fine ghost values time-interpolated between the coarse
// level's old and new states) followed by the fine-to-coarse correction.
// Here the recursion is unrolled once per forest into a fixed list of kernel
// launches; the step size, the accept / retake decision and the buffer that
// holds each level's state live in device memory, so steps are replayed from
// the graph without host round trips.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <bitset>
#include <cstring>
#include <vector>

#include "fc_forest.cuh"
#include "fc_kernels.cuh"

namespace fc {

static thread_local char g_msg[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
}

int cuda_status(cudaError_t e, const char *what)
{
    set_error("CUDA error %s (%d) in %s", cudaGetErrorString(e), (int)e, what);
    return FC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// preparation kernels
__global__ void k_flag_tile(const int *nbr, int n, int *flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int any = 0;
    for (int d = 0; d < 8; ++d) any |= nbr[(size_t)i * 32 + 4 * d] == FC_NB_FINER;
    flag[i] = any;
}
__global__ void k_flag_cf_side(const int *nbr, int n, int *flag)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n * 4) return;
    int k = nbr[(size_t)(g >> 2) * 32 + 4 * (g & 3)];
    flag[g] = k == FC_NB_FINER || k == FC_NB_COARSER;
}
// counts that size the per-forest lists, in one pass: patches per level
// [0, 16), patches with a finer neighbour per level [16, 32), patches with a
// finer face neighbour per level [32, 48), then the totals of tile patches,
// coarse-fine sides and coarse patches [48, 51), and patches with a coarser
// neighbour (in any of the 8 directions) per level [51, 67)
constexpr int kPrepCounts = 67;
__global__ void k_prep_counts(const int *nbr, const int *level, int n, int *cnt)
{
    __shared__ int sh[kPrepCounts];
    for (int k = threadIdx.x; k < kPrepCounts; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int l = level[i];
        int tile = 0, face = 0, sides = 0, coarser = 0;
        for (int d = 0; d < 8; ++d) {
            const int k = nbr[(size_t)i * 32 + 4 * d];
            tile |= k == FC_NB_FINER;
            coarser |= k == FC_NB_COARSER;
            if (d < 4) { face |= k == FC_NB_FINER; sides += k == FC_NB_FINER || k == FC_NB_COARSER; }
        }
        atomicAdd(&sh[l], 1);
        if (coarser) atomicAdd(&sh[51 + l], 1);
        if (tile) { atomicAdd(&sh[16 + l], 1); atomicAdd(&sh[48], 1); }
        if (face) { atomicAdd(&sh[32 + l], 1); atomicAdd(&sh[50], 1); }
        if (sides) atomicAdd(&sh[49], sides);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kPrepCounts; k += blockDim.x)
        if (sh[k]) atomicAdd(&cnt[k], sh[k]);
}

// All per-level lists of a forest in three launches: a stable partition of
// the leaves (SFC order kept inside every bucket) into 65 buckets: patches of
// level l without a coarser neighbour [2l] and with one [2l + 1] (so that a
// level's list holds its interior patches first, then those next to the
// coarser level), patches with a finer neighbour (tiles) of level l
// [32, 48), patches with a finer face neighbour (coarse sides) of level l
// [48, 64), and the latter of every level [64].  A leaf belongs to one bucket
// of each family at most.
constexpr int kListBuckets = 65, kListBlock = 512;
__device__ __forceinline__ void list_keys(const int *nbr, const int *level, int i, int key[4])
{
    int tile = 0, face = 0, coarser = 0;
    for (int d = 0; d < 8; ++d) {
        const int k = nbr[(size_t)i * 32 + 4 * d];
        tile |= k == FC_NB_FINER;
        coarser |= k == FC_NB_COARSER;
        if (d < 4) face |= k == FC_NB_FINER;
    }
    const int l = level[i];
    key[0] = 2 * l + coarser;
    key[1] = tile ? 32 + l : -1;
    key[2] = face ? 48 + l : -1;
    key[3] = face ? 64 : -1;
}
// per block and bucket: number of the block's leaves in the bucket
__global__ void __launch_bounds__(kListBlock) k_list_counts(const int *nbr, const int *level, int n, int *bc)
{
    __shared__ int sh[kListBuckets];
    for (int k = threadIdx.x; k < kListBuckets; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const int i = blockIdx.x * kListBlock + threadIdx.x;
    if (i < n) {
        int key[4];
        list_keys(nbr, level, i, key);
        for (int f = 0; f < 4; ++f)
            if (key[f] >= 0) atomicAdd(&sh[key[f]], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kListBuckets; k += blockDim.x) bc[(size_t)k * gridDim.x + blockIdx.x] = sh[k];
}
// exclusive scan over the blocks of every bucket, one warp per bucket
__global__ void k_list_scan(int *bc, int nblk)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= kListBuckets) return;
    int *row = bc + (size_t)b * nblk;
    int carry = 0;
    for (int c0 = 0; c0 < nblk; c0 += 32) {
        const int v = c0 + lane < nblk ? row[c0 + lane] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (c0 + lane < nblk) row[c0 + lane] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
}
// every leaf to its place: bucket base + the block's offset + its stable rank
// among the block's leaves of that bucket
struct ListOut {
    int base[kListBuckets];      // first output index of every bucket
    int *out[4];                 // output array of each family
};
__global__ void __launch_bounds__(kListBlock) k_list_scatter(const int *nbr, const int *level, int n, const int *bc,
                                                             ListOut lo)
{
    constexpr int NW = kListBlock / 32;
    __shared__ int wc[4][NW][kListBuckets];
    const int i = blockIdx.x * kListBlock + threadIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int key[4] = {-1, -1, -1, -1};
    if (i < n) list_keys(nbr, level, i, key);
    for (int k = threadIdx.x; k < 4 * NW * kListBuckets; k += blockDim.x) (&wc[0][0][0])[k] = 0;
    __syncthreads();
    int rank[4];
    const unsigned lt = (1u << lane) - 1u;
    for (int f = 0; f < 4; ++f) {
        const unsigned same = __match_any_sync(0xffffffffu, key[f]);
        rank[f] = __popc(same & lt);
        if (key[f] >= 0 && rank[f] == 0) wc[f][w][key[f]] = __popc(same);
    }
    __syncthreads();
    for (int f = 0; f < 4; ++f) {
        if (key[f] < 0) continue;
        int r = rank[f];
        for (int v = 0; v < w; ++v) r += wc[f][v][key[f]];
        const int b = key[f];
        lo.out[f][lo.base[b] + bc[(size_t)b * gridDim.x + blockIdx.x] + r] = i;
    }
}

__global__ void k_slot_of(const int *flag, const int *off, int n, int *slot)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot[i] = flag[i] ? off[i] : -1;
}
__global__ void k_iota(int *a, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}
static inline int nb256(long long n) { return (int)((n + 255) / 256); }

// network input from complete tiles [n][F][S*S] (shallow water)
template <typename T>
__global__ void k_tiles_to_input(const T *tiles, int n, int SS, double ref, double s0, double s1, double s2,
                                 float *out)
{
    size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (size_t)n * 3 * SS) return;
    int f = (int)((g / SS) % 3);
    double v = (double)tiles[g];
    out[g] = (float)(f == 0 ? (v - ref) * s0 : v * (f == 1 ? s1 : s2));
}

// combine plain flags with the network's probabilities
__global__ void k_combine_flags(int8_t *flags, const float *logits, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float pr = 1.f / (1.f + expf(-logits[2 * i])), pc = 1.f / (1.f + expf(-logits[2 * i + 1]));
    int plain = flags[i], f;
    if (pr >= 0.4f && pr <= 0.6f) f = plain;
    else if (plain == 1 || pr > 0.5f) f = 1;
    else if (plain == -1 && pc > 0.5f) f = -1;
    else f = 0;
    flags[i] = (int8_t)f;
}

// one step-plan entry
struct Launch {
    enum Kind { FILL, UPDATE, REFLUX } kind;
    enum Part { WHOLE, INTERIOR, BORDER };
    int level;        // level of the listed patches / sides, -1 = all
    int part;         // UPDATE: the level's patches without / with a coarser neighbour, or all
    int ksub;         // UPDATE: substep index of the level
    int fine_acc;
    int kdone[kMaxLevels];
    double alpha[kMaxLevels];
};

}  // namespace fc

using namespace fc;

struct fc_ctx {
    fc_params p;
    int F = 3;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Forest forest;
    size_t esize = 8;
    DBuf<unsigned char> q[3];
    // per-forest preparation
    int lmin = 0, lmax = 0;
    DBuf<int> levlist;   int lev_off[kMaxLevels + 1] = {0};
    int lev_int[kMaxLevels] = {0};   // patches of a level without a coarser neighbour (listed first)
    DBuf<int> tilelist;  int tile_off[kMaxLevels + 1] = {0};
    DBuf<int> cflist;    int cf_off[kMaxLevels + 2] = {0};   // coarse patches of coarse-fine faces; last: all levels
    DBuf<int> grslot, cfslot, iota;
    DBuf<int> nbrec;              // static neighbour records [n][kRecInts]
    DBuf<int> list_bc;            // list building: per bucket and block counts / offsets
    DBuf<unsigned char> gr;
    DBuf<unsigned char> geo;      // cubed sphere: per-patch geometry [n][geo_size(m)]
    DBuf<double> reg;
    int ntile = 0, ncf = 0;
    double dx[kMaxLevels] = {0};
    int nsub[kMaxLevels] = {0};
    int64_t updates_per_step = 0;
    // step control
    StepCtl *d_ctl = nullptr;
    StepCtl *h_ctl = nullptr;     // pinned mirror
    double *h_stage = nullptr;    // pinned staging for host -> device pushes
    double cur_dt_fixed = -1.0;   // step-size mode last pushed
    int acc_seen = 0;             // accepted-step counter value last accounted
    bool unbalanced = false;      // imported forest awaiting fc_forest_balance
    int upd_variant = 0;          // launch shape of the fused update (fc_set_variant / fc_autotune)
    int upd_variant_lv[kMaxLevels];   // per-level choice of fc_autotune, -1: upd_variant
    // learned tagger
    DBuf<float> tag_w, tag_x, tag_logits;
    double tag_xform[4] = {1.0, 1.0, 1.0, 1.0};
    int tag_bf16 = 1;
    bool tag_ready = false;
    bool dt_from_cells = true;
    bool speeds_ready = false;    // the cell-speed maxima of the current state are in StepCtl already
    std::vector<Launch> plan;
    bool plan_valid = false;
    // the step's launches spread over streams (the context stream and side
    // streams created on first use), ordered by their data dependences
    int step_streams = 2;                       // at most (fc_set_step_streams)
    int plan_nstreams = 1;                      // used by the current plan
    int plan_chain = 0;                         // launches on the longest dependence chain
    std::vector<int> plan_stream;               // stream of each launch
    std::vector<std::vector<int>> plan_waits;   // launches in other streams it waits for
    std::vector<char> plan_signal;              // launches that another stream waits for
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> sev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // counters
    int64_t cell_updates = 0, steps = 0, regrids = 0;
    // scratch
    DBuf<double> part, sums, dparams;
    DBuf<int8_t> flags;
    DBuf<unsigned char> io;
    DBuf<int> scan_tmp, scan_off;
    DBuf<int> scan_bs;
};

// ---------------------------------------------------------------------------
namespace fc {

// device address of a page-locked (pinned or registered) host buffer, through
// which kernels read and write it directly over the host link; nullptr for
// pageable memory (which then goes through a device staging buffer)
static void *pinned_device_pointer(const void *host)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();                // clear the sticky-free error of an unknown pointer
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// per-patch geometry (capacities, edge speeds): the cubed sphere, and the
// swirl velocity field on the square
static bool has_geometry(const fc_ctx *c)
{
    return fc::is_sphere_conn(c->p.conn) || (c->p.equation == FC_EQ_ADV && c->p.velocity == FC_VEL_SWIRL);
}

template <typename T>
static Env<T> make_env(const fc_ctx *c)
{
    Env<T> e;
    memset(&e, 0, sizeof e);
    e.f = c->forest.dev();
    for (int b = 0; b < 3; ++b) e.q[b] = (T *)c->q[b].p;
    e.n = c->forest.n;
    e.m = c->p.m;
    e.F = c->F;
    e.eq = c->p.equation;
    e.t2 = c->p.transverse == 2;
    e.efix = c->p.equation == FC_EQ_SWE && c->p.entropy_fix;
    e.conn = c->p.conn;
    e.subcycle = c->p.subcycle;
    e.g = (T)c->p.g;
    e.adv_u = (T)c->p.adv_u;
    e.adv_v = (T)c->p.adv_v;
    e.gr = (T *)c->gr.p;
    e.grslot = c->grslot.p;
    e.cfslot = c->ncf > 0 ? c->cfslot.p : nullptr;
    e.reg = c->reg.p;
    e.ctl = c->d_ctl;
    e.lmin = c->lmin;
    for (int l = 0; l < kMaxLevels; ++l) { e.kdone[l] = 0; e.alpha[l] = T(1); }
    e.geo = has_geometry(c) ? (const T *)c->geo.p : nullptr;
    e.nbrec = c->nbrec.p;
    return e;
}

// compact indices of flag[0..n) into out (device); with h_count the count
// is also brought to the host (a synchronisation)
// the step plan must be rebuilt; the instantiated graph is kept so that the
// next capture can update it in place when its shape is unchanged
static void invalidate_plan(fc_ctx *c)
{
    c->plan_valid = false;
}

static void release_graph(fc_ctx *c)
{
    c->plan_valid = false;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

// lists and slots that depend on the forest; state buffers sized to it
static int prepare(fc_ctx *c, bool zero_state)
{
    Forest &f = c->forest;
    int n = f.n, m = c->p.m, F = c->F;
    cudaStream_t s = c->stream;
    invalidate_plan(c);
    FC_TRY(c->scan_tmp.alloc((size_t)n * 4 + 1, s));
    FC_TRY(c->levlist.alloc(n, s));
    // all list sizes in one pass and one host round trip; the lists are then
    // built without further synchronisation
    int hc[kPrepCounts];
    {
        DBuf<int> dc;
        FC_TRY(dc.alloc(kPrepCounts, s));
        FC_CUDA(cudaMemsetAsync(dc.p, 0, sizeof(int) * kPrepCounts, s));
        if (n > 0) k_prep_counts<<<nb256(n), 256, 0, s>>>(f.nbr.p, f.level.p, n, dc.p);
        FC_CUDA(cudaGetLastError());
        FC_CUDA(cudaMemcpyAsync(hc, dc.p, sizeof(int) * kPrepCounts, cudaMemcpyDeviceToHost, s));
        FC_CUDA(cudaStreamSynchronize(s));
    }
    // list offsets from the counts
    c->lmin = 99; c->lmax = -1;
    int tot = 0;
    for (int l = 0; l < kMaxLevels; ++l) {
        c->lev_off[l] = tot;
        if (hc[l] > 0) {
            if (l < c->lmin) c->lmin = l;
            c->lmax = l;
        }
        tot += hc[l];
    }
    c->lev_off[kMaxLevels] = tot;
    for (int l = 0; l < kMaxLevels; ++l) c->lev_int[l] = hc[l] - hc[51 + l];
    tot = 0;
    for (int l = 0; l < kMaxLevels; ++l) { c->tile_off[l] = tot; tot += hc[16 + l]; }
    c->tile_off[kMaxLevels] = tot;
    tot = 0;
    for (int l = 0; l < kMaxLevels; ++l) { c->cf_off[l] = tot; tot += hc[32 + l]; }
    c->cf_off[kMaxLevels] = tot;
    c->cf_off[kMaxLevels + 1] = tot + hc[50];
    // patches with a finer neighbour keep complete tiles (coarse sources)
    DBuf<int> tflag;
    FC_TRY(tflag.alloc(n, s));
    k_flag_tile<<<nb256(n), 256, 0, s>>>(f.nbr.p, n, tflag.p);
    FC_TRY(c->grslot.alloc(n, s));
    FC_TRY(c->scan_off.alloc(n, s));
    FC_TRY(exclusive_scan(tflag.p, c->scan_off.p, n, nullptr, c->scan_bs, s));
    c->ntile = hc[48];
    k_slot_of<<<nb256(n), 256, 0, s>>>(tflag.p, c->scan_off.p, n, c->grslot.p);
    FC_TRY(c->nbrec.alloc((size_t)(n > 0 ? n : 1) * kRecInts, s));
    FC_TRY(launch_nbrec(f.dev(), c->grslot.p, c->nbrec.p, s));
    FC_TRY(c->tilelist.alloc(c->ntile + 1, s));
    size_t PP = (size_t)(m + 4) * (m + 4);
    FC_TRY(c->gr.alloc((size_t)(c->ntile > 0 ? c->ntile : 1) * F * PP * c->esize, s));
    // coarse-fine sides: register slots, and coarse sides per level
    FC_TRY(c->cfslot.alloc((size_t)n * 4, s));
    k_flag_cf_side<<<nb256((long long)n * 4), 256, 0, s>>>(f.nbr.p, n, c->scan_tmp.p);
    FC_TRY(c->scan_off.alloc((size_t)n * 4, s));
    FC_TRY(exclusive_scan(c->scan_tmp.p, c->scan_off.p, n * 4, nullptr, c->scan_bs, s));
    c->ncf = hc[49];
    k_slot_of<<<nb256((long long)n * 4), 256, 0, s>>>(c->scan_tmp.p, c->scan_off.p, n * 4, c->cfslot.p);
    FC_TRY(c->reg.alloc((size_t)(c->ncf > 0 ? c->ncf : 1) * m * F, s));
    FC_TRY(c->cflist.alloc((size_t)n * 2 + 1, s));
    // the per-level lists (levels, tiles, coarse patches) and the all-level
    // coarse-patch list after the per-level ones, in three launches
    if (n > 0) {
        const int nblk = (n + kListBlock - 1) / kListBlock;
        FC_TRY(c->list_bc.alloc((size_t)kListBuckets * nblk, s));
        ListOut lo;
        for (int l = 0; l < kMaxLevels; ++l) {
            lo.base[2 * l] = c->lev_off[l];
            lo.base[2 * l + 1] = c->lev_off[l] + c->lev_int[l];
            lo.base[32 + l] = c->tile_off[l];
            lo.base[48 + l] = c->cf_off[l];
        }
        lo.base[64] = c->cf_off[kMaxLevels];
        lo.out[0] = c->levlist.p; lo.out[1] = c->tilelist.p; lo.out[2] = c->cflist.p; lo.out[3] = c->cflist.p;
        k_list_counts<<<nblk, kListBlock, 0, s>>>(f.nbr.p, f.level.p, n, c->list_bc.p);
        k_list_scan<<<(kListBuckets + 7) / 8, 256, 0, s>>>(c->list_bc.p, nblk);
        k_list_scatter<<<nblk, kListBlock, 0, s>>>(f.nbr.p, f.level.p, n, c->list_bc.p, lo);
        FC_CUDA(cudaGetLastError());
    }
    FC_TRY(c->iota.alloc(n, s));
    k_iota<<<nb256(n), 256, 0, s>>>(c->iota.p, n);
    FC_CUDA(cudaGetLastError());
    // state
    size_t bytes = (size_t)F * n * m * m * c->esize;
    for (int b = 0; b < 3; ++b) {
        FC_TRY(c->q[b].alloc(bytes, s));
        if (zero_state) FC_CUDA(cudaMemsetAsync(c->q[b].p, 0, bytes, s));
    }
    // cubed sphere: capacities and edge speeds of every patch (constant
    // until the forest changes)
    if (has_geometry(c)) {
        FC_TRY(c->geo.alloc((size_t)(n > 0 ? n : 1) * geo_size(m) * c->esize, s));
        if (c->esize == 8) {
            Env<double> e = make_env<double>(c);
            FC_TRY(launch_geometry<double>(e, c->p.omega, c->p.omega_axis_tilt, (double *)c->geo.p, s));
        } else {
            Env<float> e = make_env<float>(c);
            FC_TRY(launch_geometry<float>(e, c->p.omega, c->p.omega_axis_tilt, (float *)c->geo.p, s));
        }
    }
    // level geometry and substep counts
    c->updates_per_step = 0;
    for (int l = 0; l < kMaxLevels; ++l) {
        c->dx[l] = 1.0 / ((double)(1 << l) * m);
        int cnt = c->lev_off[l + 1] - c->lev_off[l];
        c->nsub[l] = cnt > 0 ? (c->p.subcycle ? (1 << (l - c->lmin)) : 1) : 0;
        c->updates_per_step += (int64_t)cnt * c->nsub[l] * m * m;
    }
    FC_CUDA(cudaStreamSynchronize(s));
    return FC_OK;
}

// a new state (initial data, written fields, a new forest, a checkpoint)
// clears the sticky error flags of the previous one
static int clear_errors(fc_ctx *c)
{
    const size_t off = offsetof(StepCtl, cfl_error);
    FC_CUDA(cudaMemsetAsync((char *)c->d_ctl + off, 0, 4 * sizeof(int), c->stream));
    c->h_ctl->cfl_error = c->h_ctl->dry_error = c->h_ctl->nonfinite_error = c->h_ctl->index_error = 0;
    return FC_OK;
}

static int reset_ctl_buffers(fc_ctx *c)
{
    // every level's state in buffer 0
    FC_CUDA(cudaMemsetAsync(c->d_ctl->start_buf, 0, sizeof(int) * kMaxLevels, c->stream));
    return clear_errors(c);
}

// ---------------------------------------------------------------------------
// the step plan

// launch shape of the fused update of one level (-1: a launch over all levels)
static int variant_for(const fc_ctx *c, int level)
{
    if (level >= 0 && level < kMaxLevels && c->upd_variant_lv[level] >= 0) return c->upd_variant_lv[level];
    return c->upd_variant;
}

// the state of every level at substep time T.  Under sub-cycling a level
// whose last substep started at T is seen through the state before that
// substep (no blend, and the launch does not wait for the substep), one that
// ended at T through its newest state, and one in between through the blend
// of the two.  (The global-dt plan views every level at T = 0; its coarse-fine
// correction corrects the newest buffer, substep kdone, whatever the blend.)
static void plan_view(const fc_ctx *c, const int *kd, long long T, Launch &L)
{
    for (int l = 0; l < kMaxLevels; ++l) {
        L.kdone[l] = kd[l];
        L.alpha[l] = 1.0;
        if (c->nsub[l] == 0 || kd[l] == 0) continue;
        long long tl = 1LL << (c->lmax - l);
        long long tnew = (long long)kd[l] * tl, told = tnew - tl;
        if (c->p.subcycle && T == told) L.kdone[l] = kd[l] - 1;
        else if (T != tnew) L.alpha[l] = (double)(T - told) / (double)(tnew - told);
    }
}

// Sub-cycling recursion (Sec. 4).  last_fill[lv] is the substep time of the
// latest tile fill of level lv in the plan so far (-1 after a coarse-fine
// correction, which changes values the tiles read): a level's tiles at a time
// they were last filled for hold the same values again (the states of every
// time a tile reads stay in their buffers until the level steps on), so that
// fill is not repeated.
static void plan_level(fc_ctx *c, int l, int *kd, long long *last_fill)
{
    long long T = (long long)kd[l] << (c->lmax - l);
    for (int lv = c->lmin; lv < l; ++lv) {
        if (c->tile_off[lv + 1] - c->tile_off[lv] == 0) continue;
        if (last_fill[lv] == T) continue;
        last_fill[lv] = T;
        Launch L{};
        L.kind = Launch::FILL; L.level = lv;
        plan_view(c, kd, T, L);
        c->plan.push_back(L);
    }
    Launch U{};
    U.kind = Launch::UPDATE; U.level = l; U.ksub = kd[l] + 1;
    U.fine_acc = (l > c->lmin) && (kd[l] & 1);
    plan_view(c, kd, T, U);
    // the finest level's substep as two launches when the step runs on
    // several streams: its patches next to the coarser level (they read the
    // coarser tiles and write the fine-side registers) and the others, which
    // then need neither the fills nor the corrections before them
    const int nint = c->lev_int[l], nall = c->lev_off[l + 1] - c->lev_off[l];
    if (l == c->lmax && l > c->lmin && c->step_streams > 1 && nint > 0 && nint < nall) {
        U.part = Launch::BORDER;
        c->plan.push_back(U);
        U.part = Launch::INTERIOR;
        U.fine_acc = 0;
        c->plan.push_back(U);
    } else {
        c->plan.push_back(U);
    }
    kd[l] += 1;
    if (l < c->lmax) {
        plan_level(c, l + 1, kd, last_fill);
        plan_level(c, l + 1, kd, last_fill);
        if (c->p.refluxing && c->cf_off[l + 1] - c->cf_off[l] > 0) {
            for (int lv = 0; lv < kMaxLevels; ++lv) last_fill[lv] = -1;
            Launch R{};
            R.kind = Launch::REFLUX; R.level = l;
            plan_view(c, kd, (long long)kd[l] << (c->lmax - l), R);
            c->plan.push_back(R);
        }
    }
}

static void schedule_plan(fc_ctx *c);

static void build_plan(fc_ctx *c)
{
    c->plan.clear();
    if (c->p.subcycle) {
        int kd[kMaxLevels] = {0};
        long long last_fill[kMaxLevels];
        for (int l = 0; l < kMaxLevels; ++l) last_fill[l] = -1;
        plan_level(c, c->lmin, kd, last_fill);
    } else {
        int kd[kMaxLevels] = {0};
        for (int l = c->lmin; l < c->lmax; ++l) {
            if (c->tile_off[l + 1] - c->tile_off[l] == 0) continue;
            Launch L{};
            L.kind = Launch::FILL; L.level = l;
            plan_view(c, kd, 0, L);
            c->plan.push_back(L);
        }
        Launch U{};
        U.kind = Launch::UPDATE; U.level = -1; U.ksub = 1; U.fine_acc = 0;
        plan_view(c, kd, 0, U);
        c->plan.push_back(U);
        if (c->p.refluxing && c->cf_off[kMaxLevels + 1] - c->cf_off[kMaxLevels] > 0) {
            for (int l = 0; l < kMaxLevels; ++l) kd[l] = c->nsub[l] ? 1 : 0;
            Launch R{};
            R.kind = Launch::REFLUX; R.level = -1;
            plan_view(c, kd, 0, R);
            c->plan.push_back(R);
        }
    }
    schedule_plan(c);
}

// ---------------------------------------------------------------------------
// data dependences between the launches of a step
//
// A launch touches three levels at most.  Per level the resources are the
// state buffers of the three substep slots (slot 0: the state at the start of
// the coarse step; substeps 1, 2, 3, ... alternate between slots 1 and 2), the
// coarse-source tiles, the flux registers of the level's coarse sides (facing
// level l+1) and those of its fine sides (facing level l-1).  Two launches
// are ordered when one of them writes what the other reads or writes; any
// other two may run at the same time.
//
// The state of a level is two resources per slot: its patches without a
// coarser neighbour (in any of the 8 directions; interior) and those with
// one (border).  A finer neighbour of a level-l patch is a border patch of
// level l+1; ghost values from coarser neighbours come from the coarser
// level's tiles only, never from its states.
constexpr int kResPerLevel = 9;
using ResSet = std::bitset<kResPerLevel * kMaxLevels>;
static int res_state(int l, int k, int border)
{
    return kResPerLevel * l + 3 * border + (k == 0 ? 0 : 1 + ((k - 1) & 1));
}
static int res_tiles(int l) { return kResPerLevel * l + 6; }
static int res_reg_coarse(int l) { return kResPerLevel * l + 7; }
static int res_reg_fine(int l) { return kResPerLevel * l + 8; }

// the states of level l (interior and / or border part) that a launch's time
// view reads
static void view_reads(const Launch &L, int l, bool interior, ResSet &r)
{
    if (l < 0 || l >= kMaxLevels) return;
    for (int b = interior ? 0 : 1; b < 2; ++b) {
        r.set(res_state(l, L.kdone[l], b));
        if (L.kdone[l] > 0 && L.alpha[l] != 1.0) r.set(res_state(l, L.kdone[l] - 1, b));
    }
}

static void launch_access(const Launch &L, int lmax, ResSet &r, ResSet &w)
{
    r.reset();
    w.reset();
    const int l = L.level;
    if (l < 0) { r.set(); w.set(); return; }       // a launch over all levels
    if (L.kind == Launch::REFLUX) {                // newest state of l from both sides' registers
        r.set(res_reg_coarse(l));
        if (l + 1 < kMaxLevels) r.set(res_reg_fine(l + 1));
        for (int b = 0; b < 2; ++b) {
            r.set(res_state(l, L.kdone[l], b));
            w.set(res_state(l, L.kdone[l], b));
        }
        return;
    }
    // ghost values: same-level neighbours and the finer level's border
    // patches from their states at the launch's time, coarser neighbours
    // from the coarser level's tiles (read by border patches only)
    view_reads(L, l, true, r);
    view_reads(L, l + 1, false, r);
    if (l > 0 && !(L.kind == Launch::UPDATE && L.part == Launch::INTERIOR)) r.set(res_tiles(l - 1));
    if (L.kind == Launch::FILL) {
        w.set(res_tiles(l));
        return;
    }
    if (L.part != Launch::BORDER) w.set(res_state(l, L.ksub, 0));
    if (L.part != Launch::INTERIOR) {
        w.set(res_state(l, L.ksub, 1));
        w.set(res_reg_fine(l));
        if (L.fine_acc) r.set(res_reg_fine(l));    // adds to the first substep's sums
    }
    if (l < lmax) w.set(res_reg_coarse(l));
}

// Spread the plan over at most c->step_streams streams: a launch goes to the
// stream whose last launch it has to follow anyway (the latest such), else to
// an unused stream, else to the stream that has waited longest (an order the
// data do not need); it waits for the latest launch it depends on in each
// other stream.  The step control that ends the step follows all of them.
static constexpr int kMaxScheduled = 4096;        // longer plans run as one chain
static void schedule_plan(fc_ctx *c)
{
    const int np = (int)c->plan.size();
    c->plan_stream.assign(np, 0);
    c->plan_waits.assign(np, std::vector<int>());
    c->plan_signal.assign(np, 0);
    c->plan_nstreams = 1;
    c->plan_chain = np + 1;
    const int ns = c->step_streams;
    if (np == 0 || ns <= 1 || np > kMaxScheduled) return;
    std::vector<ResSet> R(np), W(np);
    for (int i = 0; i < np; ++i) launch_access(c->plan[i], c->lmax, R[i], W[i]);
    const int nw = (np + 63) / 64;
    std::vector<uint64_t> anc((size_t)np * nw, 0);      // ancestors of each launch
    std::vector<int> depth(np, 1);
    std::vector<std::vector<int>> dep(np);
    int chain = 0;
    for (int i = 0; i < np; ++i) {
        uint64_t *ai = &anc[(size_t)i * nw];
        for (int j = 0; j < i; ++j) {
            if (!(W[j] & R[i]).any() && !(W[j] & W[i]).any() && !(R[j] & W[i]).any()) continue;
            dep[i].push_back(j);
            const uint64_t *aj = &anc[(size_t)j * nw];
            for (int k = 0; k < nw; ++k) ai[k] |= aj[k];
            ai[j >> 6] |= 1ULL << (j & 63);
            if (depth[j] + 1 > depth[i]) depth[i] = depth[j] + 1;
        }
        if (depth[i] > chain) chain = depth[i];
    }
    std::vector<int> tail(ns, -1);
    for (int i = 0; i < np; ++i) {
        const uint64_t *ai = &anc[(size_t)i * nw];
        int best = -1;
        for (int k = 0; k < ns; ++k)
            if (tail[k] >= 0 && ((ai[tail[k] >> 6] >> (tail[k] & 63)) & 1) && (best < 0 || tail[k] > tail[best]))
                best = k;
        for (int k = 0; k < ns && best < 0; ++k)
            if (tail[k] < 0) best = k;
        if (best < 0) {
            best = 0;
            for (int k = 1; k < ns; ++k)
                if (tail[k] < tail[best]) best = k;
        }
        c->plan_stream[i] = best;
        std::vector<int> last(ns, -1);
        for (int j : dep[i])
            if (c->plan_stream[j] != best && j > last[c->plan_stream[j]]) last[c->plan_stream[j]] = j;
        for (int k = 0; k < ns; ++k)
            if (last[k] >= 0) { c->plan_waits[i].push_back(last[k]); c->plan_signal[last[k]] = 1; }
        tail[best] = i;
        if (best + 1 > c->plan_nstreams) c->plan_nstreams = best + 1;
    }
    c->plan_chain = chain + 1;
}

// side streams and events of the schedule (kept until the context goes);
// created before a capture begins
static int ensure_schedule_objects(fc_ctx *c)
{
    const size_t nside = (size_t)(c->plan_nstreams - 1), nev = c->plan.size() + (size_t)c->plan_nstreams;
    while (c->side.size() < nside) {
        cudaStream_t st;
        FC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        c->side.push_back(st);
    }
    while (c->sev.size() < nev) {
        cudaEvent_t ev;
        FC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->sev.push_back(ev);
    }
    return FC_OK;
}

// the patches of an update launch of one level: all of them, or the
// interior (first in the level's list) or the border part
static List update_list(const fc_ctx *c, const Launch &L)
{
    const int l = L.level, lo = c->lev_off[l], hi = c->lev_off[l + 1], mid = lo + c->lev_int[l];
    if (L.part == Launch::INTERIOR) return List{c->levlist.p + lo, mid - lo};
    if (L.part == Launch::BORDER) return List{c->levlist.p + mid, hi - mid};
    return List{c->levlist.p + lo, hi - lo};
}

template <typename T>
static int launch_one(fc_ctx *c, const Launch &L, cudaStream_t s)
{
    Env<T> e = make_env<T>(c);
    for (int l = 0; l < kMaxLevels; ++l) { e.kdone[l] = L.kdone[l]; e.alpha[l] = (T)L.alpha[l]; }
    if (L.kind == Launch::FILL) {
        List li{c->tilelist.p + c->tile_off[L.level], c->tile_off[L.level + 1] - c->tile_off[L.level]};
        return launch_fill_tiles<T>(e, li, s);
    }
    if (L.kind == Launch::UPDATE) {
        List li = L.level < 0 ? List{nullptr, c->forest.n} : update_list(c, L);
        return launch_update<T>(e, li, L.ksub, L.fine_acc, variant_for(c, L.level), s);
    }
    List li = L.level < 0 ? List{c->cflist.p + c->cf_off[kMaxLevels], c->cf_off[kMaxLevels + 1] - c->cf_off[kMaxLevels]}
                          : List{c->cflist.p + c->cf_off[L.level], c->cf_off[L.level + 1] - c->cf_off[L.level]};
    return launch_reflux<T>(e, li, s);
}

// one step on the schedule's streams: the side streams fork from the context
// stream and join it again before the step control
template <typename T>
static int run_plan_t(fc_ctx *c)
{
    cudaStream_t s0 = c->stream;
    const int np = (int)c->plan.size(), ns = c->plan_nstreams;
    if (c->side.size() + 1 < (size_t)ns || c->sev.size() < (size_t)(np + ns)) {
        set_error("step schedule: streams and events not created");
        return FC_ERR_INVALID_ARG;
    }
    auto stream_of = [&](int k) { return k == 0 ? s0 : c->side[k - 1]; };
    if (ns > 1) {
        FC_CUDA(cudaEventRecord(c->sev[np], s0));
        for (int k = 1; k < ns; ++k) FC_CUDA(cudaStreamWaitEvent(c->side[k - 1], c->sev[np], 0));
    }
    for (int i = 0; i < np; ++i) {
        cudaStream_t s = stream_of(c->plan_stream[i]);
        for (int j : c->plan_waits[i]) FC_CUDA(cudaStreamWaitEvent(s, c->sev[j], 0));
        FC_TRY(launch_one<T>(c, c->plan[i], s));
        if (c->plan_signal[i]) FC_CUDA(cudaEventRecord(c->sev[i], s));
    }
    for (int k = 1; k < ns; ++k) {
        FC_CUDA(cudaEventRecord(c->sev[np + k], c->side[k - 1]));
        FC_CUDA(cudaStreamWaitEvent(s0, c->sev[np + k], 0));
    }
    return launch_step_ctl(c->d_ctl, c->lmin, c->lmax, c->p.subcycle, c->dx, c->nsub, s0);
}

static int run_plan(fc_ctx *c)
{
    return c->esize == 8 ? run_plan_t<double>(c) : run_plan_t<float>(c);
}

// one step eagerly, launch after launch in plan order on the context stream,
// with an event pair around every launch
template <typename T>
static int run_plan_profiled_t(fc_ctx *c, cudaEvent_t *ev, double *ms, int64_t *cnt, int64_t *cells)
{
    cudaStream_t s = c->stream;
    int m2 = c->p.m * c->p.m;
    auto timed = [&](int kind, auto &&fn, int64_t ncell) -> int {
        FC_CUDA(cudaEventRecord(ev[0], s));
        int rc = fn();
        if (rc) return rc;
        FC_CUDA(cudaEventRecord(ev[1], s));
        FC_CUDA(cudaEventSynchronize(ev[1]));
        float t = 0.f;
        FC_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1]));
        ms[kind] += t;
        cnt[kind] += 1;
        cells[kind] += ncell;
        return FC_OK;
    };
    for (const Launch &L : c->plan) {
        const int kind = L.kind == Launch::FILL ? 0 : L.kind == Launch::UPDATE ? 1 : 2;
        const int64_t ncell = kind != 1 ? 0 : (int64_t)(L.level < 0 ? c->forest.n : update_list(c, L).count) * m2;
        FC_TRY(timed(kind, [&] { return launch_one<T>(c, L, s); }, ncell));
    }
    return timed(3, [&] { return launch_step_ctl(c->d_ctl, c->lmin, c->lmax, c->p.subcycle, c->dx, c->nsub, s); }, 0);
}

// capture one step as a CUDA graph
static int ensure_graph(fc_ctx *c)
{
    if (c->plan_valid && c->gexec) return FC_OK;
    build_plan(c);
    // configure kernel attributes outside of capture
    for (int l = -1; l < kMaxLevels; ++l) {
        const int v = variant_for(c, l);
        if (c->esize == 8) { Env<double> e = make_env<double>(c); FC_TRY(launch_update<double>(e, List{nullptr, 0}, 1, 0, v, c->stream)); }
        else { Env<float> e = make_env<float>(c); FC_TRY(launch_update<float>(e, List{nullptr, 0}, 1, 0, v, c->stream)); }
    }
    FC_TRY(ensure_schedule_objects(c));
    FC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = run_plan(c);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
    // same launches in the same order (a regrid that keeps the levels and the
    // kinds of lists): update the executable graph's parameters in place
    if (c->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->gexec, g, &info) == cudaSuccess) {
            if (c->graph) cudaGraphDestroy(c->graph);
            c->graph = g;
            c->plan_valid = true;
            return FC_OK;
        }
        cudaGetLastError();                 // an update that does not apply is not an error
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph = g;
    FC_CUDA(cudaGraphInstantiate(&c->gexec, g, 0));
    c->plan_valid = true;
    return FC_OK;
}

template <typename T>
static int cell_dt_t(fc_ctx *c)
{
    if (!c->speeds_ready) {             // a pass over the cells of the current state
        Env<T> e = make_env<T>(c);
        FC_CUDA(cudaMemsetAsync(c->d_ctl->smax_bits, 0, sizeof(c->d_ctl->smax_bits), c->stream));
        FC_TRY(launch_cell_rate<T>(e, c->stream));
    }
    c->speeds_ready = false;
    return launch_dt_from_cells(c->d_ctl, c->lmin, c->lmax, c->p.subcycle, c->dx, c->stream);
}

static int pull_ctl(fc_ctx *c)
{
    FC_CUDA(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

static int push_ctl_field(fc_ctx *c, size_t off, const void *src, size_t n)
{
    // staged through pinned memory so the copy never blocks on pageable memory
    FC_CUDA(cudaStreamSynchronize(c->stream));
    memcpy(c->h_stage, src, n);
    FC_CUDA(cudaMemcpyAsync((char *)c->d_ctl + off, c->h_stage, n, cudaMemcpyHostToDevice, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

// before a batch of steps: graph, and the step size source if it changed
static int require_balanced(const fc_ctx *c)
{
    if (c->unbalanced) { set_error("forest is not 2:1 balanced; call fc_forest_balance"); return FC_ERR_UNBALANCED; }
    return FC_OK;
}

static int begin_advance(fc_ctx *c, double dt_fixed)
{
    FC_TRY(require_balanced(c));
    FC_TRY(ensure_graph(c));
    double df = dt_fixed > 0.0 ? dt_fixed : 0.0;
    if (df != c->cur_dt_fixed) {
        FC_TRY(push_ctl_field(c, offsetof(StepCtl, dt_fixed), &df, sizeof(double)));
        if (df > 0.0) FC_TRY(push_ctl_field(c, offsetof(StepCtl, dt), &df, sizeof(double)));
        else if (!c->dt_from_cells) FC_TRY(launch_dt_from_next(c->d_ctl, c->stream));
        c->cur_dt_fixed = df;
    }
    if (df == 0.0 && c->dt_from_cells) FC_TRY(c->esize == 8 ? cell_dt_t<double>(c) : cell_dt_t<float>(c));
    if (c->speeds_ready) {              // a fixed step did not use a written state's cell speeds
        FC_CUDA(cudaMemsetAsync(c->d_ctl->smax_bits, 0, sizeof(c->d_ctl->smax_bits), c->stream));
        c->speeds_ready = false;
    }
    c->dt_from_cells = false;
    // per-level steps of the first attempt (every step's control kernel sets
    // those of the next one)
    return launch_level_dt(c->d_ctl, c->lmin, c->lmax, c->p.subcycle, c->dx, c->stream);
}

// account steps accepted since the last call (h_ctl must be fresh)
static void account(fc_ctx *c)
{
    int d = c->h_ctl->accepted - c->acc_seen;
    c->acc_seen = c->h_ctl->accepted;
    c->cell_updates += (int64_t)d * c->updates_per_step;
    c->steps += d;
}

static int check_ctl(fc_ctx *c)
{
    if (c->h_ctl->dry_error) { set_error("depth h <= 0 met by the solver"); return FC_ERR_DRY_STATE; }
    if (c->h_ctl->nonfinite_error) { set_error("non-finite state"); return FC_ERR_NONFINITE; }
    if (c->h_ctl->index_error) { set_error("inconsistent neighbour data (index outside a patch)"); return FC_ERR_INVALID_ARG; }
    return FC_OK;
}

template <typename T>
static int tiles_now(fc_ctx *c, T *tiles, const int *slotmap, bool all_levels)
{
    // complete tiles at the current time, coarsest level first
    Env<T> e = make_env<T>(c);
    e.gr = tiles;
    e.grslot = slotmap;
    for (int l = c->lmin; l <= c->lmax; ++l) {
        List li = all_levels ? List{c->levlist.p + c->lev_off[l], c->lev_off[l + 1] - c->lev_off[l]}
                             : List{c->tilelist.p + c->tile_off[l], c->tile_off[l + 1] - c->tile_off[l]};
        FC_TRY(launch_fill_tiles<T>(e, li, c->stream));
    }
    return FC_OK;
}

template <typename T>
static int export_t(fc_ctx *c, float *d_dst, const double *xf)
{
    int n = c->forest.n, S = c->p.m + 4;
    DBuf<unsigned char> tiles;
    FC_TRY(tiles.alloc((size_t)n * 3 * S * S * sizeof(T), c->stream));
    FC_TRY(tiles_now<T>(c, (T *)tiles.p, c->iota.p, true));
    k_tiles_to_input<T><<<nb256((long long)n * 3 * S * S), 256, 0, c->stream>>>((const T *)tiles.p, n, S * S, xf[0],
                                                                                  xf[1], xf[2], xf[3], d_dst);
    FC_CUDA(cudaGetLastError());
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

template <typename T>
static int tag_t(fc_ctx *c, int8_t *h_flags, bool learned)
{
    int n = c->forest.n;
    FC_TRY(c->flags.alloc(n, c->stream));
    FC_TRY(tiles_now<T>(c, (T *)c->gr.p, c->grslot.p, false));
    Env<T> e = make_env<T>(c);
    FC_TRY(launch_tag<T>(e, c->p.tag_crit, c->p.tag_threshold, c->p.min_level, c->flags.p, c->stream));
    if (learned) {
        int S = c->p.m + 4;
        FC_TRY(c->tag_x.alloc((size_t)n * 3 * S * S, c->stream));
        FC_TRY(c->tag_logits.alloc((size_t)n * 2, c->stream));
        FC_TRY(export_t<T>(c, c->tag_x.p, c->tag_xform));
        FC_TRY(fc_cnn_forward(n, S, c->tag_w.p, c->tag_x.p, c->tag_logits.p, c->tag_bf16, c->stream));
        k_combine_flags<<<nb256(n), 256, 0, c->stream>>>(c->flags.p, c->tag_logits.p, n);
        FC_CUDA(cudaGetLastError());
    }
    FC_CUDA(cudaMemcpyAsync(h_flags, c->flags.p, n, cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

template <typename T>
static int regrid_t(fc_ctx *c, const int8_t *h_flags)
{
    cudaStream_t s = c->stream;
    int nold = c->forest.n, m = c->p.m, F = c->F;
    size_t PP = (size_t)(m + 4) * (m + 4);
    // complete tiles of every old leaf (sources of interpolation)
    DBuf<unsigned char> tiles;
    FC_TRY(tiles.alloc((size_t)nold * F * PP * sizeof(T), s));
    FC_TRY(tiles_now<T>(c, (T *)tiles.p, c->iota.p, true));
    // keep the old forest and state
    DBuf<int> olev, ox, oy;
    FC_TRY(olev.alloc(nold, s)); FC_TRY(ox.alloc(nold, s)); FC_TRY(oy.alloc(nold, s));
    FC_CUDA(cudaMemcpyAsync(olev.p, c->forest.level.p, nold * sizeof(int), cudaMemcpyDeviceToDevice, s));
    FC_CUDA(cudaMemcpyAsync(ox.p, c->forest.x.p, nold * sizeof(int), cudaMemcpyDeviceToDevice, s));
    FC_CUDA(cudaMemcpyAsync(oy.p, c->forest.y.p, nold * sizeof(int), cudaMemcpyDeviceToDevice, s));
    Env<T> eo = make_env<T>(c);
    eo.f.level = olev.p;
    DBuf<unsigned char> oq[3], ogeo;
    for (int b = 0; b < 3; ++b) oq[b].swap(c->q[b]);
    for (int b = 0; b < 3; ++b) eo.q[b] = (T *)oq[b].p;
    ogeo.swap(c->geo);                   // the old leaves' geometry (cubed sphere)
    eo.geo = (const T *)ogeo.p;
    // new topology
    FC_TRY(c->flags.alloc(nold, s));
    FC_CUDA(cudaMemcpyAsync(c->flags.p, h_flags, nold, cudaMemcpyHostToDevice, s));
    DBuf<int> origin;
    int rc = c->forest.adapt(c->flags.p, c->p.min_level, c->p.max_level, &origin);
    if (rc) return rc;
    FC_TRY(prepare(c, false));
    Env<T> en = make_env<T>(c);
    FC_TRY(launch_transfer<T>(eo, en, origin.p, (const T *)tiles.p, ox.p, oy.p, s));
    FC_TRY(reset_ctl_buffers(c));
    FC_CUDA(cudaStreamSynchronize(s));
    c->dt_from_cells = true;
    c->speeds_ready = false;
    c->regrids += 1;
    return FC_OK;
}

// time the fused-update variants on every level's patch list of this
// context's forest and keep the fastest per level (a launch over all levels,
// under one global dt, takes the choice of the level with the most
// patches); the trial launches write only a scratch state buffer
template <typename T>
static int autotune_t(fc_ctx *c, double *ms_out)
{
    cudaStream_t s = c->stream;
    int lv = c->lmin;
    for (int l = c->lmin; l <= c->lmax; ++l)
        if (c->lev_off[l + 1] - c->lev_off[l] > c->lev_off[lv + 1] - c->lev_off[lv]) lv = l;
    Env<T> e = make_env<T>(c);
    cudaEvent_t ev[2];
    FC_CUDA(cudaEventCreate(&ev[0]));
    FC_CUDA(cudaEventCreate(&ev[1]));
    FC_TRY(launch_level_dt(c->d_ctl, c->lmin, c->lmax, c->p.subcycle, c->dx, s));
    // complete tiles of the coarse sources at the current time, coarsest
    // level first, so that the trials read valid ghost values
    for (int l = c->lmin; l <= c->lmax; ++l)
        FC_TRY(launch_fill_tiles<T>(e, List{c->tilelist.p + c->tile_off[l], c->tile_off[l + 1] - c->tile_off[l]}, s));
    const int nvar = fc::update_variant_count(c->p.equation, fc::has_geometry(c) ? FC_CONN_SPHERE : c->p.conn, c->p.transverse == 2, c->p.entropy_fix);
    for (int v = 0; v < kUpdateVariants; ++v)
        if (ms_out) ms_out[v] = -1.0;
    int best_lv[kMaxLevels];
    for (int l = 0; l < kMaxLevels; ++l) best_lv[l] = -1;
    for (int l = c->lmin; l <= c->lmax; ++l) {
        List li{c->levlist.p + c->lev_off[l], c->lev_off[l + 1] - c->lev_off[l]};
        if (li.count <= 0) continue;
        double bestms = 1e30;
        for (int v = 0; v < nvar; ++v) {
            FC_TRY(launch_update<T>(e, li, 1, 0, v, s));          // warm
            FC_CUDA(cudaEventRecord(ev[0], s));
            for (int r = 0; r < 5; ++r) FC_TRY(launch_update<T>(e, li, 1, 0, v, s));
            FC_CUDA(cudaEventRecord(ev[1], s));
            FC_CUDA(cudaEventSynchronize(ev[1]));
            float ms = 0.f;
            FC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            if (l == lv && ms_out) ms_out[v] = ms / 5.0;
            if (ms < bestms) { bestms = ms; best_lv[l] = v; }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    // the trials folded their wave speeds into the CFL maxima: clear them
    FC_CUDA(cudaMemsetAsync(c->d_ctl->smax_bits, 0, sizeof(c->d_ctl->smax_bits), s));
    FC_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < kMaxLevels; ++l) c->upd_variant_lv[l] = best_lv[l];
    if (best_lv[lv] >= 0) c->upd_variant = best_lv[lv];
    invalidate_plan(c);
    return FC_OK;
}

}  // namespace fc

// ===========================================================================
// C ABI
// ===========================================================================
// a table connectivity carries a forest only: the calls that need fields refuse it
static int forest_only(const fc_ctx *c, const char *what)
{
    if (c->p.conn != FC_CONN_TABLE) return FC_OK;
    set_error("%s: a table connectivity carries a forest only (no fields)", what);
    return FC_ERR_UNIMPLEMENTED;
}

extern "C" {

const char *fc_last_error(void) { return fc::g_msg; }

int fc_create(const fc_params *p, fc_ctx **out)
{
    if (!p || !out) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!(p->m == 8 || p->m == 16 || p->m == 32) || p->min_level < 0 || p->max_level < p->min_level ||
        p->max_level > 14 || (p->equation != FC_EQ_SWE && p->equation != FC_EQ_ADV) ||
        (p->precision != FC_FP64 && p->precision != FC_FP32) || !(p->cfl > 0.0) ||
        (p->conn != FC_CONN_SQUARE && p->conn != FC_CONN_PERIODIC && p->conn != FC_CONN_SPHERE &&
         p->conn != FC_CONN_PILLOW && p->conn != FC_CONN_TABLE)) {
        set_error("invalid parameters");
        return FC_ERR_INVALID_ARG;
    }
    if (fc::is_sphere_conn(p->conn) && p->equation != FC_EQ_ADV) {
        set_error("the spheres carry scalar advection (FC_EQ_ADV)");
        return FC_ERR_INVALID_ARG;
    }
    if (p->transverse < 0 || p->transverse > 2 || p->entropy_fix < 0 || p->entropy_fix > 1) {
        set_error("transverse must be 0, 1 or 2 and entropy_fix 0 or 1");
        return FC_ERR_INVALID_ARG;
    }
    if (p->velocity != FC_VEL_CONSTANT && p->velocity != FC_VEL_SWIRL) {
        set_error("velocity must be FC_VEL_CONSTANT or FC_VEL_SWIRL");
        return FC_ERR_INVALID_ARG;
    }
    if (p->velocity == FC_VEL_SWIRL && (p->equation != FC_EQ_ADV || fc::is_sphere_conn(p->conn) || p->transverse == 2)) {
        set_error("the swirl is an advection velocity on the square (T1 transverse terms)");
        return FC_ERR_INVALID_ARG;
    }
    if (p->conn == FC_CONN_TABLE && p->velocity != FC_VEL_CONSTANT) {
        set_error("a table connectivity carries a forest only");
        return FC_ERR_INVALID_ARG;
    }
    if (p->transverse == 2 && fc::is_sphere_conn(p->conn)) {
        set_error("the T2 transverse variant is for the square and the periodic square");
        return FC_ERR_UNIMPLEMENTED;
    }
    if (p->equation == FC_EQ_SWE && p->m == 32 && p->precision == FC_FP64) {
        set_error("m = 32 shallow water needs FC_FP32 (shared memory)");
        return FC_ERR_UNIMPLEMENTED;
    }
    fc_ctx *c = new fc_ctx();
    for (int l = 0; l < fc::kMaxLevels; ++l) c->upd_variant_lv[l] = -1;
    c->p = *p;
    c->F = p->equation == FC_EQ_SWE ? 3 : 1;
    c->esize = p->precision == FC_FP64 ? 8 : 4;
    int rc = FC_OK;
    if (p->device >= 0) {
        cudaError_t e = cudaSetDevice(p->device);
        if (e != cudaSuccess) { delete c; return cuda_status(e, "cudaSetDevice"); }
    }
    cudaGetDevice(&c->device);
    if (p->stream) c->stream = (cudaStream_t)p->stream;
    else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return cuda_status(e, "cudaStreamCreate"); }
        c->own_stream = true;
    }
    c->forest.stream = c->stream;
    c->forest.conn = p->conn;
    if (cudaMalloc(&c->d_ctl, sizeof(StepCtl)) != cudaSuccess ||
        cudaMallocHost(&c->h_ctl, sizeof(StepCtl)) != cudaSuccess ||
        cudaMallocHost(&c->h_stage, 64) != cudaSuccess) {
        delete c;
        return cuda_status(cudaGetLastError(), "step control allocation");
    }
    memset(c->h_ctl, 0, sizeof(StepCtl));
    c->h_ctl->cfl = p->cfl;
    cudaMemcpy(c->d_ctl, c->h_ctl, sizeof(StepCtl), cudaMemcpyHostToDevice);
    if (p->conn == FC_CONN_TABLE) {
        // one tree bounded on every side until fc_set_connectivity
        const int32_t walls[12] = {-1, 0, 0, -1, 0, 0, -1, 0, 0, -1, 0, 0};
        rc = c->forest.ctab.alloc(12, c->stream);
        if (!rc && cudaMemcpyAsync(c->forest.ctab.p, walls, sizeof walls, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            rc = cuda_status(cudaGetLastError(), "connectivity table");
        if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = cuda_status(cudaGetLastError(), "connectivity table");
        if (rc) { fc_destroy(c); return rc; }
        c->forest.ntab = 1;
    }
    rc = c->forest.uniform(p->min_level);
    if (!rc) rc = prepare(c, true);
    if (rc) { fc_destroy(c); return rc; }
    *out = c;
    return FC_OK;
}

void fc_destroy(fc_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (cudaStream_t st : c->side) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (cudaEvent_t ev : c->sev) cudaEventDestroy(ev);
    fc::release_graph(c);
    if (c->d_ctl) cudaFree(c->d_ctl);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    cudaStream_t s = c->stream;
    bool own = c->own_stream;
    delete c;      // DBuf destructors free asynchronously on s
    cudaStreamSynchronize(s);
    if (own) cudaStreamDestroy(s);
}

int fc_forest_uniform(fc_ctx *c, int level)
{
    if (!c) return FC_ERR_INVALID_ARG;
    FC_TRY(c->forest.uniform(level));
    c->unbalanced = false;
    FC_TRY(fc::prepare(c, true));
    FC_TRY(fc::reset_ctl_buffers(c));
    c->dt_from_cells = true;
    c->speeds_ready = false;
    return FC_OK;
}

int fc_set_connectivity(fc_ctx *c, int ntrees, const int32_t *table)
{
    if (!c || !table || c->p.conn != FC_CONN_TABLE || ntrees < 1 || ntrees > FC_MAX_TREES) {
        set_error("fc_set_connectivity: needs a FC_CONN_TABLE context and 1..%d trees", FC_MAX_TREES);
        return FC_ERR_INVALID_ARG;
    }
    for (int k = 0; k < ntrees * 4; ++k) {
        const int32_t *e = table + 3 * k;
        if (e[0] < -1 || e[0] >= ntrees || (e[0] >= 0 && (e[1] < 0 || e[1] > 3 || e[2] < 0 || e[2] > 1))) {
            set_error("fc_set_connectivity: bad entry for tree %d side %d", k / 4, k % 4);
            return FC_ERR_INVALID_ARG;
        }
    }
    FC_TRY(c->forest.ctab.alloc((size_t)ntrees * 12, c->stream));
    FC_CUDA(cudaMemcpyAsync(c->forest.ctab.p, table, sizeof(int32_t) * 12 * (size_t)ntrees, cudaMemcpyHostToDevice,
                            c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));       // the caller's table may go once this returns
    c->forest.ntab = ntrees;
    return fc_forest_uniform(c, c->p.min_level);
}

int fc_forest_set_leaves(fc_ctx *c, int64_t n, const int32_t *tree, const int32_t *level, const int32_t *x,
                         const int32_t *y)
{
    if (!c || !tree || !level || !x || !y) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    FC_TRY(c->forest.set_leaves(n, tree, level, x, y));
    int rc = c->forest.rebuild_tables();
    if (rc && rc != FC_ERR_UNBALANCED) return rc;
    c->unbalanced = rc == FC_ERR_UNBALANCED;
    FC_TRY(fc::prepare(c, true));
    FC_TRY(fc::reset_ctl_buffers(c));
    c->dt_from_cells = true;
    c->speeds_ready = false;
    return FC_OK;
}

int fc_forest_num_leaves(const fc_ctx *c, int64_t *n)
{
    if (!c || !n) return FC_ERR_INVALID_ARG;
    *n = c->forest.n;
    return FC_OK;
}

int fc_forest_get_leaves(const fc_ctx *c, int32_t *tree, int32_t *level, int32_t *x, int32_t *y, int64_t cap)
{
    if (!c) return FC_ERR_INVALID_ARG;
    if (cap < c->forest.n) { set_error("capacity %lld < %d leaves", (long long)cap, c->forest.n); return FC_ERR_CAPACITY; }
    std::vector<int> t, l, xx, yy;
    FC_TRY(c->forest.download(t, l, xx, yy));
    for (int i = 0; i < c->forest.n; ++i) {
        if (tree) tree[i] = t[i];
        if (level) level[i] = l[i];
        if (x) x[i] = xx[i];
        if (y) y[i] = yy[i];
    }
    return FC_OK;
}

int fc_forest_get_neighbors(const fc_ctx *c, int32_t *table, int64_t cap)
{
    if (!c || !table) return FC_ERR_INVALID_ARG;
    if (cap < (int64_t)c->forest.n * 32) { set_error("capacity too small"); return FC_ERR_CAPACITY; }
    FC_CUDA(cudaMemcpyAsync(table, c->forest.nbr.p, sizeof(int) * 32 * (size_t)c->forest.n,
                            cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

int fc_forest_balance(fc_ctx *c)
{
    if (!c) return FC_ERR_INVALID_ARG;
    FC_TRY(c->forest.balance(nullptr));
    c->unbalanced = false;
    FC_TRY(fc::prepare(c, true));
    FC_TRY(fc::reset_ctl_buffers(c));
    c->dt_from_cells = true;
    c->speeds_ready = false;
    return FC_OK;
}

int fc_num_fields(const fc_ctx *c) { return c ? c->F : 0; }

int fc_set_initial(fc_ctx *c, int kind, const double *p, int np)
{
    if (!c || !p || np < 0 || np > 4096) { set_error("bad initial-condition arguments"); return FC_ERR_INVALID_ARG; }
    FC_TRY(forest_only(c, "fc_set_initial"));
    bool swe = c->p.equation == FC_EQ_SWE;
    bool sph = fc::is_sphere_conn(c->p.conn);
    bool ok = swe ? ((kind == FC_INIT_DAMBREAK && np >= 5) || (kind == FC_INIT_HUMPS && np >= 1 && (np - 1) % 4 == 0))
                  : sph ? ((kind == FC_INIT_HILL && np >= 3) || (kind == FC_INIT_HALF && np >= 2))
                        : ((kind == FC_INIT_ADV_BOX && np >= 6) || (kind == FC_INIT_ADV_SINE && np >= 4));
    if (!ok) { set_error("initial condition %d does not fit the equation", kind); return FC_ERR_INVALID_ARG; }
    FC_TRY(fc::clear_errors(c));
    FC_TRY(c->dparams.alloc(np + 1, c->stream));
    FC_CUDA(cudaMemcpyAsync(c->dparams.p, p, np * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->esize == 8) { Env<double> e = fc::make_env<double>(c); FC_TRY(fc::launch_init<double>(e, kind, c->dparams.p, np, c->stream)); }
    else { Env<float> e = fc::make_env<float>(c); FC_TRY(fc::launch_init<float>(e, kind, c->dparams.p, np, c->stream)); }
    FC_CUDA(cudaStreamSynchronize(c->stream));
    c->dt_from_cells = true;
    c->speeds_ready = false;
    return FC_OK;
}

int fc_tag(fc_ctx *c, int8_t *flags_out, int tagger)
{
    fc::Range nvtx_range("fc_tag");
    if (!c || !flags_out) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_tag"));
    if (tagger != FC_TAGGER_PLAIN && tagger != FC_TAGGER_LEARNED) { set_error("unknown tagger"); return FC_ERR_INVALID_ARG; }
    bool learned = tagger == FC_TAGGER_LEARNED;
    if (learned && (!c->tag_ready || c->p.equation != FC_EQ_SWE)) {
        set_error("learned tagger needs fc_set_tagger and shallow water");
        return FC_ERR_INVALID_ARG;
    }
    FC_TRY(fc::require_balanced(c));
    return c->esize == 8 ? fc::tag_t<double>(c, flags_out, learned) : fc::tag_t<float>(c, flags_out, learned);
}

int fc_export_tiles(fc_ctx *c, float *dst, int64_t cap, const double *xform, int dst_is_device)
{
    if (!c || !dst || !xform) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_export_tiles"));
    if (c->p.equation != FC_EQ_SWE) { set_error("tile export needs shallow water"); return FC_ERR_INVALID_ARG; }
    FC_TRY(fc::require_balanced(c));
    int S = c->p.m + 4;
    size_t need = (size_t)c->forest.n * 3 * S * S;
    if ((size_t)cap < need) { set_error("capacity %lld < %zu floats", (long long)cap, need); return FC_ERR_CAPACITY; }
    float *tgt = dst;
    DBuf<float> tmp;
    if (!dst_is_device) { FC_TRY(tmp.alloc(need, c->stream)); tgt = tmp.p; }
    FC_TRY(c->esize == 8 ? fc::export_t<double>(c, tgt, xform) : fc::export_t<float>(c, tgt, xform));
    if (!dst_is_device) {
        FC_CUDA(cudaMemcpyAsync(dst, tmp.p, need * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        FC_CUDA(cudaStreamSynchronize(c->stream));
    }
    return FC_OK;
}

int fc_set_tagger(fc_ctx *c, const float *w, const double *xform, int bf16)
{
    if (!c || !w || !xform) return FC_ERR_INVALID_ARG;
    FC_TRY(c->tag_w.alloc(3058, c->stream));
    FC_CUDA(cudaMemcpyAsync(c->tag_w.p, w, 3058 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 4; ++k) c->tag_xform[k] = xform[k];
    c->tag_bf16 = bf16 ? 1 : 0;
    c->tag_ready = true;
    return FC_OK;
}

int fc_regrid(fc_ctx *c, const int8_t *flags)
{
    fc::Range nvtx_range("fc_regrid");
    if (!c || !flags) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_regrid"));
    FC_TRY(fc::require_balanced(c));
    return c->esize == 8 ? fc::regrid_t<double>(c, flags) : fc::regrid_t<float>(c, flags);
}

int fc_init_refine(fc_ctx *c, int kind, const double *p, int np)
{
    fc::Range nvtx_range("fc_init_refine");
    if (!c) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_init_refine"));
    FC_TRY(fc_forest_uniform(c, c->p.min_level));
    for (int r = 0; r < c->p.max_level - c->p.min_level; ++r) {
        FC_TRY(fc_set_initial(c, kind, p, np));
        std::vector<int8_t> fl(c->forest.n);
        FC_TRY(fc_tag(c, fl.data(), FC_TAGGER_PLAIN));
        for (auto &v : fl) if (v < 0) v = 0;
        FC_TRY(c->flags.alloc(fl.size(), c->stream));
        FC_CUDA(cudaMemcpyAsync(c->flags.p, fl.data(), fl.size(), cudaMemcpyHostToDevice, c->stream));
        DBuf<int> origin;
        FC_TRY(c->forest.adapt(c->flags.p, c->p.min_level, c->p.max_level, &origin));
        FC_TRY(fc::prepare(c, true));
        FC_TRY(fc::reset_ctl_buffers(c));
    }
    FC_TRY(fc_set_initial(c, kind, p, np));
    return FC_OK;
}

}  // extern "C"

// field transfers in the caller's layout [leaf][field][j][i]; with wait, the
// call returns after the stream finished them, else they stay enqueued
// (page-locked or device buffers only)
static int read_fields(fc_ctx *c, int field, void *dst, int64_t cap_bytes, int dst_is_device, bool wait)
{
    if (!c || !dst || field < -1 || field >= c->F) return FC_ERR_INVALID_ARG;
    size_t nf = field < 0 ? c->F : 1;
    size_t bytes = nf * (size_t)c->forest.n * c->p.m * c->p.m * c->esize;
    if ((size_t)cap_bytes < bytes) { set_error("capacity %lld < %zu bytes", (long long)cap_bytes, bytes); return FC_ERR_CAPACITY; }
    // host buffers: the layout kernel writes a device staging buffer and the
    // copy engines move it over the host link (no SM waits on the link, so
    // another context's kernels keep the SMs meanwhile)
    void *tgt = dst;
    bool staged = false;
    if (!dst_is_device) {
        if (!wait && !fc::pinned_device_pointer(dst)) {
            set_error("asynchronous transfers need page-locked host memory");
            return FC_ERR_INVALID_ARG;
        }
        FC_TRY(c->io.alloc(bytes, c->stream));
        tgt = c->io.p;
        staged = true;
    }
    if (c->esize == 8) { Env<double> e = fc::make_env<double>(c); FC_TRY(fc::launch_read<double>(e, field, (double *)tgt, c->stream)); }
    else { Env<float> e = fc::make_env<float>(c); FC_TRY(fc::launch_read<float>(e, field, (float *)tgt, c->stream)); }
    if (staged) FC_CUDA(cudaMemcpyAsync(dst, c->io.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (wait) FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

static int write_fields(fc_ctx *c, const void *src, int64_t nbytes, int src_is_device, bool wait)
{
    if (!c || !src) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_write_fields"));
    size_t bytes = (size_t)c->F * c->forest.n * c->p.m * c->p.m * c->esize;
    if ((size_t)nbytes != bytes) { set_error("expected %zu bytes", bytes); return FC_ERR_INVALID_ARG; }
    // host buffers: copy engines into a device staging buffer, then the
    // layout kernel from device memory
    const void *from = src;
    if (!src_is_device) {
        if (!wait && !fc::pinned_device_pointer(src)) {
            set_error("asynchronous transfers need page-locked host memory");
            return FC_ERR_INVALID_ARG;
        }
        FC_TRY(c->io.alloc(bytes, c->stream));
        FC_CUDA(cudaMemcpyAsync(c->io.p, src, bytes, cudaMemcpyHostToDevice, c->stream));
        from = c->io.p;
    }
    FC_TRY(fc::clear_errors(c));
    // shallow water: the write also leaves the new state's cell-speed maxima
    // in the step control for the next step's size
    const bool swe = c->F == 3;
    if (swe) FC_CUDA(cudaMemsetAsync(c->d_ctl->smax_bits, 0, sizeof(c->d_ctl->smax_bits), c->stream));
    if (c->esize == 8) {
        Env<double> e = fc::make_env<double>(c);
        FC_TRY(swe ? fc::launch_write_speed<double>(e, (const double *)from, c->stream)
                   : fc::launch_write<double>(e, (const double *)from, c->stream));
    } else {
        Env<float> e = fc::make_env<float>(c);
        FC_TRY(swe ? fc::launch_write_speed<float>(e, (const float *)from, c->stream)
                   : fc::launch_write<float>(e, (const float *)from, c->stream));
    }
    if (wait) FC_CUDA(cudaStreamSynchronize(c->stream));
    c->dt_from_cells = true;
    c->speeds_ready = swe;
    return FC_OK;
}

extern "C" {

int fc_read_fields(const fc_ctx *cc, int field, void *dst, int64_t cap_bytes, int dst_is_device)
{
    return read_fields(const_cast<fc_ctx *>(cc), field, dst, cap_bytes, dst_is_device, true);
}

int fc_read_fields_async(const fc_ctx *cc, int field, void *dst, int64_t cap_bytes, int dst_is_device)
{
    return read_fields(const_cast<fc_ctx *>(cc), field, dst, cap_bytes, dst_is_device, false);
}

int fc_write_fields(fc_ctx *c, const void *src, int64_t nbytes, int src_is_device)
{
    return write_fields(c, src, nbytes, src_is_device, true);
}

int fc_write_fields_async(fc_ctx *c, const void *src, int64_t nbytes, int src_is_device)
{
    return write_fields(c, src, nbytes, src_is_device, false);
}

int fc_conservation_sums(const fc_ctx *cc, double *sums)
{
    fc_ctx *c = const_cast<fc_ctx *>(cc);
    if (!c || !sums) return FC_ERR_INVALID_ARG;
    FC_TRY(c->part.alloc((size_t)c->forest.n * c->F, c->stream));
    FC_TRY(c->sums.alloc(c->F, c->stream));
    if (c->esize == 8) { Env<double> e = fc::make_env<double>(c); FC_TRY(fc::launch_sums<double>(e, c->part.p, c->sums.p, c->stream)); }
    else { Env<float> e = fc::make_env<float>(c); FC_TRY(fc::launch_sums<float>(e, c->part.p, c->sums.p, c->stream)); }
    FC_CUDA(cudaMemcpyAsync(sums, c->sums.p, c->F * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

int fc_advance_async(fc_ctx *c, double dt_fixed, int nsteps)
{
    fc::Range nvtx_range("fc_advance_async");
    if (!c || nsteps < 0) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_advance_async"));
    if (nsteps == 0) return FC_OK;
    FC_TRY(fc::begin_advance(c, dt_fixed));
    for (int i = 0; i < nsteps; ++i) FC_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    return FC_OK;
}

int fc_sync(fc_ctx *c)
{
    if (!c) return FC_ERR_INVALID_ARG;
    FC_TRY(fc::pull_ctl(c));
    fc::account(c);
    FC_TRY(fc::check_ctl(c));
    if (c->h_ctl->cfl_error) { set_error("Courant number above 1 (a fixed step, or three retakes)"); return FC_ERR_CFL_VIOLATION; }
    return FC_OK;
}

int fc_advance(fc_ctx *c, double dt_fixed, int nsteps, double *t_out, double *dt_out)
{
    fc::Range nvtx_range("fc_advance");
    if (!c || nsteps < 0) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_advance"));
    FC_TRY(fc::pull_ctl(c));
    fc::account(c);
    if (nsteps > 0) {
        FC_TRY(fc::begin_advance(c, dt_fixed));
        int base = c->h_ctl->accepted, done = 0;
        for (int guard = 0; done < nsteps && guard < 64; ++guard) {
            for (int i = done; i < nsteps; ++i) FC_CUDA(cudaGraphLaunch(c->gexec, c->stream));
            FC_TRY(fc::pull_ctl(c));
            FC_TRY(fc::check_ctl(c));
            done = c->h_ctl->accepted - base;
        }
        fc::account(c);
    }
    if (t_out) *t_out = c->h_ctl->t;
    if (dt_out) *dt_out = c->h_ctl->last_dt;
    if (c->h_ctl->cfl_error) { set_error("Courant number above 1 (a fixed step, or three retakes)"); return FC_ERR_CFL_VIOLATION; }
    return FC_OK;
}

int fc_profile_steps(fc_ctx *c, double dt_fixed, int nsteps, double *ms, int64_t *cnt, int64_t *cells)
{
    if (!c || nsteps < 0 || !ms || !cnt || !cells) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_profile_steps"));
    for (int k = 0; k < 4; ++k) { ms[k] = 0.0; cnt[k] = 0; cells[k] = 0; }
    if (nsteps == 0) return FC_OK;
    FC_TRY(fc::begin_advance(c, dt_fixed));
    cudaEvent_t ev[2];
    FC_CUDA(cudaEventCreate(&ev[0]));
    FC_CUDA(cudaEventCreate(&ev[1]));
    int rc = FC_OK;
    for (int i = 0; i < nsteps && !rc; ++i)
        rc = c->esize == 8 ? fc::run_plan_profiled_t<double>(c, ev, ms, cnt, cells)
                           : fc::run_plan_profiled_t<float>(c, ev, ms, cnt, cells);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    return fc_sync(c);
}

int fc_set_step_streams(fc_ctx *c, int nstreams)
{
    if (!c || nstreams < 1 || nstreams > FC_MAX_STEP_STREAMS) {
        set_error("step streams must be 1..%d", FC_MAX_STEP_STREAMS);
        return FC_ERR_INVALID_ARG;
    }
    c->step_streams = nstreams;
    fc::invalidate_plan(c);
    return FC_OK;
}

int fc_step_schedule(fc_ctx *c, int *launches, int *streams, int *chain)
{
    if (!c || !launches || !streams || !chain) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_step_schedule"));
    if (!c->plan_valid) fc::build_plan(c);
    *launches = (int)c->plan.size() + 1;
    *streams = c->plan_nstreams;
    *chain = c->plan_chain;
    return FC_OK;
}

int fc_set_variant(fc_ctx *c, int variant)
{
    if (!c) return FC_ERR_INVALID_ARG;
    int nvar = fc::update_variant_count(c->p.equation, fc::has_geometry(c) ? FC_CONN_SPHERE : c->p.conn, c->p.transverse == 2, c->p.entropy_fix);
    if (variant < 0 || variant >= nvar) { set_error("launch variant %d not available", variant); return FC_ERR_INVALID_ARG; }
    c->upd_variant = variant;
    for (int l = 0; l < fc::kMaxLevels; ++l) c->upd_variant_lv[l] = -1;
    fc::invalidate_plan(c);
    return FC_OK;
}

int fc_autotune(fc_ctx *c, int *variant_out, double *ms_by_variant)
{
    fc::Range nvtx_range("fc_autotune");
    if (!c) return FC_ERR_INVALID_ARG;
    FC_TRY(forest_only(c, "fc_autotune"));
    FC_TRY(fc::begin_advance(c, c->cur_dt_fixed > 0.0 ? c->cur_dt_fixed : 0.0));
    FC_TRY(c->esize == 8 ? fc::autotune_t<double>(c, ms_by_variant) : fc::autotune_t<float>(c, ms_by_variant));
    if (variant_out) *variant_out = c->upd_variant;
    return FC_OK;
}

int fc_stats(const fc_ctx *cc, fc_stats_t *st)
{
    fc_ctx *c = const_cast<fc_ctx *>(cc);
    if (!c || !st) return FC_ERR_INVALID_ARG;
    FC_TRY(fc::pull_ctl(c));
    memset(st, 0, sizeof *st);
    st->num_leaves = c->forest.n;
    for (int l = 0; l < 16; ++l) st->leaves_per_level[l] = c->lev_off[l + 1] - c->lev_off[l];
    st->cell_updates = c->cell_updates;
    st->steps = c->steps;
    st->retries = c->h_ctl->retries;
    st->regrids = c->regrids;
    st->time = c->h_ctl->t;
    st->last_dt = c->h_ctl->last_dt;
    st->last_courant = c->h_ctl->last_courant;
    st->next_dt = c->h_ctl->next_dt;
    return FC_OK;
}

// checkpoint: header, leaves, fields in the context precision
struct CkptHeader {
    char magic[8];
    int32_t version, conn, m, equation, precision, F;
    int64_t n;
    double t, next_dt;
    int32_t dt_from_cells, pad;
};

int fc_save(const fc_ctx *cc, const char *path)
{
    fc_ctx *c = const_cast<fc_ctx *>(cc);
    if (!c || !path) return FC_ERR_INVALID_ARG;
    FC_TRY(fc::pull_ctl(c));
    std::vector<int> t, l, x, y;
    FC_TRY(c->forest.download(t, l, x, y));
    size_t bytes = (size_t)c->F * c->forest.n * c->p.m * c->p.m * c->esize;
    std::vector<unsigned char> q(bytes);
    FC_TRY(fc_read_fields(c, -1, q.data(), (int64_t)bytes, 0));
    CkptHeader h{};
    memcpy(h.magic, "FCGB300", 8);
    h.version = 1; h.conn = c->p.conn; h.m = c->p.m; h.equation = c->p.equation; h.precision = c->p.precision;
    h.F = c->F; h.n = c->forest.n; h.t = c->h_ctl->t; h.next_dt = c->h_ctl->dt;
    h.dt_from_cells = c->dt_from_cells;
    FILE *fp = fopen(path, "wb");
    if (!fp) { set_error("cannot open %s", path); return FC_ERR_INVALID_ARG; }
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1;
    for (auto *v : {&t, &l, &x, &y}) ok = ok && fwrite(v->data(), sizeof(int), v->size(), fp) == v->size();
    ok = ok && fwrite(q.data(), 1, bytes, fp) == bytes;
    fclose(fp);
    if (!ok) { set_error("short write to %s", path); return FC_ERR_INVALID_ARG; }
    return FC_OK;
}

int fc_load(fc_ctx *c, const char *path)
{
    if (!c || !path) return FC_ERR_INVALID_ARG;
    FILE *fp = fopen(path, "rb");
    if (!fp) { set_error("cannot open %s", path); return FC_ERR_INVALID_ARG; }
    CkptHeader h{};
    bool ok = fread(&h, sizeof h, 1, fp) == 1 && memcmp(h.magic, "FCGB300", 8) == 0 && h.conn == c->p.conn &&
              h.m == c->p.m && h.equation == c->p.equation && h.precision == c->p.precision && h.F == c->F &&
              h.n > 0 && h.n < (1 << 26);
    if (!ok) { fclose(fp); set_error("checkpoint %s does not match this context", path); return FC_ERR_INVALID_ARG; }
    std::vector<int> t(h.n), l(h.n), x(h.n), y(h.n);
    for (auto *v : {&t, &l, &x, &y}) ok = ok && fread(v->data(), sizeof(int), v->size(), fp) == v->size();
    size_t bytes = (size_t)c->F * h.n * c->p.m * c->p.m * c->esize;
    std::vector<unsigned char> q(bytes);
    ok = ok && fread(q.data(), 1, bytes, fp) == bytes;
    fclose(fp);
    if (!ok) { set_error("short checkpoint %s", path); return FC_ERR_INVALID_ARG; }
    FC_TRY(fc_forest_set_leaves(c, h.n, t.data(), l.data(), x.data(), y.data()));
    FC_TRY(fc_write_fields(c, q.data(), (int64_t)bytes, 0));
    FC_TRY(fc::push_ctl_field(c, offsetof(StepCtl, t), &h.t, sizeof(double)));
    FC_TRY(fc::push_ctl_field(c, offsetof(StepCtl, dt), &h.next_dt, sizeof(double)));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    c->dt_from_cells = h.dt_from_cells != 0;
    c->speeds_ready = false;
    return FC_OK;
}

}  // extern "C"
