// fc_update_launch.cuh -- launchers of the fused patch update (Sec. 3 and
// Sec. 4 of the paper: ghost fill, wave propagation with limited
// corrections and transverse propagation, conservative update, CFL maximum,
// coarse-fine registers), one CTA per patch, and its persistent pipelined
// form.  Instantiated per precision in fc_update_f32.cu and fc_update_f64.cu.
//
// Work decomposition of k_update: one CTA per patch.  The CTA gathers the
// patch and its two ghost layers into shared memory straight from the
// neighbours' interiors (neighbour table lookup; same-level copy and 2x2
// averages read neighbour interiors, which the neighbouring CTAs are reading
// at the same time, so the reread hits L2), or from the complete tile of a
// coarser neighbour.  Every edge's Riemann problem is solved once into shared
// memory; corrections, transverse parts and the update are gathered from
// there in fixed order (deterministic, no atomics except the CFL maximum).
#pragma once
#include "fc_update.cuh"

namespace fc {

// ---------------------------------------------------------------------------
// Persistent, software-pipelined variant of the fused update.  Each CTA walks
// the patch list with stride gridDim.x and, while it computes patch b, has the
// interior and the same-level ghost layers of its next patch in flight as
// asynchronous global-to-shared copies (cp.async), and the static neighbour
// record of the patch after that.  Ghost cells from finer or coarser
// neighbours (L2-resident sources that need arithmetic) and the walls are
// completed after the copies land.  The arithmetic is that of k_update.


// issue the copies of patch p's interior and of its same-level ghost layers
// (a same-level neighbour at the patch's own time, weight 1) into tile
template <typename T, int M, int F, int NT>
__device__ __forceinline__ void issue_patch_copies(const Env<T> &e, const NbMeta<T> *meta, T *tile)
{
    constexpr int PP = (M + 4) * (M + 4), MM = M * M, NV = 16 / sizeof(T), RV = M / NV;
    const NbMeta<T> &me = meta[8];
    const int p = me.id[0];
    const T *own = qbuf(e, me.bnew[0]) + (size_t)p * MM;
    const size_t fstride = (size_t)e.n * MM;
    // interior: F x M rows x RV 16-byte pieces
    for (int v = threadIdx.x; v < F * M * RV; v += NT) {
        const int f = v / (M * RV), r = v - f * (M * RV), j = r / RV, c = (r - j * RV) * NV;
        cp_async16(tile + f * PP + tix<M>(c, j), own + f * fstride + j * M + c);
    }
    // ghost rows of the -y / +y faces: 2 rows each from the neighbour's rows
    // M-2, M-1 (below) or 0, 1 (above)
    for (int v = threadIdx.x; v < 2 * F * 2 * RV; v += NT) {
        const int d = 2 + v / (F * 2 * RV), r = v % (F * 2 * RV), f = r / (2 * RV), h = (r / RV) & 1;
        const int c = (r % RV) * NV;
        const NbMeta<T> &m = meta[d];
        if (m.kind != FC_NB_SAME || m.alpha[0] != T(1) || m.id[0] < 0) continue;
        const int j = d == 2 ? -2 + h : M + h, sj = d == 2 ? M - 2 + h : h;
        const T *src = qbuf(e, m.bnew[0]) + (size_t)m.id[0] * MM + f * fstride;
        cp_async16(tile + f * PP + tix<M>(c, j), src + sj * M + c);
    }
    // ghost columns of the -x / +x faces (M rows) and the four 2 x 2 corner
    // blocks (2 rows), as pairs of adjacent cells
    for (int v = threadIdx.x; v < F * (2 * M + 8); v += NT) {
        const int f = v / (2 * M + 8), r = v - f * (2 * M + 8);
        int d, j, sj;
        if (r < 2 * M) { d = r / M; j = r % M; sj = j; }
        else { d = 4 + (r - 2 * M) / 2; const int h = (r - 2 * M) & 1;
               const bool up = d >= 6; j = up ? M + h : -2 + h; sj = up ? h : M - 2 + h; }
        const NbMeta<T> &m = meta[d];
        if (m.kind != FC_NB_SAME || m.alpha[0] != T(1) || m.id[0] < 0) continue;
        const bool plus = d == 1 || d == 5 || d == 7;
        const int i = plus ? M : -2, si = plus ? 0 : M - 2;
        const T *src = qbuf(e, m.bnew[0]) + (size_t)m.id[0] * MM + f * fstride + sj * M + si;
        T *dst = tile + f * PP + tix<M>(i, j);
        if constexpr (sizeof(T) == 4) cp_async8(dst, src);
        else cp_async16(dst, src);
    }
}

// at least MINB CTAs of NT threads per SM (a register budget: without it the
// compiler keeps far more registers live across the patch loop)
template <int M, int NT> struct PipeMinBlocks { static constexpr int v = 65536 / (NT * 40) > 4 ? 4 : 65536 / (NT * 40); };

template <typename T, int M, int EQ, int NT>
__global__ void __launch_bounds__(NT, PipeMinBlocks<M, NT>::v)
k_update_pipe(Env<T> e, const int *list, int count, int ksub, int fine_acc)
{
    pdl_begin();
    using L = UpdLayout<T, M, EQ>;
    constexpr int F = L::F, PP = L::PP, ER = L::ER;
    constexpr int NXE = L::NXE, NYE = L::NYE, NF = L::NF;
    extern __shared__ __align__(16) unsigned char smem[];
    double *red = (double *)smem;                                   // 64 doubles
    int *recb = (int *)(red + 64);                                  // 3 records of kRecInts
    int *sbuf = recb + 3 * kRecInts;                                // start buffer per level
    NbMeta<T> *meta = (NbMeta<T> *)(sbuf + kMaxLevels);             // 2 x 9 entries
    // tiles: interior rows of FP32 tiles start 16-byte aligned when the tile
    // base is 8 modulo 16 (the interior starts 2 cells into each row)
    uintptr_t tb = (uintptr_t)(meta + 18);
    tb = (tb + 15) & ~(uintptr_t)15;
    if (sizeof(T) == 4) tb += 8;
    T *tiles = (T *)tb;
    T *ex = tiles + 2 * F * PP;
    T *ey = ex + ER * NXE;
    T *s2x = ey + ER * NYE;
    T *s2y = s2x + 4 * F * NF;

    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    const int G = gridDim.x;
    if ((int)blockIdx.x >= count) return;
    if (threadIdx.x < kMaxLevels) sbuf[threadIdx.x] = e.ctl->start_buf[threadIdx.x];
    auto patch_of = [&](int b) { return list ? list[b] : b; };
    auto issue_rec = [&](int b, int slot) {
        const int4 *src = reinterpret_cast<const int4 *>(e.nbrec + (size_t)patch_of(b) * kRecInts);
        for (int v = threadIdx.x; v < kRecInts / 4; v += NT) cp_async16(recb + slot * kRecInts + 4 * v, src + v);
    };
    // prologue: records of the first two patches, then the first patch's data
    int b = blockIdx.x;
    issue_rec(b, 0);
    if (b + G < count) issue_rec(b + G, 1);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (threadIdx.x < 9) meta_from_rec(e, recb + 6 * threadIdx.x, sbuf, (int)threadIdx.x, meta[threadIdx.x]);
    __syncthreads();
    issue_patch_copies<T, M, F, NT>(e, meta, tiles);
    cp_async_commit();
    for (int it = 0; b < count; ++it, b += G) {
        const int cur = it & 1;
        NbMeta<T> *mc = meta + 9 * cur, *mn = meta + 9 * (cur ^ 1);
        T *tile = tiles + cur * F * PP;
        const int p = mc[8].id[0], lev = e.f.level[p];
        cp_async_wait_all();
        __syncthreads();
        if (mc[8].alpha[0] != T(1)) {              // the updated level is always at its own time
            if (threadIdx.x == 0) e.ctl->index_error = 1;
            return;
        }
        if (b + G < count && threadIdx.x < 9)
            meta_from_rec(e, recb + ((it + 1) % 3) * kRecInts + 6 * threadIdx.x, sbuf, (int)threadIdx.x,
                          mn[threadIdx.x]);
        // ghost cells the copies did not bring
        const int xp = mc[8].x[0], yp = mc[8].y[0];
        int bad = 0;
        for (int g = threadIdx.x; g < 8 * M + 16; g += NT) {
            int i, j;
            constexpr int P = M + 4;
            if (g < 2 * P) { j = -2 + g / P; i = g % P - 2; }
            else if (g < 4 * P) { int h = g - 2 * P; j = M + h / P; i = h % P - 2; }
            else { int h = g - 4 * P; j = h >> 2; int c = h & 3; i = c < 2 ? c - 2 : M + c - 2; }
            const int d = dir_of(i < 0 ? -1 : (i >= M ? 1 : 0), j < 0 ? -1 : (j >= M ? 1 : 0));
            const NbMeta<T> &m = mc[d];
            if (m.kind == FC_NB_NONE || (m.kind == FC_NB_SAME && m.alpha[0] == T(1) && m.id[0] >= 0)) continue;
            bad |= cart_ghost<T, M, F>(e, m, d, i, j, xp, yp, lev, tile);
        }
        __syncthreads();
        if (e.conn == FC_CONN_SQUARE) apply_walls<T, M, F>(xp, yp, lev, tile);
        if constexpr (F == 3)
            for (int t = threadIdx.x; t < PP; t += NT)
                if (!(tile[t] > T(0))) bad = 1;
        if (__syncthreads_or(bad)) {               // also publishes the next patch's metadata
            if (threadIdx.x == 0) e.ctl->dry_error = 1;
            cp_async_wait_all();
            return;
        }
        // next patch's data and the record after it, in flight during the update
        if (b + G < count) issue_patch_copies<T, M, F, NT>(e, mn, tiles + (cur ^ 1) * F * PP);
        if (b + 2 * G < count) issue_rec(b + 2 * G, (it + 2) % 3);
        cp_async_commit();
        const T dtl = sizeof(T) == 8 ? (T)e.ctl->dtl_d[lev] : (T)e.ctl->dtl_f[lev];
        const T dtdx = sizeof(T) == 8 ? (T)e.ctl->dtdx_d[lev] : (T)e.ctl->dtdx_f[lev];
        update_body<T, M, EQ, NT>(e, p, lev, dtl, dtdx, mc, tile, ex, ey, s2x, s2y, nullptr, red, ksub, fine_acc);
    }
    cp_async_wait_all();
}

template <typename T, int M, int EQ, int V>
static int launch_update_t(const Env<T> &e, List l, int ksub, int fine_acc, cudaStream_t s)
{
    using Lay = UpdLayout<T, M, EQ>;
    constexpr int NT = UpdCfg<M, V>::NT;
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(k_update<T, M, EQ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Lay::bytes);
        if (err != cudaSuccess) return cuda_status(err, "cudaFuncSetAttribute(k_update)");
        configured = true;
    }
    if (l.count <= 0) return FC_OK;
    FC_CUDA(launch_pdl(k_update<T, M, EQ, NT>, l.count, NT, Lay::bytes, s, e, l.idx, l.count, ksub, fine_acc));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

// shared memory of the pipelined variant: records, start buffers, two
// metadata sets, two tiles (plus alignment), edge records and slots
template <typename T, int M, int EQ>
struct PipeLayout {
    using L = UpdLayout<T, M, EQ>;
    static constexpr size_t bytes = 64 * sizeof(double) + 3 * kRecInts * sizeof(int) + kMaxLevels * sizeof(int) +
                                    18 * sizeof(NbMeta<T>) + 32 +
                                    (2 * (size_t)L::F * L::PP + (size_t)L::ER * (L::NXE + L::NYE) + L::SLOTS) * sizeof(T);
};

template <typename T, int M, int EQ, int V>
static int launch_pipe_t(const Env<T> &e, List l, int ksub, int fine_acc, cudaStream_t s)
{
    using Lay = PipeLayout<T, M, EQ>;
    constexpr int NT = UpdCfg<M, V>::NT;
    static int resident = 0;      // CTAs of this shape that fit on the device at once
    if (!resident) {
        cudaError_t err = cudaFuncSetAttribute(k_update_pipe<T, M, EQ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Lay::bytes);
        if (err != cudaSuccess) return cuda_status(err, "cudaFuncSetAttribute(k_update_pipe)");
        int dev = 0, sms = 0, per = 0;
        FC_CUDA(cudaGetDevice(&dev));
        FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_update_pipe<T, M, EQ, NT>, NT, Lay::bytes));
        resident = sms * (per > 0 ? per : 1);
    }
    if (l.count <= 0) return FC_OK;
    int grid = l.count < resident ? l.count : resident;
    FC_CUDA(launch_pdl(k_update_pipe<T, M, EQ, NT>, grid, NT, Lay::bytes, s, e, l.idx, l.count, ksub, fine_acc));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

// variant: bit 0 = threads per CTA, bit 1 = persistent pipelined kernel
// (square and periodic square)
template <typename T, int M, int EQ>
static int launch_update_v(const Env<T> &e, List l, int ksub, int fine_acc, int variant, cudaStream_t s)
{
    if constexpr (EQ == FC_EQ_SWE)
        if (variant >= 4) return launch_sweep<T>(e, l, fine_acc, variant - 4, s);
    if constexpr (EQ != kEqSphere) {
        if (variant & 2)
            return (variant & 1) ? launch_pipe_t<T, M, EQ, 1>(e, l, ksub, fine_acc, s)
                                 : launch_pipe_t<T, M, EQ, 0>(e, l, ksub, fine_acc, s);
    }
    return (variant & 1) ? launch_update_t<T, M, EQ, 1>(e, l, ksub, fine_acc, s)
                         : launch_update_t<T, M, EQ, 0>(e, l, ksub, fine_acc, s);
}

template <typename T>
int launch_update(const Env<T> &e, List l, int ksub, int fine_acc, int variant, cudaStream_t s)
{
    if (e.t2 || e.efix) return launch_update_ext<T>(e, l, ksub, fine_acc, variant, s);
    if (e.eq == FC_EQ_SWE) {
        if (e.m == 8) return launch_update_v<T, 8, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
        if (e.m == 16) return launch_update_v<T, 16, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
        if constexpr (sizeof(T) == 4)      // FP64 m = 32 shallow water does not fit shared memory
            if (e.m == 32) return launch_update_v<T, 32, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
    } else if (e.geo) {                   // capacity form with per-patch geometry
        if (e.m == 8) return launch_update_v<T, 8, kEqSphere>(e, l, ksub, fine_acc, variant, s);
        if (e.m == 16) return launch_update_v<T, 16, kEqSphere>(e, l, ksub, fine_acc, variant, s);
        if (e.m == 32) return launch_update_v<T, 32, kEqSphere>(e, l, ksub, fine_acc, variant, s);
    } else {
        if (e.m == 8) return launch_update_v<T, 8, FC_EQ_ADV>(e, l, ksub, fine_acc, variant, s);
        if (e.m == 16) return launch_update_v<T, 16, FC_EQ_ADV>(e, l, ksub, fine_acc, variant, s);
        if (e.m == 32) return launch_update_v<T, 32, FC_EQ_ADV>(e, l, ksub, fine_acc, variant, s);
    }
    set_error("unsupported patch size %d for this precision / equation", e.m);
    return FC_ERR_UNIMPLEMENTED;
}

}  // namespace fc
