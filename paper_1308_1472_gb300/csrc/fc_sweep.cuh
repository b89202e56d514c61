// fc_sweep.cuh -- row-sweep form of the fused shallow-water patch update
// (kernels and launchers; instantiated per patch size in fc_sweep_m*.cu).
//
// The same method as k_update (Sec. 3: ghost fill, Roe Riemann solves,
// MC-limited second-order corrections with transverse propagation,
// conservative update; Sec. 4: CFL maximum and coarse-fine registers), with
// the edge records kept in registers instead of shared memory.
//
// Work decomposition: a lane owns C adjacent columns of a patch's padded
// (m+4) x (m+4) tile, so a patch takes LP = (m+4)/C lanes and a warp carries
// PPW = 32/LP patches side by side; a CTA is W such warps.  Each warp fills
// its patches' tiles in shared memory (the ghost fill of k_update, run by
// the warp alone), then sweeps the tile rows from bottom to top.  At row r a
// lane solves the Riemann problems of the x-edge left of each of its cells
// (row r) and of the y-edge below it (between rows r-1 and r).  Everything a
// later row needs stays in registers:
//   * x-edge limiters read the neighbouring columns' records of the same row
//     (in the lane, or from the next lane by a warp shuffle);
//   * y-edge limiters read the records of rows r-2, r-1, r of the same
//     column, so the y-edge between rows r-2 and r-1 is completed at row r;
//   * transverse parts travel at most one column (shuffle) and one row;
//   * a cell's update is complete once the y-edge above it is, two rows
//     after the cell was loaded.
// No shared-memory round trip per edge and no block-wide barrier: the warp
// synchronises with itself only after the ghost fill.
//
// Transverse parts entering an edge's correction flux are taken in the order
// below-left, below-right, above-left, above-right (as in k_update); the x
// edges subtract them one by one after their own correction, the y edges
// add them up first and subtract the sum (the sum is formed before the y
// edge's own correction is known), a different rounding of the same sum.
#pragma once
#include "fc_patch.cuh"

namespace fc {

// columns per lane (C) of the three sweep variants for each patch size
template <int M> struct SweepCols;
template <> struct SweepCols<8> { static constexpr int c[3] = {1, 2, 4}; };
template <> struct SweepCols<16> { static constexpr int c[3] = {1, 2, 4}; };
template <> struct SweepCols<32> { static constexpr int c[3] = {2, 3, 4}; };

template <typename T, int M, int C>
struct SweepShape {
    static constexpr int P = M + 4, PP = P * P, F = 3;
    static_assert(P % C == 0, "the padded tile width is a whole number of lane strips");
    static constexpr int LP = P / C;              // lanes per patch
    static_assert(LP <= 32, "a patch fits in one warp");
    static constexpr int PPW = 32 / LP;           // patches per warp
    // warps per CTA: about 64 KB of shared memory per CTA
    static constexpr size_t warp_bytes = (size_t)PPW * (F * PP * sizeof(T) + 9 * sizeof(NbMeta<T>)) + 32 * sizeof(T);
    static constexpr int W = warp_bytes * 4 <= 72 * 1024 ? 4 : (warp_bytes * 2 <= 72 * 1024 ? 2 : 1);
    static constexpr size_t meta_bytes = (((size_t)W * PPW * 9 * sizeof(NbMeta<T>)) + 15) / 16 * 16;
    static constexpr size_t bytes = meta_bytes + (size_t)W * PPW * F * PP * sizeof(T) + (size_t)W * 32 * sizeof(T);
};

// shared memory of a sweep CTA: per warp the metadata of its patch group
// (and of the next group, for the persistent form), the tiles (FP32: 8 bytes
// past a 16-byte boundary, see prefetch_row) and the CFL scratch
template <typename T, int M, int C, bool PIPE>
struct SweepLayout {
    using S = SweepShape<T, M, C>;
    static constexpr int W = S::W, PPW = S::PPW, F = 3, PP = S::PP;
    static constexpr int NMETA = PPW * 9 * (PIPE ? 2 : 1);                  // entries per warp
    static constexpr size_t meta_bytes = ((size_t)W * NMETA * sizeof(NbMeta<T>) + 15) / 16 * 16;
    static constexpr size_t tile_off = meta_bytes + (sizeof(T) == 4 ? 8 : 0);
    static constexpr size_t red_off = (tile_off + (size_t)W * PPW * F * PP * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t bytes = red_off + (size_t)W * 32 * sizeof(T);
};

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_dn1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// C consecutive values of one tile row (pairs as one 8- or 16-byte access)
template <typename T, int C>
__device__ __forceinline__ void load_cols(const T *src, T *v)
{
    if constexpr (C % 2 == 0) {
        using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        #pragma unroll
        for (int c = 0; c < C; c += 2) {
            V2 w = *reinterpret_cast<const V2 *>(src + c);
            v[c] = w.x; v[c + 1] = w.y;
        }
    } else {
        #pragma unroll
        for (int c = 0; c < C; ++c) v[c] = src[c];
    }
}

// physical x- and y-direction fluxes of a cell state (coarse-fine registers;
// every product and sum rounded on its own: no contraction, so that the
// registers do not depend on how a launch shape's code was scheduled)
template <typename T>
__device__ __forceinline__ T swe_flux(int dir, int f, T h, T hu, T hv, T g)
{
    const T u = hu / h, v = hv / h;
    const T p = rmul(rmul(rmul(T(0.5), g), h), h);
    if (dir == 0) return f == 0 ? hu : (f == 1 ? radd(rmul(hu, u), p) : rmul(hu, v));
    return f == 0 ? hv : (f == 2 ? radd(rmul(hv, v), p) : rmul(hv, u));
}

// register of one coarse-fine side: dt times the effective flux through it
template <typename T>
__device__ __forceinline__ void put_register(const Env<T> &e, const NbMeta<T> &ms, int along, int fine_acc, T dtl,
                                             const T *val)
{
    const int slot = ms.cfslot;
    const bool acc = ms.kind == FC_NB_COARSER && fine_acc;
    double *rg = e.reg + ((size_t)slot * e.m + along) * 3;
    #pragma unroll
    for (int f = 0; f < 3; ++f) {
        const double r = __dmul_rn((double)dtl, (double)val[f]);
        rg[f] = acc ? __dadd_rn(rg[f], r) : r;
    }
}

template <typename T, int M, int C, int W>
__global__ void __launch_bounds__(32 * W)
k_sweep(Env<T> e, const int *list, int count, int fine_acc)
{
    pdl_trigger();
    using S = SweepShape<T, M, C>;
    constexpr int F = 3, P = S::P, PP = S::PP, LP = S::LP, PPW = S::PPW;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    NbMeta<T> *meta = reinterpret_cast<NbMeta<T> *>(smem) + (size_t)warp * PPW * 9;
    T *tiles = reinterpret_cast<T *>(smem + S::meta_bytes) + (size_t)warp * PPW * F * PP;
    T *red = reinterpret_cast<T *>(smem + S::meta_bytes) + (size_t)W * PPW * F * PP + warp * 32;

    const int b0 = (blockIdx.x * W + warp) * PPW;
    if (b0 >= count) return;                                // whole warp
    // metadata and ghost-filled tiles of this warp's patches (a slot past the
    // end of the list repeats the last patch and writes nothing); the
    // forest's part of the metadata before the wait for the previous kernel
    warp_load_meta<T, PPW, true>(e, list, count, b0, meta);
    pdl_wait();
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    warp_meta_time<T, PPW>(e, meta);
    {
        // the updated level is at its own time (weight 1) by construction
        // of the step plan
        bool own_time = true;
        #pragma unroll
        for (int s = 0; s < PPW; ++s) own_time = own_time && meta[9 * s + 8].alpha[0] == T(1);
        if (!own_time) {
            if (lane == 0) e.ctl->index_error = 1;
            return;
        }
    }
    const int dry = warp_fill_tiles<T, M, PPW>(e, meta, tiles);
    if (dry) {                                              // warp-uniform
        if (lane == 0) e.ctl->dry_error = 1;
        return;
    }

    // this lane's patch and columns i0 .. i0 + C - 1 (lanes past the last
    // patch of the warp shadow real columns and write nothing)
    int seg = lane / LP, kl = lane - seg * LP;
    const bool idle = seg >= PPW;
    if (idle) { seg = PPW - 1; kl = LP - 1; }
    const bool live = !idle && b0 + seg < count;
    const NbMeta<T> *mm = meta + 9 * seg;
    const int p = mm[8].id[0];
    const int lev = mm[8].lev;
    const T dtl = sizeof(T) == 8 ? (T)e.ctl->dtl_d[lev] : (T)e.ctl->dtl_f[lev];
    const T dtdx = sizeof(T) == 8 ? (T)e.ctl->dtdx_d[lev] : (T)e.ctl->dtdx_f[lev];
    const T kk = T(0.5) * dtdx, g = e.g;
    const T *tile = tiles + seg * F * PP;
    const int i0 = kl * C - 2;
    T *qout = qbuf(e, buf_out(e.ctl->start_buf[lev], e.kdone[lev] + 1)) + (size_t)p * (M * M);
    const size_t fstride = (size_t)e.n * (M * M);
    const bool cf0 = mm[0].cfslot >= 0, cf1 = mm[1].cfslot >= 0, cf2 = mm[2].cfslot >= 0, cf3 = mm[3].cfslot >= 0;

    // carried state, per column: row r-1 (conserved and primitive), y-edge
    // records of rows r-1 and r-2, transverse sums into y-edges r-1
    // (complete) and r (partial), x-edge row r-1 (partial correction flux and
    // fluctuations), cell row r-2 (q - dt/dx X and its lower y contribution)
    T ph[C], pu_[C], pv_[C], qu[C], qv[C], ps[C];
    T ry1[C][6], ry2[C][6];
    T typ[C][3], tyc[C][3];
    T vxp[C][3], apxp[C][3], amxp[C][3];
    T qpp[C][3], clyp[C][3];
    #pragma unroll
    for (int c = 0; c < C; ++c)
        #pragma unroll
        for (int f = 0; f < 3; ++f) { tyc[c][f] = T(0); typ[c][f] = T(0); }
    T smax = T(0);
    int bad = 0;

    #pragma unroll 1
    for (int r = -2; r <= M + 1; ++r) {
        // ---- cells of row r
        T h[C], hu[C], hv[C], u[C], v[C], sq[C];
        {
            const T *row = tile + (r + 2) * P + kl * C;
            load_cols<T, C>(row, h);
            load_cols<T, C>(row + PP, hu);
            load_cols<T, C>(row + 2 * PP, hv);
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                const T ih = fdiv(T(1), h[c]);
                u[c] = hu[c] * ih; v[c] = hv[c] * ih; sq[c] = fsqrt(h[c]);
            }
        }
        // ---- y-edge records of row r (edge below each cell; frame h, hv, hu)
        T ryc[C][6];
        if (r >= -1) {
            #pragma unroll
            for (int c = 0; c < C; ++c)
                swe_roe(ph[c], qv[c], qu[c], pv_[c], pu_[c], ps[c], h[c], hv[c], hu[c], v[c], u[c], sq[c], g, ryc[c]);
        }
        // ---- x-edge records of row r (edge left of each cell)
        T rx[C][6];
        if (r >= -1 && r <= M) {
            const T lh = shfl_up1(h[C - 1]), lhu = shfl_up1(hu[C - 1]), lhv = shfl_up1(hv[C - 1]);
            const T lu = shfl_up1(u[C - 1]), lv = shfl_up1(v[C - 1]), ls = shfl_up1(sq[C - 1]);
            swe_roe(lh, lhu, lhv, lu, lv, ls, h[0], hu[0], hv[0], u[0], v[0], sq[0], g, rx[0]);
            #pragma unroll
            for (int c = 1; c < C; ++c)
                swe_roe(h[c - 1], hu[c - 1], hv[c - 1], u[c - 1], v[c - 1], sq[c - 1], h[c], hu[c], hv[c], u[c], v[c],
                        sq[c], g, rx[c]);
        }
        // ---- CFL maximum over the patch's interior edges; subsonic test of
        // every fluctuation formed in this row (one form per warp and row)
        bool ok = true;
        #pragma unroll
        for (int c = 0; c < C; ++c) {
            const int i = i0 + c;
            if (r >= -1 && r <= M && i >= 0 && i <= M) {
                if (r >= 0 && r <= M - 1) smax = tmax(smax, fabs(rx[c][3]) + rx[c][5]);
                ok = ok && fabs(rx[c][3]) < rx[c][5] && fabs(rx[c][4]) < rx[c][5];
            }
            if (r >= 0 && r <= M && i >= -1 && i <= M) {
                if (i >= 0 && i <= M - 1) smax = tmax(smax, fabs(ryc[c][3]) + ryc[c][5]);
                ok = ok && fabs(ryc[c][3]) < ryc[c][5] && fabs(ryc[c][4]) < ryc[c][5];
            }
            if (r >= 1 && i >= 0 && i <= M - 1) ok = ok && fabs(ry1[c][3]) < ry1[c][5];
        }
        const bool sub = __all_sync(0xffffffffu, ok || !live);

        // ---- the y-edges of row r-1 are complete: correction flux and the
        // contributions to the cells above and below; cell row r-2 is updated
        if (r >= 1) {
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                const int i = i0 + c;
                T own[3], am[3], ap[3], cly[3], cry[3];
                own_correction<T, FC_EQ_SWE>(ry1[c], ry2[c], ryc[c], dtdx, own);
                if (sub) swe_fluct_sub(ry1[c], am, ap);
                else swe_fluct(ry1[c], am, ap);
                #pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const int fe = f == 0 ? 0 : 3 - f;        // frame index of global component f
                    const T w = own[fe] - typ[c][f];
                    cly[f] = ap[fe] - w;
                    cry[f] = am[fe] + w;
                }
                const bool cell = live && i >= 0 && i <= M - 1;
                if (r >= 2 && cell) {
                    const int j = r - 2;
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        const T qn = qpp[c][f] - dtdx * (clyp[c][f] + cry[f]);
                        if (!isfinite(qn)) bad = 1;
                        qpp[c][f] = qn;                        // stored below
                    }
                    (void)j;
                }
                if (cell && r == 1 && cf2) {                   // lower side, cell (i, 0)
                    T val[3];
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) val[f] = rsub(swe_flux(1, f, ph[c], qu[c], qv[c], g), cly[f]);
                    put_register(e, mm[2], i, fine_acc, dtl, val);
                }
                if (cell && r == M + 1 && cf3) {               // upper side, cell (i, M - 1)
                    const T *q1 = tile + (M + 1) * P + (i + 2);
                    T val[3];
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) val[f] = radd(swe_flux(1, f, q1[0], q1[PP], q1[2 * PP], g), cry[f]);
                    put_register(e, mm[3], i, fine_acc, dtl, val);
                }
                #pragma unroll
                for (int f = 0; f < 3; ++f) clyp[c][f] = cly[f];
            }
            if (r >= 2 && live) {
                // new values of cell row r-2 (pairs of columns as one store)
                T *dst = qout + (r - 2) * M + i0;
                if constexpr (C % 2 == 0) {
                    using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
                    #pragma unroll
                    for (int c = 0; c < C; c += 2)
                        if (i0 + c >= 0 && i0 + c <= M - 1)
                            #pragma unroll
                            for (int f = 0; f < 3; ++f) {
                                V2 w; w.x = qpp[c][f]; w.y = qpp[c + 1][f];
                                *reinterpret_cast<V2 *>(dst + f * fstride + c) = w;
                            }
                } else {
                    #pragma unroll
                    for (int c = 0; c < C; ++c)
                        if (i0 + c >= 0 && i0 + c <= M - 1)
                            #pragma unroll
                            for (int f = 0; f < 3; ++f) dst[f * fstride + c] = qpp[c][f];
                }
            }
        }

        // ---- y-edges of row r: fluctuations split into the x-edges of rows r
        // (below-left from column i-1, below-right from column i) and r-1
        // (above-left, above-right); then the x-edges of row r-1 are complete
        // and cell row r-1 takes q - dt/dx X
        if (r >= 0 && r <= M) {
            T bl[C][3], br[C][3], al[C][3], ar[C][3];
            T sendp[3], sendm[3];
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                T am[3], ap[3], amm[3], amp[3], apm[3], app[3];
                if (sub) {
                    swe_fluct_sub(ryc[c], am, ap);
                    swe_trans_sub(ryc[c], am, amm, amp);
                    swe_trans_sub(ryc[c], ap, apm, app);
                } else {
                    swe_fluct(ryc[c], am, ap);
                    swe_trans(ryc[c], am, amm, amp);
                    swe_trans(ryc[c], ap, apm, app);
                }
                // frame (h, hv, hu) -> global (h, hu, hv)
                const T apm_g[3] = {apm[0], apm[2], apm[1]}, app_g[3] = {app[0], app[2], app[1]};
                const T amm_g[3] = {amm[0], amm[2], amm[1]}, amp_g[3] = {amp[0], amp[2], amp[1]};
                #pragma unroll
                for (int f = 0; f < 3; ++f) {
                    br[c][f] = apm_g[f];
                    ar[c][f] = amm_g[f];
                    if (c + 1 < C) { bl[c + 1][f] = app_g[f]; al[c + 1][f] = amp_g[f]; }
                    else { sendp[f] = app_g[f]; sendm[f] = amp_g[f]; }
                }
            }
            #pragma unroll
            for (int f = 0; f < 3; ++f) { bl[0][f] = shfl_up1(sendp[f]); al[0][f] = shfl_up1(sendm[f]); }

            if (r >= 1) {
                T clx[C][3], crx[C][3];
                #pragma unroll
                for (int c = 0; c < C; ++c)
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        T w = vxp[c][f] - kk * al[c][f];
                        w = w - kk * ar[c][f];
                        clx[c][f] = apxp[c][f] - w;
                        crx[c][f] = amxp[c][f] + w;
                    }
                T crn[3];
                #pragma unroll
                for (int f = 0; f < 3; ++f) crn[f] = shfl_dn1(crx[0][f]);
                #pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int i = i0 + c;
                    const T *cr_next = c + 1 < C ? crx[c + 1] : crn;
                    const T qc[3] = {ph[c], qu[c], qv[c]};
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) qpp[c][f] = qc[f] - dtdx * (clx[c][f] + cr_next[f]);
                    if (live && cf0 && i == 0) {               // left side, cell (0, r - 1)
                        T val[3];
                        #pragma unroll
                        for (int f = 0; f < 3; ++f) val[f] = rsub(swe_flux(0, f, qc[0], qc[1], qc[2], g), clx[c][f]);
                        put_register(e, mm[0], r - 1, fine_acc, dtl, val);
                    }
                    if (live && cf1 && i == M - 1) {           // right side, cell (M - 1, r - 1)
                        T val[3];
                        #pragma unroll
                        for (int f = 0; f < 3; ++f) val[f] = radd(swe_flux(0, f, qc[0], qc[1], qc[2], g), cr_next[f]);
                        put_register(e, mm[1], r - 1, fine_acc, dtl, val);
                    }
                }
            }
            if (r <= M - 1) {
                // x-edges of row r: own correction (records of the columns
                // beside), then the two lower transverse parts
                T nl[6], nr[6];
                #pragma unroll
                for (int k = 0; k < 6; ++k) { nl[k] = shfl_up1(rx[C - 1][k]); nr[k] = shfl_dn1(rx[0][k]); }
                #pragma unroll
                for (int c = 0; c < C; ++c) {
                    const T *rl = c > 0 ? rx[c - 1] : nl;
                    const T *rr = c + 1 < C ? rx[c + 1] : nr;
                    T own[3];
                    own_correction<T, FC_EQ_SWE>(rx[c], rl, rr, dtdx, own);
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        const T w = own[f] - kk * bl[c][f];
                        vxp[c][f] = w - kk * br[c][f];
                    }
                }
            }
        }

        // ---- x-edges of row r: fluctuations (kept for row r+1) split into the
        // y-edges of rows r (above-left from column i, above-right from column
        // i+1) and r+1 (below-left, below-right)
        if (r >= -1 && r <= M) {
            T amm[C][3], amp[C][3], apm[C][3], app[C][3];
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                if (sub) {
                    swe_fluct_sub(rx[c], amxp[c], apxp[c]);
                    swe_trans_sub(rx[c], amxp[c], amm[c], amp[c]);
                    swe_trans_sub(rx[c], apxp[c], apm[c], app[c]);
                } else {
                    swe_fluct(rx[c], amxp[c], apxp[c]);
                    swe_trans(rx[c], amxp[c], amm[c], amp[c]);
                    swe_trans(rx[c], apxp[c], apm[c], app[c]);
                }
            }
            T rm[3], rp[3];
            #pragma unroll
            for (int f = 0; f < 3; ++f) { rm[f] = shfl_dn1(amm[0][f]); rp[f] = shfl_dn1(amp[0][f]); }
            #pragma unroll
            for (int c = 0; c < C; ++c) {
                const T *nmm = c + 1 < C ? amm[c + 1] : rm;
                const T *nmp = c + 1 < C ? amp[c + 1] : rp;
                #pragma unroll
                for (int f = 0; f < 3; ++f) {
                    typ[c][f] = (tyc[c][f] + kk * apm[c][f]) + kk * nmm[f];   // y-edge row r: complete
                    tyc[c][f] = kk * app[c][f] + kk * nmp[f];                 // y-edge row r+1: lower parts
                }
            }
        } else {
            #pragma unroll
            for (int c = 0; c < C; ++c)
                #pragma unroll
                for (int f = 0; f < 3; ++f) { typ[c][f] = tyc[c][f]; tyc[c][f] = T(0); }
        }

        // ---- shift the row window
        #pragma unroll
        for (int c = 0; c < C; ++c) {
            ph[c] = h[c]; qu[c] = hu[c]; qv[c] = hv[c]; pu_[c] = u[c]; pv_[c] = v[c]; ps[c] = sq[c];
            #pragma unroll
            for (int k = 0; k < 6; ++k) { ry2[c][k] = ry1[c][k]; ry1[c][k] = ryc[c][k]; }
        }
    }

    if (bad) e.ctl->nonfinite_error = 1;          // every writer stores the same value
    // CFL maximum of each patch: one atomic per patch from its first lane
    red[lane] = live ? smax : T(0);
    __syncwarp();
    if (live && kl == 0) {
        T mx = T(0);
        #pragma unroll 1
        for (int k = 0; k < LP; ++k) mx = tmax(mx, red[seg * LP + k]);
        atomic_max_nonneg(&e.ctl->smax_bits[lev], (double)mx);
    }
}

}  // namespace fc

// ---------------------------------------------------------------------------
// FP32 row sweep with two columns per lane in packed form.  The two columns
// of a lane go through the same arithmetic, so they are held as one float2
// and every add, multiply and fused multiply-add acts on both at once
// (Blackwell's paired FP32 instructions: one issue for two columns).
// Reciprocals, square roots, comparisons, minima and maxima stay per column.
namespace fc {
namespace pk {

typedef float2 f2;
__device__ __forceinline__ f2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }   // exact a - b
__device__ __forceinline__ f2 rcp(f2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
__device__ __forceinline__ f2 sqrt_(f2 a) { return mul(a, make_float2(rsqrtf(a.x), rsqrtf(a.y))); }
__device__ __forceinline__ f2 minz(f2 a) { return make_float2(fminf(a.x, 0.f), fminf(a.y, 0.f)); }
__device__ __forceinline__ f2 maxz(f2 a) { return make_float2(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f)); }
struct b2 { bool x, y; };
__device__ __forceinline__ f2 pick(b2 c, f2 a, f2 b) { return make_float2(c.x ? a.x : b.x, c.y ? a.y : b.y); }
// (left neighbour, this) and (this, right neighbour) column pairs of a
// packed value across the lanes of the warp
__device__ __forceinline__ f2 lpair(f2 a) { return make_float2(__shfl_up_sync(0xffffffffu, a.y, 1), a.x); }
__device__ __forceinline__ f2 rpair(f2 a) { return make_float2(a.y, __shfl_down_sync(0xffffffffu, a.x, 1)); }

// Roe record {a1, a2, a3, u, v, c} of two edges (edge frame) and 0.5 / c
__device__ __forceinline__ void roe(f2 hL, f2 nL, f2 tL, f2 uL, f2 vL, f2 sqL, f2 hR, f2 nR, f2 tR, f2 uR, f2 vR,
                                    f2 sqR, f2 gh, f2 *rec, f2 &inv2c)
{
    const f2 inv = rcp(add(sqL, sqR));
    const f2 u = mul(fma(sqL, uL, mul(sqR, uR)), inv);
    const f2 v = mul(fma(sqL, vL, mul(sqR, vR)), inv);
    // c = sqrt(g (hL + hR) / 2) and 1 / c from one reciprocal square root
    const f2 c2 = mul(gh, add(hL, hR));
    const f2 rc = make_float2(rsqrtf(c2.x), rsqrtf(c2.y));
    const f2 c = mul(c2, rc);
    const f2 d0 = sub(hR, hL), nd1 = sub(nL, nR), d2 = sub(tR, tL);
    inv2c = mul(bc(0.5f), rc);
    const f2 ninv2c = mul(bc(-0.5f), rc);
    rec[0] = mul(fma(add(u, c), d0, nd1), inv2c);              // ((u + c) d0 - d1) / 2c
    rec[1] = sub(d2, mul(v, d0));                              // d2 - v d0
    rec[2] = mul(fma(sub(u, c), d0, nd1), ninv2c);             // (d1 - (u - c) d0) / 2c
    rec[3] = u; rec[4] = v; rec[5] = c;
}

// fluctuations of two edges: subsonic form (|u| < c) and general form
__device__ __forceinline__ void fluct_sub(const f2 *r, f2 *am, f2 *ap)
{
    const f2 u = r[3], v = r[4], c = r[5];
    const f2 s1 = sub(u, c), s3 = add(u, c);
    const f2 m1 = mul(s1, r[0]), p3 = mul(s3, r[2]);
    const f2 m2 = mul(minz(u), r[1]), p2 = mul(maxz(u), r[1]);
    am[0] = m1; am[1] = mul(m1, s1); am[2] = fma(m1, v, m2);
    ap[0] = p3; ap[1] = mul(p3, s3); ap[2] = fma(p3, v, p2);
}
__device__ __forceinline__ void fluct_gen(const f2 *r, f2 *am, f2 *ap)
{
    const f2 u = r[3], v = r[4], c = r[5];
    const f2 s1 = sub(u, c), s3 = add(u, c);
    const f2 m1 = mul(minz(s1), r[0]), m2 = mul(minz(u), r[1]), m3 = mul(minz(s3), r[2]);
    const f2 p1 = mul(maxz(s1), r[0]), p2 = mul(maxz(u), r[1]), p3 = mul(maxz(s3), r[2]);
    const f2 sm = add(m1, m3), sp = add(p1, p3);
    am[0] = sm; am[1] = fma(m3, s3, mul(m1, s1)); am[2] = fma(sm, v, m2);
    ap[0] = sp; ap[1] = fma(p3, s3, mul(p1, s1)); ap[2] = fma(sp, v, p2);
}

// split a fluctuation d of two edges along the other direction's
// eigenvectors (speeds v - c, v, v + c): subsonic (|v| < c) and general form
__device__ __forceinline__ void trans_sub(const f2 *r, f2 inv2c, const f2 *d, f2 *bm, f2 *bp)
{
    const f2 u = r[3], v = r[4], c = r[5];
    const f2 l1 = sub(v, c), l3 = add(v, c);
    const f2 b1 = mul(sub(mul(l3, d[0]), d[2]), inv2c);
    const f2 b2 = sub(d[1], mul(u, d[0]));
    const f2 b3 = mul(sub(d[2], mul(l1, d[0])), inv2c);
    const f2 g1 = mul(l1, b1), g3 = mul(l3, b3);
    const f2 m2 = mul(minz(v), b2), p2 = mul(maxz(v), b2);
    bm[0] = g1; bm[1] = fma(g1, u, m2); bm[2] = mul(g1, l1);
    bp[0] = g3; bp[1] = fma(g3, u, p2); bp[2] = mul(g3, l3);
}
__device__ __forceinline__ void trans_gen(const f2 *r, f2 inv2c, const f2 *d, f2 *bm, f2 *bp)
{
    const f2 u = r[3], v = r[4], c = r[5];
    const f2 l1 = sub(v, c), l3 = add(v, c);
    const f2 b1 = mul(sub(mul(l3, d[0]), d[2]), inv2c);
    const f2 b2 = sub(d[1], mul(u, d[0]));
    const f2 b3 = mul(sub(d[2], mul(l1, d[0])), inv2c);
    const f2 mb1 = mul(minz(l1), b1), mb3 = mul(minz(l3), b3), mb2 = mul(minz(v), b2);
    const f2 pb1 = mul(maxz(l1), b1), pb3 = mul(maxz(l3), b3), pb2 = mul(maxz(v), b2);
    bm[0] = add(mb1, mb3); bm[1] = fma(mb3, u, fma(mb1, u, mb2)); bm[2] = fma(mb3, l3, mul(mb1, l1));
    bp[0] = add(pb1, pb3); bp[1] = fma(pb3, u, fma(pb1, u, pb2)); bp[2] = fma(pb3, l3, mul(pb1, l1));
}

// half the MC limiter, phi(th) / 2 = clamp(min((1 + th) / 4, th), 0, 1)
// (the same rounding as max(0, min((1 + th) / 2, 2, 2 th)) / 2: the scalings
// are powers of two); saturation maps the NaN of a zero wave (th = 0 / 0) to
// 0, and the wave itself is 0 then, so its correction is 0 as for W.W = 0
__device__ __forceinline__ f2 mc_half(f2 th)
{
    const f2 t = fma(bc(0.25f), th, bc(0.25f));
    return make_float2(__saturatef(fminf(t.x, th.x)), __saturatef(fminf(t.y, th.y)));
}

// MC-limited own correction (times 0.5) of two edges; recL / recR are the
// records of the edges before and after each (the upwind one is chosen per
// wave and column)
// SUB: the edges' u - c < 0 < u + c (the subsonic rows), so waves 1 and 3
// take the right and the left edge as upwind without a comparison, and |s|
// without an absolute value: the same values
template <bool SUB>
__device__ __forceinline__ void own(const f2 *r, const f2 *rl, const f2 *rr, f2 dtdx, f2 *out)
{
    const f2 u = r[3], v = r[4], c = r[5];
    const f2 one = bc(1.f), ndtdx = mul(dtdx, bc(-1.f));
    f2 kc[3];                     // half of |s| (1 - dt/dx |s|) phi a per wave
    #pragma unroll
    for (int p = 0; p < 3; ++p) {
        const f2 s = p == 1 ? u : (p == 0 ? sub(u, c) : add(u, c));
        const bool known = SUB && p != 1;
        const b2 left = known ? b2{p == 2, p == 2} : b2{s.x >= 0.f, s.y >= 0.f};
        const f2 a = r[p], au = pick(left, rl[p], rr[p]);
        f2 ww, wu;
        if (p == 1) { ww = mul(a, a); wu = mul(au, a); }
        else {
            const f2 cu = pick(left, rl[5], rr[5]);
            const f2 su = p == 0 ? sub(pick(left, rl[3], rr[3]), cu) : add(pick(left, rl[3], rr[3]), cu);
            const f2 vu = pick(left, rl[4], rr[4]);
            ww = mul(mul(a, a), fma(v, v, fma(s, s, one)));
            wu = mul(mul(au, a), fma(vu, v, fma(su, s, one)));
        }
        const f2 ph = mc_half(mul(wu, rcp(ww)));
        const f2 as = known ? (p == 0 ? make_float2(-s.x, -s.y) : s) : make_float2(fabsf(s.x), fabsf(s.y));
        kc[p] = mul(fma(ndtdx, mul(as, as), as), mul(ph, a));
    }
    const f2 s1 = sub(u, c), s3 = add(u, c), k13 = add(kc[0], kc[2]);
    out[0] = k13;
    out[1] = fma(kc[2], s3, mul(kc[0], s1));
    out[2] = fma(k13, v, kc[1]);
}

}  // namespace pk

// the updated level is at its own time (weight 1) by construction of the
// step plan; anything else is reported as an index error
template <typename T, int PPW>
__device__ __forceinline__ bool group_own_time(const NbMeta<T> *meta)
{
    bool ok = true;
    #pragma unroll
    for (int s = 0; s < PPW; ++s) ok = ok && meta[9 * s + 8].alpha[0] == T(1);
    return ok;
}

// PIPE: persistent form.  Each warp walks the patch list in groups of PPW
// with stride gridDim.x * W * PPW; while it sweeps one group, the copies of
// the next group's interiors and same-level ghost cells go into the tile
// rows the sweep has finished with (row r-1 once row r is loaded), and only
// the remaining ghost cells are filled between the groups.
template <int M, int W, bool PIPE>
__global__ void __launch_bounds__(32 * W, 3)
k_sweep2(Env<float> e, const int *list, int count, int fine_acc)
{
    pdl_trigger();
    using namespace pk;
    using S = SweepShape<float, M, 2>;
    using L = SweepLayout<float, M, 2, PIPE>;
    constexpr int F = 3, P = S::P, PP = S::PP, LP = S::LP, PPW = S::PPW;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    NbMeta<float> *meta = reinterpret_cast<NbMeta<float> *>(smem) + (size_t)warp * L::NMETA;
    NbMeta<float> *meta_next = PIPE ? meta + PPW * 9 : meta;
    float *tiles = reinterpret_cast<float *>(smem + L::tile_off) + (size_t)warp * PPW * F * PP;
    float *red = reinterpret_cast<float *>(smem + L::red_off) + warp * 32;

    int b0 = (blockIdx.x * W + warp) * PPW;
    if (b0 >= count) return;
    const int stride = gridDim.x * W * PPW;
    // the forest's part of the metadata before the wait for the previous kernel
    warp_load_meta<float, PPW, true>(e, list, count, b0, meta);
    pdl_wait();
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    warp_meta_time<float, PPW>(e, meta);
    if (!group_own_time<float, PPW>(meta)) {
        if (lane == 0) e.ctl->index_error = 1;
        return;
    }
    int seg = lane / LP, kl = lane - seg * LP;
    const bool idle = seg >= PPW;
    if (idle) { seg = PPW - 1; kl = LP - 1; }
    if (warp_fill_cols<M, PPW>(e, meta, tiles, seg, kl, idle)) {
        if (lane == 0) e.ctl->dry_error = 1;
        return;
    }
    int dry = 0;

    for (;;) {
    const int bn = b0 + stride;
    const bool next = PIPE && bn < count;
    if (next) {
        warp_load_meta<float, PPW>(e, list, count, bn, meta_next);
        if (!group_own_time<float, PPW>(meta_next)) {
            if (lane == 0) e.ctl->index_error = 1;
            return;
        }
    }
    const bool live = !idle && b0 + seg < count;
    const NbMeta<float> *mm = meta + 9 * seg;
    const int p = mm[8].id[0];
    const int lev = mm[8].lev;
    const float dtl = e.ctl->dtl_f[lev], dtdx = e.ctl->dtdx_f[lev], g = e.g;
    const f2 dtdx2 = bc(dtdx), kk2 = bc(0.5f * dtdx), nkk2 = bc(-0.5f * dtdx), ndtdx2 = bc(-dtdx);
    const f2 gh = bc(0.5f * g), gsub2 = bc(0.45f * g);
    bool cok1 = true, cok2 = true;             // subsonic margin held in rows r-1, r-2
    const float *tile = tiles + seg * F * PP;
    const int i0 = kl * 2 - 2;                     // columns i0, i0 + 1
    const bool cols_in = i0 >= 0 && i0 <= M - 2;  // both cells of the lane are interior
    float *qout = qbuf(e, buf_out(e.ctl->start_buf[lev], e.kdone[lev] + 1)) + (size_t)p * (M * M);
    const size_t fstride = (size_t)e.n * (M * M);
    const bool cf0 = mm[0].cfslot >= 0, cf1 = mm[1].cfslot >= 0, cf2 = mm[2].cfslot >= 0, cf3 = mm[3].cfslot >= 0;

    f2 ph, phu, phv, pu, pv, ps;               // row r-1
    f2 ry1[6], ry2[6];                          // y-edge records rows r-1, r-2
    f2 typ[3], tyc[3];                          // transverse sums into y-edges rows r-1, r
    f2 vxp[3], apxp[3], amxp[3];                // x-edges row r-1
    f2 qpp[3], clyp[3];                         // cell row r-2
    #pragma unroll
    for (int f = 0; f < 3; ++f) { typ[f] = bc(0.f); tyc[f] = bc(0.f); }
    float smax = 0.f;
    f2 nf = bc(0.f);          // 0 * q summed over the lane's new values: NaN once one is not finite

    #pragma unroll 1
    for (int r = -2; r <= M + 1; ++r) {
        const float *row = tile + (r + 2) * P + kl * 2;
        const f2 h = *reinterpret_cast<const f2 *>(row), hu = *reinterpret_cast<const f2 *>(row + PP),
                 hv = *reinterpret_cast<const f2 *>(row + 2 * PP);
        if constexpr (PIPE) {
            // copies of the next group into the rows this sweep is done with
            if (!(h.x > 0.f) || !(h.y > 0.f)) dry = 1;
            if (next && r >= -1) {
                __syncwarp();
                prefetch_row<float, M, PPW>(e, meta_next, tiles, r - 1);
                if (r == M + 1) prefetch_row<float, M, PPW>(e, meta_next, tiles, M + 1);
                cp_async_commit();
            }
        }
        // 1 / h and sqrt(h) from one reciprocal square root
        const f2 rh = make_float2(rsqrtf(h.x), rsqrtf(h.y));
        const f2 ih = mul(rh, rh), u = mul(hu, ih), v = mul(hv, ih), sq = mul(h, rh);
        f2 ryc[6], yinv2c;
        if (r >= -1) roe(ph, phv, phu, pv, pu, ps, h, hv, hu, v, u, sq, gh, ryc, yinv2c);
        f2 rx[6], xinv2c;
        if (r >= -1 && r <= M)
            roe(lpair(h), lpair(hu), lpair(hv), lpair(u), lpair(v), lpair(sq), h, hu, hv, u, v, sq, gh, rx, xinv2c);

        #pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = i0 + k;
            if (r >= 0 && r <= M - 1 && i >= 0 && i <= M)
                smax = fmaxf(smax, fabsf(k ? rx[3].y : rx[3].x) + (k ? rx[5].y : rx[5].x));
            if (r >= 0 && r <= M && i >= 0 && i <= M - 1)
                smax = fmaxf(smax, fabsf(k ? ryc[3].y : ryc[3].x) + (k ? ryc[5].y : ryc[5].x));
        }
        // Subsonic forms of the fluctuations and transverse splits when
        // u^2 + v^2 < 0.45 g h in every cell of rows r-2 .. r of the warp's
        // tiles: then |u|, |v| < sqrt(0.45) c in each cell, and the Roe
        // averages of two such cells satisfy |u_hat|, |v_hat| < sqrt(0.9)
        // c_hat (|u_hat| <= max |u| / c * sqrt(2) c_hat), so every wave of
        // the edges this row completes has the sign the subsonic forms take.
        const f2 sp = fma(u, u, mul(v, v)), lim = mul(gsub2, h);
        const bool cok = sp.x < lim.x && sp.y < lim.y;
        const bool subs = __all_sync(0xffffffffu, (cok && cok1 && cok2) || !live);
        cok2 = cok1; cok1 = cok;

        // y-edges of row r-1: correction flux, contributions; cell row r-2
        if (r >= 1) {
            f2 ow[3], am[3], ap[3], cly[3], cry[3];
            if (subs) own<true>(ry1, ry2, ryc, dtdx2, ow);
            else own<false>(ry1, ry2, ryc, dtdx2, ow);
            if (subs) fluct_sub(ry1, am, ap);
            else fluct_gen(ry1, am, ap);
            #pragma unroll
            for (int f = 0; f < 3; ++f) {
                const int fe = f == 0 ? 0 : 3 - f;
                const f2 w = sub(ow[fe], typ[f]);
                cly[f] = sub(ap[fe], w);
                cry[f] = add(am[fe], w);
            }
            if (r >= 2) {
                #pragma unroll
                for (int f = 0; f < 3; ++f) {
                    qpp[f] = fma(ndtdx2, add(clyp[f], cry[f]), qpp[f]);
                    nf = fma(bc(0.f), qpp[f], nf);
                }
                if (live && cols_in) {
                    float *dst = qout + (r - 2) * M + i0;
                    #pragma unroll
                    for (int f = 0; f < 3; ++f) *reinterpret_cast<f2 *>(dst + f * fstride) = qpp[f];
                }
            }
            if (live && cols_in && ((r == 1 && cf2) || (r == M + 1 && cf3))) {
                #pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int i = i0 + k;
                    float val[3];
                    if (r == 1) {                                   // lower side, cell (i, 0)
                        const float qh = k ? ph.y : ph.x, qhu = k ? phu.y : phu.x, qhv = k ? phv.y : phv.x;
                        #pragma unroll
                        for (int f = 0; f < 3; ++f) val[f] = rsub(swe_flux(1, f, qh, qhu, qhv, g), (k ? cly[f].y : cly[f].x));
                        put_register(e, mm[2], i, fine_acc, dtl, val);
                    } else {                                        // upper side, cell (i, M - 1)
                        const float *q1 = mm[8].b0 + (M - 1) * M + i;
                        #pragma unroll
                        for (int f = 0; f < 3; ++f)
                            val[f] = radd(swe_flux(1, f, q1[0], q1[fstride], q1[2 * fstride], g), (k ? cry[f].y : cry[f].x));
                        put_register(e, mm[3], i, fine_acc, dtl, val);
                    }
                }
            }
            #pragma unroll
            for (int f = 0; f < 3; ++f) clyp[f] = cly[f];
        }

        // y-edges of row r: transverse parts into the x-edges of rows r and
        // r-1; x-edges of row r-1 complete; cell row r-1 takes q - dt/dx X
        if (r >= 0 && r <= M) {
            f2 am[3], ap[3], amm[3], amp[3], apm[3], app[3];
            if (subs) {
                fluct_sub(ryc, am, ap);
                trans_sub(ryc, yinv2c, am, amm, amp);
                trans_sub(ryc, yinv2c, ap, apm, app);
            } else {
                fluct_gen(ryc, am, ap);
                trans_gen(ryc, yinv2c, am, amm, amp);
                trans_gen(ryc, yinv2c, ap, apm, app);
            }
            // frame (h, hv, hu) -> global (h, hu, hv)
            const f2 br[3] = {apm[0], apm[2], apm[1]}, ar[3] = {amm[0], amm[2], amm[1]};
            const f2 bl[3] = {lpair(app[0]), lpair(app[2]), lpair(app[1])};
            const f2 al[3] = {lpair(amp[0]), lpair(amp[2]), lpair(amp[1])};
            if (r >= 1) {
                f2 clx[3], crx[3];
                #pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const f2 w = fma(nkk2, ar[f], fma(nkk2, al[f], vxp[f]));
                    clx[f] = sub(apxp[f], w);
                    crx[f] = add(amxp[f], w);
                }
                const f2 qc[3] = {ph, phu, phv};
                f2 crn[3];
                #pragma unroll
                for (int f = 0; f < 3; ++f) {
                    crn[f] = rpair(crx[f]);
                    qpp[f] = fma(ndtdx2, add(clx[f], crn[f]), qc[f]);
                }
                if (live && ((cf0 && i0 == 0) || (cf1 && i0 == M - 2))) {
                    float val[3];
                    if (cf0 && i0 == 0) {                           // left side, cell (0, r - 1)
                        #pragma unroll
                        for (int f = 0; f < 3; ++f) val[f] = rsub(swe_flux(0, f, ph.x, phu.x, phv.x, g), clx[f].x);
                        put_register(e, mm[0], r - 1, fine_acc, dtl, val);
                    }
                    if (cf1 && i0 == M - 2) {                       // right side, cell (M - 1, r - 1)
                        #pragma unroll
                        for (int f = 0; f < 3; ++f) val[f] = radd(swe_flux(0, f, ph.y, phu.y, phv.y, g), crn[f].y);
                        put_register(e, mm[1], r - 1, fine_acc, dtl, val);
                    }
                }
            }
            if (r <= M - 1) {
                f2 rl[6], rr[6], ow[3];
                if (subs) {
                    // waves 1 and 3 read only the right and the left neighbour
                    #pragma unroll
                    for (int k = 1; k < 6; ++k) rl[k] = lpair(rx[k]);
                    #pragma unroll
                    for (int k = 0; k < 6; ++k)
                        if (k != 2) rr[k] = rpair(rx[k]);
                    rl[0] = rr[2] = bc(0.f);
                    own<true>(rx, rl, rr, dtdx2, ow);
                } else {
                    #pragma unroll
                    for (int k = 0; k < 6; ++k) { rl[k] = lpair(rx[k]); rr[k] = rpair(rx[k]); }
                    own<false>(rx, rl, rr, dtdx2, ow);
                }
                #pragma unroll
                for (int f = 0; f < 3; ++f) vxp[f] = fma(nkk2, br[f], fma(nkk2, bl[f], ow[f]));
            }
        }

        // x-edges of row r: fluctuations (kept for row r+1), transverse parts
        // into the y-edges of rows r and r+1
        if (r >= -1 && r <= M) {
            f2 amm[3], amp[3], apm[3], app[3];
            if (subs) {
                fluct_sub(rx, amxp, apxp);
                trans_sub(rx, xinv2c, amxp, amm, amp);
                trans_sub(rx, xinv2c, apxp, apm, app);
            } else {
                fluct_gen(rx, amxp, apxp);
                trans_gen(rx, xinv2c, amxp, amm, amp);
                trans_gen(rx, xinv2c, apxp, apm, app);
            }
            #pragma unroll
            for (int f = 0; f < 3; ++f) {
                typ[f] = fma(kk2, rpair(amm[f]), fma(kk2, apm[f], tyc[f]));
                tyc[f] = fma(kk2, rpair(amp[f]), mul(kk2, app[f]));
            }
        } else {
            #pragma unroll
            for (int f = 0; f < 3; ++f) { typ[f] = tyc[f]; tyc[f] = bc(0.f); }
        }

        ph = h; phu = hu; phv = hv; pu = u; pv = v; ps = sq;
        #pragma unroll
        for (int k = 0; k < 6; ++k) { ry2[k] = ry1[k]; ry1[k] = ryc[k]; }
    }

    if (live && cols_in && (nf.x != nf.x || nf.y != nf.y)) e.ctl->nonfinite_error = 1;
    __syncwarp();
    red[lane] = live ? smax : 0.f;
    __syncwarp();
    if (live && kl == 0) {
        float mx = 0.f;
        #pragma unroll 1
        for (int k = 0; k < LP; ++k) mx = fmaxf(mx, red[seg * LP + k]);
        atomic_max_nonneg(&e.ctl->smax_bits[lev], (double)mx);
    }
    if (!next) break;
    // the next group: wait for its copies, fill the remaining ghost cells
    cp_async_wait_all();
    __syncwarp();
    dry |= warp_fill_tiles<float, M, PPW, true>(e, meta_next, tiles);
    NbMeta<float> *t = meta; meta = meta_next; meta_next = t;
    b0 = bn;
    }
    if (PIPE && __any_sync(0xffffffffu, dry) && lane == 0) e.ctl->dry_error = 1;
}

}  // namespace fc

namespace fc {

template <typename T, int M, int C>
static int launch_sweep_t(const Env<T> &e, List l, int fine_acc, cudaStream_t s)
{
    using S = SweepShape<T, M, C>;
    constexpr int W = S::W;
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(k_sweep<T, M, C, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)S::bytes);
        if (err != cudaSuccess) return cuda_status(err, "cudaFuncSetAttribute(k_sweep)");
        configured = true;
    }
    if (l.count <= 0) return FC_OK;
    constexpr int per = W * S::PPW;
    FC_CUDA(launch_pdl(k_sweep<T, M, C, W>, (l.count + per - 1) / per, 32 * W, S::bytes, s, e, l.idx, l.count, fine_acc));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <int M, bool PIPE>
static int launch_sweep2_t(const Env<float> &e, List l, int fine_acc, cudaStream_t s)
{
    using S = SweepShape<float, M, 2>;
    using L = SweepLayout<float, M, 2, PIPE>;
    constexpr int W = S::W;
    static int resident = 0;          // CTAs of this shape that fit on the device at once
    if (!resident) {
        cudaError_t err = cudaFuncSetAttribute(k_sweep2<M, W, PIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)L::bytes);
        if (err != cudaSuccess) return cuda_status(err, "cudaFuncSetAttribute(k_sweep2)");
        int dev = 0, sms = 0, per = 0;
        FC_CUDA(cudaGetDevice(&dev));
        FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep2<M, W, PIPE>, 32 * W, L::bytes));
        resident = sms * (per > 0 ? per : 1);
    }
    if (l.count <= 0) return FC_OK;
    constexpr int per = W * S::PPW;
    int grid = (l.count + per - 1) / per;
    if (PIPE && grid > resident) grid = resident;
    FC_CUDA(launch_pdl(k_sweep2<M, W, PIPE>, grid, 32 * W, L::bytes, s, e, l.idx, l.count, fine_acc));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T, int M>
int launch_sweep_m(const Env<T> &e, List l, int fine_acc, int k, cudaStream_t s)
{
    if (k == 0) return launch_sweep_t<T, M, SweepCols<M>::c[0]>(e, l, fine_acc, s);
    if constexpr (sizeof(T) == 4) {         // FP32: two columns per lane in packed form
        if (k == 1) return launch_sweep2_t<M, false>(e, l, fine_acc, s);
        return launch_sweep2_t<M, true>(e, l, fine_acc, s);
    } else {
        if (k == 1) return launch_sweep_t<T, M, SweepCols<M>::c[1]>(e, l, fine_acc, s);
        return launch_sweep_t<T, M, SweepCols<M>::c[2]>(e, l, fine_acc, s);
    }
}

}  // namespace fc
