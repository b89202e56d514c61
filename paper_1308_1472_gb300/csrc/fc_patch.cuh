// fc_patch.cuh -- device building blocks shared by the patch kernels
// (fc_kernels.cu, fc_sweep.cuh): rounding helpers, neighbour metadata, the
// ghost fill of a padded patch tile (Sec. 3: same-level copy, fine-to-coarse
// average, limited coarse-to-fine interpolation; reflecting walls), and the
// per-edge solvers of the wave-propagation update (Roe shallow water, MC
// limiter, transverse split).
//
// The ghost fill is written for a cooperating thread group: a whole CTA (one
// patch per CTA) or a single warp (several patches per CTA, one warp each).
#pragma once
#include <type_traits>

#include "fc_kernels.cuh"
#include "fc_sphere.cuh"

namespace fc {

// thread groups that fill a tile together
struct CtaGroup {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int sync_or(int v) const { return __syncthreads_or(v); }
};
struct WarpGroup {
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ int sync_or(int v) const { return __any_sync(0xffffffffu, v); }
};

// ---------------------------------------------------------------------------
// small arithmetic helpers with explicit rounding where a result must not
// depend on multiply-add contraction
template <typename T> __device__ __forceinline__ T rmul(T a, T b);
template <typename T> __device__ __forceinline__ T radd(T a, T b);
template <> __device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
template <typename T> __device__ __forceinline__ T rsub(T a, T b) { return radd(a, -b); }

// division and square root: IEEE in FP64; in FP32 the hardware approximate
// reciprocal / square root (a couple of ulp), well inside the FP32 tolerance
template <typename T> __device__ __forceinline__ T fdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
template <typename T> __device__ __forceinline__ T fsqrt(T a) { return sqrt(a); }
template <> __device__ __forceinline__ float fsqrt(float a) { return a * rsqrtf(a); }

template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a > T(0) && b > T(0)) return tmin(a, b);
    if (a < T(0) && b < T(0)) return tmax(a, b);
    return T(0);
}

// time blend (1 - a) old + a new, rounded step by step
template <typename T>
__device__ __forceinline__ T blend(T a, T vo, T vn)
{
    return radd(rmul(rsub(T(1), a), vo), rmul(a, vn));
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v)
{
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T *qbuf(const Env<T> &e, int b) { return b == 0 ? e.q[0] : (b == 1 ? e.q[1] : e.q[2]); }

// ---------------------------------------------------------------------------
// neighbour metadata of a patch, staged once per CTA in shared memory: the
// patch itself (index 8) and its neighbour(s) in each of the 8 directions,
// with coordinates, the buffers holding their level's newest and previous
// values and the time weight of the newest at this launch
template <typename T>
struct NbMeta {
    int kind;
    int id[2], x[2], y[2], bnew[2], bold[2];
    T alpha[2];
    int slot;            // complete tile of a coarser neighbour
    int cfslot;          // face entries: flux-register slot of this side of the patch, or -1
    int lev;             // level of id[0] (0 if there is none)
    const T *b0;         // newest values of neighbour id[0] (field 0), or null
};

template <typename T>
__device__ void load_meta(const Env<T> &e, int p, NbMeta<T> *meta, int t)
{
    if (t >= 9) return;
    NbMeta<T> m;
    if (t == 8) { m.kind = FC_NB_SAME; m.id[0] = p; m.id[1] = -1; }
    else {
        const int *en = e.f.nbr + (size_t)p * 32 + 4 * t;
        m.kind = en[0]; m.id[0] = en[1]; m.id[1] = en[2];
    }
    m.slot = -1;
    m.lev = 0;
    for (int k = 0; k < 2; ++k) {
        int q = m.id[k];
        if ((unsigned)q < (unsigned)e.n) {
            int l = e.f.level[q], s = e.ctl->start_buf[l], kd = e.kdone[l];
            if (k == 0) m.lev = l;
            m.x[k] = e.f.x[q]; m.y[k] = e.f.y[q];
            m.bnew[k] = kd == 0 ? s : buf_out(s, kd);
            m.bold[k] = kd == 0 ? s : buf_in(s, kd);
            m.alpha[k] = e.alpha[l];
        } else {
            m.id[k] = -1; m.x[k] = m.y[k] = 0; m.bnew[k] = m.bold[k] = 0; m.alpha[k] = T(1);
        }
    }
    if (m.kind == FC_NB_COARSER && m.id[0] >= 0) m.slot = e.grslot ? e.grslot[m.id[0]] : m.id[0];
    m.cfslot = (t < 4 && e.cfslot) ? e.cfslot[p * 4 + t] : -1;
    m.b0 = m.id[0] >= 0 ? qbuf(e, m.bnew[0]) + (size_t)m.id[0] * (e.m * e.m) : nullptr;
    meta[t] = m;
}
template <typename T>
__device__ __forceinline__ void load_meta(const Env<T> &e, int p, NbMeta<T> *meta)
{
    load_meta(e, p, meta, (int)threadIdx.x);
}

// value of cell c, field f, of neighbour k of a metadata entry at this time
template <typename T>
__device__ __forceinline__ T mval(const Env<T> &e, const NbMeta<T> &m, int k, int f, int c)
{
    size_t o = ((size_t)f * e.n + m.id[k]) * (size_t)(e.m * e.m) + c;
    T vn = qbuf(e, m.bnew[k])[o];
    if (m.alpha[k] == T(1)) return vn;
    T vo = qbuf(e, m.bold[k])[o];
    if (m.alpha[k] == T(0)) return vo;
    return blend(m.alpha[k], vo, vn);
}

// ---------------------------------------------------------------------------
// ghost fill of one patch into a padded shared-memory tile [F][(M+4)^2]
template <int M> __device__ __forceinline__ int tix(int i, int j) { return (j + 2) * (M + 4) + (i + 2); }

__device__ __forceinline__ int dir_of(int ox, int oy)
{
    if (oy == 0) return ox < 0 ? 0 : 1;
    if (ox == 0) return oy < 0 ? 2 : 3;
    return 4 + (ox > 0 ? 1 : 0) + (oy > 0 ? 2 : 0);
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// reflecting walls of the unit square: mirror the two nearest interior layers,
// normal momentum negated; x walls over the full padded height, then y walls
// over the full padded width (contains barriers: call from every thread)
template <typename T, int M, int F, typename G = CtaGroup>
__device__ __forceinline__ void apply_walls(int xp, int yp, int lp, T *tile, G grp = G{})
{
    constexpr int P = M + 4, PP = P * P;
    const int last = (1 << lp) - 1;
    const bool wx = xp == 0 || xp == last, wy = yp == 0 || yp == last;
    if (wx) {   // x walls over the full padded height, normal momentum negated
        for (int t = grp.rank(); t < P * 2 * F; t += grp.size()) {
            int j = t % P - 2, k = (t / P) % 2, f = t / (2 * P);
            T sg = (F == 3 && f == 1) ? T(-1) : T(1);
            T *A = tile + f * PP;
            if (xp == 0) A[tix<M>(-1 - k, j)] = sg * A[tix<M>(k, j)];
            if (xp == last) A[tix<M>(M + k, j)] = sg * A[tix<M>(M - 1 - k, j)];
        }
        grp.sync();
    }
    if (wy) {
        for (int t = grp.rank(); t < P * 2 * F; t += grp.size()) {
            int i = t % P - 2, k = (t / P) % 2, f = t / (2 * P);
            T sg = (F == 3 && f == 2) ? T(-1) : T(1);
            T *A = tile + f * PP;
            if (yp == 0) A[tix<M>(i, -1 - k)] = sg * A[tix<M>(i, k)];
            if (yp == last) A[tix<M>(i, M + k)] = sg * A[tix<M>(i, M - 1 - k)];
        }
        grp.sync();
    }
}

template <int M> struct Log2M { static constexpr int v = M == 8 ? 3 : (M == 16 ? 4 : 5); };

// Cubed sphere: ghost cell (i, j) of patch (tree tp, level lp, xp, yp) from
// neighbour entry m, by locating the ghost centre (or, next to a finer
// neighbour, the centres of its four quarter cells) in the neighbouring tree
// (Sec. 4 coordinate transformations).  Same-level copy, 2x2 average in the
// receiving patch's axes ((SW + SE) + (NW + NE)), or limited interpolation
// from the coarser neighbour's complete tile in that tile's own axes.
template <typename T, int M, int F>
__device__ __forceinline__ void sphere_ghost(const Env<T> &e, const NbMeta<T> &m, int tp, int lp, int xp, int yp,
                                             int i, int j, T *tile)
{
    constexpr int P = M + 4, PP = P * P, LM = Log2M<M>::v;
    const int sh = kMaxBits - lp - LM;                  // finest units per cell: 1 << sh
    const long long w = 1LL << sh;
    const long long gi = (long long)xp * M + i, gj = (long long)yp * M + j;
    const int t = tix<M>(i, j);
    long long Xm, Ym;
    if (m.kind == FC_NB_SAME || m.kind == FC_NB_COARSER) {
        if (sphere_map_point(e.conn, tp, gi * w + w / 2, gj * w + w / 2, &Xm, &Ym) < 0) { e.ctl->index_error = 1; return; }
        if (m.kind == FC_NB_SAME) {
            const int ci = (int)(Xm >> sh) - m.x[0] * M, cj = (int)(Ym >> sh) - m.y[0] * M;
            if (m.id[0] < 0 || (unsigned)ci >= (unsigned)M || (unsigned)cj >= (unsigned)M) {
                e.ctl->index_error = 1;
                return;
            }
            for (int f = 0; f < F; ++f) tile[f * PP + t] = mval(e, m, 0, f, cj * M + ci);
            return;
        }
        const long long wc = 2 * w;
        const int ci = (int)(Xm >> (sh + 1)) - m.x[0] * M, cj = (int)(Ym >> (sh + 1)) - m.y[0] * M;
        if (m.slot < 0 || (unsigned)ci >= (unsigned)M || (unsigned)cj >= (unsigned)M) {
            e.ctl->index_error = 1;
            return;
        }
        const long long cx = ((long long)m.x[0] * M + ci) * wc + wc / 2;
        const long long cy = ((long long)m.y[0] * M + cj) * wc + wc / 2;
        const T sgx = Xm > cx ? T(0.25) : T(-0.25), sgy = Ym > cy ? T(0.25) : T(-0.25);
        const T *ct = e.gr + (size_t)m.slot * F * PP;
        for (int f = 0; f < F; ++f) {
            const T *A = ct + f * PP;
            T qc = A[tix<M>(ci, cj)];
            T sx = minmod(A[tix<M>(ci + 1, cj)] - qc, qc - A[tix<M>(ci - 1, cj)]);
            T sy = minmod(A[tix<M>(ci, cj + 1)] - qc, qc - A[tix<M>(ci, cj - 1)]);
            tile[f * PP + t] = radd(radd(qc, rmul(sgx, sx)), rmul(sgy, sy));
        }
        return;
    }
    // finer: quarter cells (a, b) in this patch's axes
    const long long wf = w / 2;
    T val[F][2][2];
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            if (sphere_map_point(e.conn, tp, (2 * gi + a) * wf + wf / 2, (2 * gj + b) * wf + wf / 2, &Xm, &Ym) < 0) {
                e.ctl->index_error = 1;
                return;
            }
            const int fx = (int)(Xm >> (sh - 1)), fy = (int)(Ym >> (sh - 1));
            int k = -1;
            for (int kk = 0; kk < 2; ++kk)
                if (m.id[kk] >= 0 && (fx >> LM) == m.x[kk] && (fy >> LM) == m.y[kk]) k = kk;
            if (k < 0) { e.ctl->index_error = 1; return; }
            const int c = (fy - m.y[k] * M) * M + (fx - m.x[k] * M);
            for (int f = 0; f < F; ++f) val[f][b][a] = mval(e, m, k, f, c);
        }
    for (int f = 0; f < F; ++f)
        tile[f * PP + t] = T(0.25) * ((val[f][0][0] + val[f][0][1]) + (val[f][1][0] + val[f][1][1]));
}

// Square / periodic square: ghost cell (i, j) of the patch at (xp, yp, level
// lp) from neighbour entry m (direction d): same-level copy, 2x2 average of a
// finer neighbour ((SW + SE) + (NW + NE)), or limited interpolation from the
// coarser neighbour's complete tile.  Returns 1 if a depth is not positive.
template <typename T, int M, int F>
__device__ __forceinline__ int cart_ghost(const Env<T> &e, const NbMeta<T> &m, int d, int i, int j, int xp, int yp,
                                          int lp, T *tile)
{
    constexpr int PP = (M + 4) * (M + 4);
    const int W = (1 << lp) * M;
    const bool periodic = e.conn == FC_CONN_PERIODIC;
    const int kind = m.kind;
    int bad = 0;
    int t = tix<M>(i, j);
    if (kind == FC_NB_SAME && m.alpha[0] == T(1) && m.b0) {
        // same-level neighbour at this time: cell (i - ox M, j - oy M) of it
        const int ox = i < 0 ? -1 : (i >= M ? 1 : 0), oy = j < 0 ? -1 : (j >= M ? 1 : 0);
        const T *src = m.b0 + (j - oy * M) * M + (i - ox * M);
        const size_t fs = (size_t)e.n * (M * M);
        T v[F];
        #pragma unroll
        for (int f = 0; f < F; ++f) v[f] = src[f * fs];
        #pragma unroll
        for (int f = 0; f < F; ++f) tile[f * PP + t] = v[f];
        return F == 3 && !(v[0] > T(0));
    }
    // every field's loads are issued before the first store into the tile
    // (the source pointers are generic, so a store in between would order
    // the loads of the next field behind it)
    T v[F];
    int gi = xp * M + i, gj = yp * M + j;
    if (periodic) { gi = (gi + W) % W; gj = (gj + W) % W; }
    if (kind == FC_NB_SAME) {
        int ci = gi - m.x[0] * M, cj = gj - m.y[0] * M;
        if (m.id[0] < 0 || (unsigned)ci >= (unsigned)M || (unsigned)cj >= (unsigned)M) {
            e.ctl->index_error = 1;
            return bad;
        }
        #pragma unroll
        for (int f = 0; f < F; ++f) v[f] = mval(e, m, 0, f, cj * M + ci);
    } else if (kind == FC_NB_FINER) {
        int k = d < 2 ? (j >= M / 2) : (d < 4 ? (i >= M / 2) : 0);
        int fi = 2 * gi - m.x[k] * M, fj = 2 * gj - m.y[k] * M;
        if (m.id[k] < 0 || (unsigned)fi >= (unsigned)(M - 1) || (unsigned)fj >= (unsigned)(M - 1)) {
            e.ctl->index_error = 1;
            return bad;
        }
        int c00 = fj * M + fi;
        #pragma unroll
        for (int f = 0; f < F; ++f) {
            T a00 = mval(e, m, k, f, c00), a10 = mval(e, m, k, f, c00 + 1);
            T a01 = mval(e, m, k, f, c00 + M), a11 = mval(e, m, k, f, c00 + M + 1);
            v[f] = T(0.25) * ((a00 + a10) + (a01 + a11));
        }
    } else {                                    // coarser: limited linear interpolation
        int ci = (gi >> 1) - m.x[0] * M, cj = (gj >> 1) - m.y[0] * M;
        if (m.slot < 0 || (unsigned)ci >= (unsigned)M || (unsigned)cj >= (unsigned)M) {
            e.ctl->index_error = 1;
            return bad;
        }
        T sgx = (gi & 1) ? T(0.25) : T(-0.25), sgy = (gj & 1) ? T(0.25) : T(-0.25);
        const T *ct = e.gr + (size_t)m.slot * F * PP;
        #pragma unroll
        for (int f = 0; f < F; ++f) {
            const T *A = ct + f * PP;
            T qc = A[tix<M>(ci, cj)];
            T sx = minmod(A[tix<M>(ci + 1, cj)] - qc, qc - A[tix<M>(ci - 1, cj)]);
            T sy = minmod(A[tix<M>(ci, cj + 1)] - qc, qc - A[tix<M>(ci, cj - 1)]);
            v[f] = radd(radd(qc, rmul(sgx, sx)), rmul(sgy, sy));
        }
    }
    #pragma unroll
    for (int f = 0; f < F; ++f) tile[f * PP + t] = v[f];
    return F == 3 && !(v[0] > T(0));
}

// Fills interior + two ghost layers.  Returns nonzero in every thread of the
// CTA if some depth in the tile is not positive (shallow water only).  SG:
// cubed-sphere ghost rules (compiled only into the sphere's kernels, so the
// square's kernels keep their register budget).
template <typename T, int M, int F, bool SG, typename G = CtaGroup>
__device__ int gather_tile(const Env<T> &e, const NbMeta<T> *meta, T *tile, G grp = G{})
{
    constexpr int P = M + 4, PP = P * P, MM = M * M;
    const NbMeta<T> &me = meta[8];
    const int p = me.id[0], xp = me.x[0], yp = me.y[0];
    const int lp = me.lev;
    int bad = 0;
    // interior: 16-byte vector loads when the patch's own level needs no blend
    if (me.alpha[0] == T(1)) {
        using V = typename Vec16<T>::type;
        constexpr int NV = Vec16<T>::n, PER = MM / NV;
        const T *src = qbuf(e, me.bnew[0]);
        for (int v = grp.rank(); v < F * PER; v += grp.size()) {
            int f = v / PER, c = (v % PER) * NV;
            V w = *reinterpret_cast<const V *>(src + ((size_t)f * e.n + p) * MM + c);
            const T *ws = reinterpret_cast<const T *>(&w);
            int i = c % M, j = c / M;
            T *dst = tile + f * PP + tix<M>(i, j);
            for (int k = 0; k < NV; ++k) {
                dst[k] = ws[k];
                if (F == 3 && f == 0 && !(ws[k] > T(0))) bad = 1;
            }
        }
    } else {
        // between the level's steps: both time levels as 16-byte vectors (both
        // loads in flight), blended per component as mval does
        using V = typename Vec16<T>::type;
        constexpr int NV = Vec16<T>::n, PER = MM / NV;
        const T a = me.alpha[0];
        const T *srcn = qbuf(e, me.bnew[0]), *srco = qbuf(e, me.bold[0]);
        for (int v = grp.rank(); v < F * PER; v += grp.size()) {
            int f = v / PER, c = (v % PER) * NV;
            const size_t o = ((size_t)f * e.n + p) * MM + c;
            const V wo = *reinterpret_cast<const V *>(srco + o), wn = *reinterpret_cast<const V *>(srcn + o);
            const T *po = reinterpret_cast<const T *>(&wo), *pn = reinterpret_cast<const T *>(&wn);
            T *dst = tile + f * PP + tix<M>(c % M, c / M);
            for (int k = 0; k < NV; ++k) {
                const T w = a == T(0) ? po[k] : blend(a, po[k], pn[k]);
                dst[k] = w;
                if (F == 3 && f == 0 && !(w > T(0))) bad = 1;
            }
        }
    }
    // ghost ring: rows -2,-1 and M,M+1 over the full padded width, then the
    // columns -2,-1,M,M+1 of rows 0..M-1
    for (int g = grp.rank(); g < 8 * M + 16; g += grp.size()) {
        int i, j;
        if (g < 2 * P) { j = -2 + g / P; i = g % P - 2; }
        else if (g < 4 * P) { int h = g - 2 * P; j = M + h / P; i = h % P - 2; }
        else { int h = g - 4 * P; j = h >> 2; int c = h & 3; i = c < 2 ? c - 2 : M + c - 2; }
        int ox = i < 0 ? -1 : (i >= M ? 1 : 0), oy = j < 0 ? -1 : (j >= M ? 1 : 0);
        const NbMeta<T> &m = meta[dir_of(ox, oy)];
        int kind = m.kind;
        if (kind == FC_NB_NONE) continue;            // wall: filled by reflection below
        if constexpr (SG) {
            sphere_ghost<T, M, F>(e, m, e.f.tree[p], lp, xp, yp, i, j, tile);
            continue;
        }
        bad |= cart_ghost<T, M, F>(e, m, dir_of(ox, oy), i, j, xp, yp, lp, tile);
    }
    bad = grp.sync_or(bad);
    if constexpr (SG) {
        // beyond a cube corner (three trees meet, no diagonal neighbour): the
        // mean of the face ghosts of the same row and of the same column
        for (int g = grp.rank(); g < 16; g += grp.size()) {
            int c = g >> 2, i = (c & 1) ? M + (g & 1) : -1 - (g & 1), j = (c & 2) ? M + ((g >> 1) & 1) : -1 - ((g >> 1) & 1);
            if (meta[4 + c].kind != FC_NB_NONE) continue;
            int ic = i < 0 ? 0 : M - 1, jc = j < 0 ? 0 : M - 1;
            for (int f = 0; f < F; ++f)
                tile[f * PP + tix<M>(i, j)] = T(0.5) * (tile[f * PP + tix<M>(i, jc)] + tile[f * PP + tix<M>(ic, j)]);
        }
        grp.sync();
        return bad;
    }
    if (e.conn != FC_CONN_SQUARE) return bad;
    apply_walls<T, M, F, G>(xp, yp, lp, tile, grp);
    return bad;
}

// ---------------------------------------------------------------------------
// edge solvers in the edge frame (h, normal momentum, transverse momentum)
//
// shallow water, Roe linearisation: u_hat, v_hat sqrt(h)-weighted averages,
// c_hat = sqrt(g (hL + hR)/2); waves a_p r_p with r1 = (1, u - c, v),
// r2 = (0, 0, 1), r3 = (1, u + c, v) and speeds u - c, u, u + c.
// Record layout: {a1, a2, a3, u_hat, v_hat, c_hat}.
// fluctuations amdq, apdq of an edge record (edge frame), from the wave
// strengths and speeds directly: sum over waves of min(s,0) W and max(s,0) W
// Subsonic edge (|u| < c, so s1 < 0 < s3): the left-going wave is wave 1, the
// right-going wave 3, and wave 2 goes with the sign of u; every min/max of the
// general form then selects a known operand: the same values up to the order in
// which products are rounded.  The form is chosen per warp, so the rounding of
// an edge can depend on the launch shape (results agree to ~1e-16 relative).
template <typename T>
__device__ __forceinline__ void swe_fluct_sub(const T *rec, T *am, T *ap)
{
    T u = rec[3], v = rec[4], c = rec[5];
    T s1 = u - c, s3 = u + c;
    T m1 = s1 * rec[0], p3 = s3 * rec[2];
    T w2 = u * rec[1];
    T m2 = u < T(0) ? w2 : T(0), p2 = u > T(0) ? w2 : T(0);
    am[0] = m1; am[1] = m1 * s1; am[2] = m1 * v + m2;
    ap[0] = p3; ap[1] = p3 * s3; ap[2] = p3 * v + p2;
}

template <typename T>
__device__ __forceinline__ void swe_fluct(const T *rec, T *am, T *ap)
{
    T u = rec[3], v = rec[4], c = rec[5];
    T s1 = u - c, s3 = u + c;
    T m1 = tmin(s1, T(0)) * rec[0], m2 = tmin(u, T(0)) * rec[1], m3 = tmin(s3, T(0)) * rec[2];
    T p1 = tmax(s1, T(0)) * rec[0], p2 = tmax(u, T(0)) * rec[1], p3 = tmax(s3, T(0)) * rec[2];
    am[0] = m1 + m3; am[1] = m1 * s1 + m3 * s3; am[2] = (m1 + m3) * v + m2;
    ap[0] = p1 + p3; ap[1] = p1 * s1 + p3 * s3; ap[2] = (p1 + p3) * v + p2;
}

// split a fluctuation d (edge frame) along the other direction's eigenvectors
// at this edge's averages: speeds (v - c, v, v + c), r1 = (1, u, v - c),
// r2 = (0, 1, 0), r3 = (1, u, v + c)
template <typename T>
__device__ __forceinline__ void swe_trans(const T *rec, const T *d, T *bm, T *bp)
{
    T u = rec[3], v = rec[4], c = rec[5];
    T inv2c = fdiv(T(0.5), c);
    T b1 = ((v + c) * d[0] - d[2]) * inv2c;
    T b2 = d[1] - u * d[0];
    T b3 = (d[2] - (v - c) * d[0]) * inv2c;
    T l1 = v - c, l3 = v + c;
    T m1 = tmin(l1, T(0)), p1 = tmax(l1, T(0)), m2 = tmin(v, T(0)), p2 = tmax(v, T(0));
    T m3 = tmin(l3, T(0)), p3 = tmax(l3, T(0));
    bm[0] = m1 * b1 + m3 * b3;
    bm[1] = (m1 * b1 * u + m2 * b2) + m3 * b3 * u;
    bm[2] = m1 * b1 * l1 + m3 * b3 * l3;
    bp[0] = p1 * b1 + p3 * b3;
    bp[1] = (p1 * b1 * u + p2 * b2) + p3 * b3 * u;
    bp[2] = p1 * b1 * l1 + p3 * b3 * l3;
}

// transverse split when |v| < c: the down-going part is eigenvector 1, the
// up-going part eigenvector 3, eigenvector 2 goes with the sign of v
template <typename T>
__device__ __forceinline__ void swe_trans_sub(const T *rec, const T *d, T *bm, T *bp)
{
    T u = rec[3], v = rec[4], c = rec[5];
    T inv2c = fdiv(T(0.5), c);
    T l1 = v - c, l3 = v + c;
    T b1 = ((v + c) * d[0] - d[2]) * inv2c;
    T b2 = d[1] - u * d[0];
    T b3 = (d[2] - l1 * d[0]) * inv2c;
    T g1 = l1 * b1, g3 = l3 * b3, g2 = v * b2;
    T m2 = v < T(0) ? g2 : T(0), p2 = v > T(0) ? g2 : T(0);
    bm[0] = g1; bm[1] = g1 * u + m2; bm[2] = g1 * l1;
    bp[0] = g3; bp[1] = p2 + g3 * u; bp[2] = g3 * l3;
}

template <typename T>
__device__ __forceinline__ void swe_roe(T hL, T nL, T tL, T uL, T vL, T sqL, T hR, T nR, T tR, T uR, T vR, T sqR,
                                        T g, T *rec)
{
    T inv = fdiv(T(1), sqL + sqR);
    T u = (sqL * uL + sqR * uR) * inv;
    T v = (sqL * vL + sqR * vR) * inv;
    T c = fsqrt(g * (T(0.5) * (hL + hR)));
    T d0 = hR - hL, d1 = nR - nL, d2 = tR - tL;
    T inv2c = fdiv(T(0.5), c);
    rec[0] = ((u + c) * d0 - d1) * inv2c;
    rec[1] = d2 - v * d0;
    rec[2] = (d1 - (u - c) * d0) * inv2c;
    rec[3] = u; rec[4] = v; rec[5] = c;
}

// Harten-Hyman entropy fix of an edge's fluctuations (edge frame).  With
// W1 = a1 (1, u - c, v), W2 = a2 (0, 0, 1), W3 = a3 (1, u + c, v): the 1-wave
// is a transonic rarefaction when the normal characteristic speed n/h - c is
// negative in the left state and positive in qL + W1, the 3-wave when
// n/h + c is negative in qR - W3 and positive in the right state.  Such a
// wave with Roe speed s and end speeds l0 < 0 < l1 contributes
// l0 beta W to A-dQ and l1 (1 - beta) W to A+dQ, beta = (l1 - s) / (l1 - l0);
// the other waves contribute min(s, 0) W and max(s, 0) W.  am / ap are
// replaced only when a wave is transonic.
template <typename T>
__device__ __forceinline__ void swe_efix(const T *rec, T hL, T nL, T hR, T nR, T g, T *am, T *ap)
{
    const T a1 = rec[0], a2 = rec[1], a3 = rec[2], u = rec[3], v = rec[4], c = rec[5];
    const T s1 = u - c, s3 = u + c;
    const T l10 = nL / hL - sqrt(g * hL);
    const T hm1 = hL + a1, l11 = (nL + a1 * s1) / hm1 - sqrt(g * hm1);
    const T l31 = nR / hR + sqrt(g * hR);
    const T hm3 = hR - a3, l30 = (nR - a3 * s3) / hm3 + sqrt(g * hm3);
    const bool t1 = l10 < T(0) && l11 > T(0), t3 = l30 < T(0) && l31 > T(0);
    if (!t1 && !t3) return;
    // per-wave left / right speed factors
    T m1, p1, m3, p3;
    if (t1) { const T b = (l11 - s1) / (l11 - l10); m1 = l10 * b; p1 = l11 * (T(1) - b); }
    else { m1 = tmin(s1, T(0)); p1 = tmax(s1, T(0)); }
    if (t3) { const T b = (l31 - s3) / (l31 - l30); m3 = l30 * b; p3 = l31 * (T(1) - b); }
    else { m3 = tmin(s3, T(0)); p3 = tmax(s3, T(0)); }
    const T m2 = tmin(u, T(0)), p2 = tmax(u, T(0));
    am[0] = m1 * a1 + m3 * a3;
    am[1] = m1 * (a1 * s1) + m3 * (a3 * s3);
    am[2] = (m1 * (a1 * v) + m2 * a2) + m3 * (a3 * v);
    ap[0] = p1 * a1 + p3 * a3;
    ap[1] = p1 * (a1 * s1) + p3 * (a3 * s3);
    ap[2] = (p1 * (a1 * v) + p2 * a2) + p3 * (a3 * v);
}

__device__ __forceinline__ float mc_phi(float th) { return fmaxf(0.f, fminf(fminf(0.5f * (1.f + th), 2.f), 2.f * th)); }
__device__ __forceinline__ double mc_phi(double th) { return fmax(0.0, fmin(fmin(0.5 * (1.0 + th), 2.0), 2.0 * th)); }

// MC-limited own correction of an edge (edge frame), times 0.5.  Shallow
// water: waves 1 and 3 are a (1, s, v) with s = u -/+ c, wave 2 is a (0, 0, 1),
// so W.W and W_up.W follow from the strengths and averages directly.
template <typename T, int EQ>
__device__ __forceinline__ void own_correction(const T *rec, const T *recL, const T *recR, T dtdx, T *out)
{
    if constexpr (EQ == FC_EQ_SWE) {
        const T u = rec[3], v = rec[4], c = rec[5];
        T kc[3];
        #pragma unroll
        for (int p = 0; p < 3; ++p) {
            const T sgn = p == 0 ? T(-1) : T(1);
            const T s = p == 1 ? u : u + sgn * c;
            const bool left = s >= T(0);         // upwind edge: select values, not arrays
            const T a = rec[p], au = left ? recL[p] : recR[p];
            T ww, wu;
            if (p == 1) { ww = a * a; wu = au * a; }
            else {
                const T su = (left ? recL[3] : recR[3]) + sgn * (left ? recL[5] : recR[5]);
                const T vu = left ? recL[4] : recR[4];
                ww = a * a * ((T(1) + s * s) + v * v);
                wu = au * a * ((T(1) + su * s) + vu * v);
            }
            T phi = ww != T(0) ? mc_phi(fdiv(wu, ww)) : T(0);
            T as = fabs(s);
            kc[p] = (as * (T(1) - dtdx * as)) * (phi * a);
        }
        const T s1 = u - c, s3 = u + c;
        out[0] = T(0.5) * (kc[0] + kc[2]);
        out[1] = T(0.5) * (kc[0] * s1 + kc[2] * s3);
        out[2] = T(0.5) * ((kc[0] + kc[2]) * v + kc[1]);
    } else {
        T w = rec[0], s = rec[1];
        T wu = s >= T(0) ? recL[0] : recR[0];
        T phi = w * w != T(0) ? mc_phi(fdiv(wu * w, w * w)) : T(0);
        T as = fabs(s);
        out[0] = T(0.5) * ((as * (T(1) - dtdx * as)) * (phi * w));
    }
}

// block-wide maximum of non-negative values (valid in thread 0)
template <int NT, typename V>
__device__ __forceinline__ V block_max(V v, V *red)
{
    for (int o = 16; o > 0; o >>= 1) v = tmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < NT / 32 ? red[lane] : V(0);
        for (int o = 16; o > 0; o >>= 1) v = tmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// ---------------------------------------------------------------------------
// geometry helpers of the square
__device__ __forceinline__ double level_dx(int level, int m) { return 1.0 / ((double)(1 << level) * m); }

// asynchronous global-to-shared copies (per-thread cp.async)
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// NbMeta of one record entry, in two parts.  meta_static: the fields that stay
// fixed while the forest does (kind, ids, positions, the coarse-tile slot from
// this launch's slot map -- fills into a scratch tile buffer, for tagging and
// regrid, use their own map -- and the register slot), with the level of each
// id kept in bnew until meta_time sets the time fields from the launch: the
// buffers of the level's current and previous states and the time weight.
template <typename T>
__device__ __forceinline__ void meta_static(const Env<T> &e, const int *r, int t, NbMeta<T> &m)
{
    // the loads of the record, then the loads that depend on it, are each
    // issued together
    const int r0 = r[0], id0 = r[1], id1 = r[2], xy0 = r[4], xy1 = r[5];
    const int p = (r - 6 * t)[6 * 8 + 1];                                // the record's own entry
    m.kind = r0 & 0xff;
    m.id[0] = id0; m.id[1] = id1;
    m.slot = (m.kind == FC_NB_COARSER && id0 >= 0) ? (e.grslot ? e.grslot[id0] : id0) : -1;
    m.cfslot = (t < 4 && e.cfslot) ? e.cfslot[p * 4 + t] : -1;
    m.lev = (unsigned)id0 < (unsigned)e.n ? (r0 >> 8) & 0xff : 0;
    #pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int q = k ? id1 : id0;
        if ((unsigned)q < (unsigned)e.n) {
            const int xy = k ? xy1 : xy0;
            m.x[k] = xy & 0xffff; m.y[k] = xy >> 16;
            m.bnew[k] = (r0 >> (8 + 8 * k)) & 0xff;                       // level, until meta_time
        } else {
            m.id[k] = -1; m.x[k] = m.y[k] = 0; m.bnew[k] = 0;
        }
    }
}
template <typename T>
__device__ __forceinline__ void meta_time(const Env<T> &e, const int *sbuf, NbMeta<T> &m)
{
    #pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (m.id[k] >= 0) {
            const int l = m.bnew[k], s0 = sbuf[l], kd = e.kdone[l];
            m.bnew[k] = kd == 0 ? s0 : buf_out(s0, kd);
            m.bold[k] = kd == 0 ? s0 : buf_in(s0, kd);
            m.alpha[k] = e.alpha[l];
        } else {
            m.bnew[k] = m.bold[k] = 0; m.alpha[k] = T(1);
        }
    }
    m.b0 = m.id[0] >= 0 ? qbuf(e, m.bnew[0]) + (size_t)m.id[0] * (e.m * e.m) : nullptr;
}
template <typename T>
__device__ __forceinline__ void meta_from_rec(const Env<T> &e, const int *r, const int *sbuf, int t, NbMeta<T> &out)
{
    NbMeta<T> m;
    meta_static(e, r, t, m);
    meta_time(e, sbuf, m);
    out = m;
}

// cell (i, j) of ghost-ring entry gg (0 .. 8M+15) of a padded tile: rows
// -2, -1 and M, M+1 over the padded width, then columns -2, -1, M, M+1 of
// rows 0..M-1
template <int M>
__device__ __forceinline__ void ghost_ring_ij(int gg, int &i, int &j)
{
    constexpr int P = M + 4;
    if (gg < 2 * P) { j = -2 + gg / P; i = gg % P - 2; }
    else if (gg < 4 * P) { const int h = gg - 2 * P; j = M + h / P; i = h % P - 2; }
    else { const int h = gg - 4 * P; j = h >> 2; const int c = h & 3; i = c < 2 ? c - 2 : M + c - 2; }
}

// Ghost fill of the PPW patches of one warp at once (the same values as
// gather_tile): the interiors, then the ghost cells of same-level neighbours
// at their own time with all loads issued before any is used, then the other
// ghost cells (finer and coarser neighbours), then the walls.  meta holds
// 9 * PPW entries; returns nonzero in every lane if a depth is not positive.
template <typename T, int M, int PPW, bool PRE = false>
__device__ int warp_fill_tiles(const Env<T> &e, const NbMeta<T> *meta, T *tiles)
{
    constexpr int F = 3, P = M + 4, PP = P * P, MM = M * M, NG = 8 * M + 16;
    using V = typename Vec16<T>::type;
    constexpr int NV = Vec16<T>::n, PER = MM / NV;
    const int lane = threadIdx.x & 31;
    const size_t fs = (size_t)e.n * MM;
    int bad = 0;
    // interiors (the updated level is at its own time: weight 1); with PRE
    // the interiors and the same-level ghost cells are in place already
    // (copied by prefetch_row) and their depths are checked by the caller
    constexpr int NI = PRE ? 0 : PPW * F * PER, NIT = (NI + 31) / 32;
    auto ghost_ij = [](int gg, int &i, int &j) { ghost_ring_ij<M>(gg, i, j); };
    constexpr int NGT = PPW * NG, NGIT = (NGT + 31) / 32;
    // Every load of the interiors and of the same-level ghost cells is
    // issued before the first store into the tiles (the source pointers are
    // generic, so a store in between would order the loads behind it).
    const T *src[PRE ? 1 : NGIT];
    if constexpr (!PRE) {
        #pragma unroll
        for (int it = 0; it < NGIT; ++it) {
            const int g = lane + 32 * it;
            src[it] = nullptr;
            if (g < NGT) {
                const int s = g / NG;
                int i, j;
                ghost_ij(g - s * NG, i, j);
                const int ox = i < 0 ? -1 : (i >= M ? 1 : 0), oy = j < 0 ? -1 : (j >= M ? 1 : 0);
                const NbMeta<T> &m = meta[9 * s + dir_of(ox, oy)];
                if (m.kind == FC_NB_SAME && m.alpha[0] == T(1) && m.b0) src[it] = m.b0 + (j - oy * M) * M + (i - ox * M);
            }
        }
    }
    V win[NIT > 0 ? NIT : 1];
    #pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int v = lane + 32 * it;
        if (v < NI) {
            const int s = v / (F * PER), rr = v - s * (F * PER), f = rr / PER, c = (rr - f * PER) * NV;
            const NbMeta<T> &me = meta[9 * s + 8];
            if (me.alpha[0] == T(1)) win[it] = *reinterpret_cast<const V *>(me.b0 + f * fs + c);
        }
    }
    T val[PRE ? 1 : NGIT][F];
    if constexpr (!PRE) {
        #pragma unroll
        for (int it = 0; it < NGIT; ++it)
            if (src[it])
                #pragma unroll
                for (int f = 0; f < F; ++f) val[it][f] = src[it][f * fs];
    }
    // interiors (the updated level is at its own time: weight 1); with PRE
    // the interiors and the same-level ghost cells are in place already
    // (copied by prefetch_row) and their depths are checked by the caller
    #pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int v = lane + 32 * it;
        if (v < NI) {
            const int s = v / (F * PER), rr = v - s * (F * PER), f = rr / PER, c = (rr - f * PER) * NV;
            const NbMeta<T> &me = meta[9 * s + 8];
            T *dst = tiles + s * F * PP + f * PP + tix<M>(c % M, c / M);
            if (me.alpha[0] == T(1)) {
                const V w = win[it];
                const T *ws = reinterpret_cast<const T *>(&w);
                #pragma unroll
                for (int k = 0; k < NV; ++k) {
                    dst[k] = ws[k];
                    if (f == 0 && !(ws[k] > T(0))) bad = 1;
                }
            } else {               // a level between its steps: time blend
                #pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const T w = mval(e, me, 0, f, c + k);
                    dst[k] = w;
                    if (f == 0 && !(w > T(0))) bad = 1;
                }
            }
        }
    }
    if constexpr (PRE) {
        // only the ghost cells that prefetch_row did not copy
        #pragma unroll 1
        for (int g = lane; g < NGT; g += 32) {
            const int s = g / NG;
            int i, j;
            ghost_ij(g - s * NG, i, j);
            const int ox = i < 0 ? -1 : (i >= M ? 1 : 0), oy = j < 0 ? -1 : (j >= M ? 1 : 0), d = dir_of(ox, oy);
            const NbMeta<T> &m = meta[9 * s + d];
            if (m.kind == FC_NB_NONE || (m.kind == FC_NB_SAME && m.alpha[0] == T(1) && m.b0)) continue;
            const NbMeta<T> &me = meta[9 * s + 8];
            bad |= cart_ghost<T, M, F>(e, m, d, i, j, me.x[0], me.y[0], me.lev, tiles + s * F * PP);
        }
    } else {
        #pragma unroll
        for (int it = 0; it < NGIT; ++it) {
            const int g = lane + 32 * it;
            if (g >= NGT) continue;
            const int s = g / NG;
            int i, j;
            ghost_ij(g - s * NG, i, j);
            T *tile = tiles + s * F * PP;
            if (src[it]) {
                #pragma unroll
                for (int f = 0; f < F; ++f) tile[f * PP + tix<M>(i, j)] = val[it][f];
                if (!(val[it][0] > T(0))) bad = 1;
            } else {
                const int ox = i < 0 ? -1 : (i >= M ? 1 : 0), oy = j < 0 ? -1 : (j >= M ? 1 : 0), d = dir_of(ox, oy);
                const NbMeta<T> &m = meta[9 * s + d];
                const NbMeta<T> &me = meta[9 * s + 8];
                if (m.kind != FC_NB_NONE)
                    bad |= cart_ghost<T, M, F>(e, m, d, i, j, me.x[0], me.y[0], me.lev, tile);
            }
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
    if (e.conn == FC_CONN_SQUARE) {
        #pragma unroll 1
        for (int s = 0; s < PPW; ++s) {
            const NbMeta<T> &me = meta[9 * s + 8];
            apply_walls<T, M, F, WarpGroup>(me.x[0], me.y[0], me.lev, tiles + s * F * PP, WarpGroup{});
        }
    }
    return bad;
}

// Ghost fill of the PPW patches of one warp for the two-column FP32 row
// sweep, by tile columns: the lane that sweeps columns i0, i0 + 1 of a patch
// (i0 = 2 kl - 2) copies those two columns of every padded row with 8-byte
// asynchronous copies, from the patch itself or from the same-level
// neighbour at its own time that holds them (one source per band of rows:
// below, the patch, above); the remaining ghost cells (finer and coarser
// neighbours) are computed while the copies are in flight, the walls after
// them.  The same tile values as warp_fill_tiles; returns nonzero in every
// lane if a depth in the tiles is not positive.  tiles: FP32 tiles 8 bytes
// past a 16-byte boundary (every column pair is 8-byte aligned).
template <int M, int PPW>
__device__ int warp_fill_cols(const Env<float> &e, const NbMeta<float> *meta, float *tiles, int seg, int kl,
                              bool idle)
{
    constexpr int P = M + 4, PP = P * P, LP = P / 2;
    const size_t fs = (size_t)e.n * (M * M);
    const int i0 = 2 * kl - 2;
    const int ox = kl == 0 ? -1 : (kl == LP - 1 ? 1 : 0);
    float *tile = tiles + seg * 3 * PP;
    if (!idle) {
        #pragma unroll
        for (int band = 0; band < 3; ++band) {
            const int oy = band - 1, j0 = band == 0 ? -2 : (band == 1 ? 0 : M), nj = band == 1 ? M : 2;
            const NbMeta<float> &m = meta[9 * seg + (ox == 0 && oy == 0 ? 8 : dir_of(ox, oy))];
            if (m.kind != FC_NB_SAME || m.alpha[0] != 1.f || !m.b0) continue;
            const float *src = m.b0 + (j0 - oy * M) * M + (i0 - ox * M);
            float *dst = tile + (j0 + 2) * P + (i0 + 2);
            #pragma unroll 1
            for (int j = 0; j < nj; ++j)
                #pragma unroll
                for (int f = 0; f < 3; ++f) cp_async8(dst + f * PP + j * P, src + f * fs + j * M);
        }
    }
    cp_async_commit();
    // meanwhile the ghost cells of finer and coarser neighbours, if the
    // warp's patches have any (they read no tile cell)
    constexpr int NG = 8 * M + 16, NGT = PPW * NG;
    bool other = false;
    for (int k = threadIdx.x & 31; k < 9 * PPW; k += 32) {
        const NbMeta<float> &m = meta[k];
        if (k % 9 != 8 && m.kind != FC_NB_NONE && !(m.kind == FC_NB_SAME && m.alpha[0] == 1.f && m.b0)) other = true;
    }
    int bad = 0;
    if (__any_sync(0xffffffffu, other)) {
        #pragma unroll 1
        for (int g = threadIdx.x & 31; g < NGT; g += 32) {
            const int s = g / NG;
            int i, j;
            ghost_ring_ij<M>(g - s * NG, i, j);
            const int gx = i < 0 ? -1 : (i >= M ? 1 : 0), gy = j < 0 ? -1 : (j >= M ? 1 : 0), d = dir_of(gx, gy);
            const NbMeta<float> &m = meta[9 * s + d];
            if (m.kind == FC_NB_NONE || (m.kind == FC_NB_SAME && m.alpha[0] == 1.f && m.b0)) continue;
            const NbMeta<float> &me = meta[9 * s + 8];
            bad |= cart_ghost<float, M, 3>(e, m, d, i, j, me.x[0], me.y[0], me.lev, tiles + s * 3 * PP);
        }
    }
    cp_async_wait_all();
    __syncwarp();
    if (e.conn == FC_CONN_SQUARE) {
        #pragma unroll 1
        for (int s = 0; s < PPW; ++s) {
            const NbMeta<float> &me = meta[9 * s + 8];
            apply_walls<float, M, 3, WarpGroup>(me.x[0], me.y[0], me.lev, tiles + s * 3 * PP, WarpGroup{});
        }
    }
    // depths of the copied cells (and of the rest): the lane's column pair
    if (!idle) {
        const float *t = tile + (i0 + 2);
        #pragma unroll 4
        for (int j = 0; j < P; ++j) {
            const float2 h = *reinterpret_cast<const float2 *>(t + j * P);
            if (!(h.x > 0.f) || !(h.y > 0.f)) bad = 1;
        }
    }
    return __any_sync(0xffffffffu, bad);
}

// metadata of a warp's PPW patches b0 .. b0 + PPW - 1 (slots past the end of
// the list repeat the last patch) from the static neighbour records; with
// STATIC only the fields that stay fixed while the forest does (the time
// fields follow with warp_meta_time)
template <typename T, int PPW, bool STATIC = false>
__device__ void warp_load_meta(const Env<T> &e, const int *list, int count, int b0, NbMeta<T> *meta)
{
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < 9 * PPW; k += 32) {
        const int s = k / 9, t = k - 9 * s, b = min(b0 + s, count - 1);
        const int p = list ? list[b] : b;
        if constexpr (STATIC) {
            NbMeta<T> m;
            meta_static(e, e.nbrec + (size_t)p * kRecInts + 6 * t, t, m);
            meta[k] = m;
        } else {
            meta_from_rec(e, e.nbrec + (size_t)p * kRecInts + 6 * t, e.ctl->start_buf, t, meta[k]);
        }
    }
    __syncwarp();
}
template <typename T, int PPW>
__device__ void warp_meta_time(const Env<T> &e, NbMeta<T> *meta)
{
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < 9 * PPW; k += 32) {
        NbMeta<T> m = meta[k];
        meta_time(e, e.ctl->start_buf, m);
        meta[k] = m;
    }
    __syncwarp();
}

// Asynchronous copies of padded row j (-2 .. M+1) of the tiles of a warp's
// PPW patches: the part of the row that comes unchanged from the patch
// itself or from a same-level neighbour at its own time (16-byte pieces of
// the M middle cells, 2-cell pieces of the ghost columns); the rest of the
// row is left to warp_fill_tiles<..., PRE = true>.  FP32 tiles start 8 bytes
// past a 16-byte boundary (so that the middle cells of every row are
// 16-byte aligned), FP64 tiles on a 16-byte boundary.
template <typename T, int M, int PPW>
__device__ __forceinline__ void prefetch_row(const Env<T> &e, const NbMeta<T> *meta, T *tiles, int j)
{
    constexpr int PP = (M + 4) * (M + 4), NV = 16 / sizeof(T), NVM = M / NV, PIE = NVM + 2;
    constexpr int NIT = PPW * 3 * PIE;
    const int lane = threadIdx.x & 31;
    const size_t fs = (size_t)e.n * (M * M);
    const int band = j < 0 ? 0 : (j < M ? 1 : 2);                 // rows below / own / above
    const int jr = j < 0 ? j + M : (j < M ? j : j - M);           // row in the source patch
    #pragma unroll
    for (int it = 0; it < (NIT + 31) / 32; ++it) {
        const int k = lane + 32 * it;
        if (k >= NIT) break;
        const int s = k / (3 * PIE), rr = k - s * (3 * PIE), f = rr / PIE, pc = rr - f * PIE;
        int d, i;
        if (pc < NVM) { d = band == 0 ? 2 : (band == 1 ? 8 : 3); i = pc * NV; }
        else if (pc == NVM) { d = band == 0 ? 4 : (band == 1 ? 0 : 6); i = -2; }
        else { d = band == 0 ? 5 : (band == 1 ? 1 : 7); i = M; }
        const NbMeta<T> &m = meta[9 * s + d];
        if (m.kind != FC_NB_SAME || m.alpha[0] != T(1) || !m.b0) continue;
        const int si = i < 0 ? M - 2 : (i >= M ? 0 : i);
        const T *src = m.b0 + f * fs + jr * M + si;
        T *dst = tiles + s * 3 * PP + f * PP + tix<M>(i, j);
        if (pc < NVM || sizeof(T) == 8) cp_async16(dst, src);
        else cp_async8(dst, src);
    }
}

}  // namespace fc
