// fc_kernels.cu -- sm_103a kernels of the patch method.
//
// Sec. 3 of the paper (LeVeque's wave propagation on an m x m patch with two
// ghost layers; ghost values by same-level copy, fine-to-coarse averaging and
// limited conservative coarse-to-fine interpolation, time-interpolated under
// sub-cycling; regrid by interpolation / averaging) and Sec. 4 (global or
// per-level dt, fine-to-coarse correction), Sec. 5 (per-patch tagging).
//
// Work decomposition: one CTA per patch.  The CTA gathers the patch and its
// two ghost layers into shared memory straight from the neighbours'
// interiors (neighbour table lookup; same-level copy and 2x2 averages read
// neighbour interiors, which the neighbouring CTAs are reading at the same
// time, so the reread hits L2), or from the complete tile of a coarser
// neighbour.  Every edge's Riemann problem is solved once into shared memory;
// corrections, transverse parts and the update are gathered from there in
// fixed order (deterministic, no atomics except the CFL maximum).
#include <cstdio>

#include "fc_kernels.cuh"

namespace fc {

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

// per-level buffers at this launch, resolved from the device step state
struct LvBufs {
    int inew[kMaxLevels], iold[kMaxLevels];
};

template <typename T>
__device__ void resolve_levels(const Env<T> &e, LvBufs *lb)
{
    for (int l = threadIdx.x; l < kMaxLevels; l += blockDim.x) {
        int s = e.ctl->start_buf[l], k = e.kdone[l];
        lb->inew[l] = k == 0 ? s : buf_out(s, k);
        lb->iold[l] = k == 0 ? s : buf_in(s, k);
    }
}

// value of cell c of patch p, field f, at this launch's time
template <typename T>
__device__ __forceinline__ T cell_value(const Env<T> &e, const LvBufs &lb, int p, int f, int c)
{
    int l = e.f.level[p];
    size_t o = ((size_t)f * e.n + p) * (size_t)(e.m * e.m) + c;
    T a = e.alpha[l];
    T vn = qbuf(e, lb.inew[l])[o];
    if (a == T(1)) return vn;
    T vo = qbuf(e, lb.iold[l])[o];
    if (a == T(0)) return vo;
    return blend(a, vo, vn);
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

template <typename T, int M, int F>
__device__ void fill_tile(const Env<T> &e, const LvBufs &lb, int p, const int *nb, T *tile)
{
    constexpr int P = M + 4, PP = P * P;
    const int lp = e.f.level[p], xp = e.f.x[p], yp = e.f.y[p];
    const int W = (1 << lp) * M;
    const bool periodic = e.conn == FC_CONN_PERIODIC;
    for (int t = threadIdx.x; t < PP; t += blockDim.x) {
        int i = t % P - 2, j = t / P - 2;
        if (i >= 0 && i < M && j >= 0 && j < M) {
            for (int f = 0; f < F; ++f) tile[f * PP + t] = cell_value(e, lb, p, f, j * M + i);
            continue;
        }
        int ox = i < 0 ? -1 : (i >= M ? 1 : 0), oy = j < 0 ? -1 : (j >= M ? 1 : 0);
        int d = dir_of(ox, oy);
        const int *en = nb + 4 * d;
        int kind = en[0];
        if (kind == FC_NB_NONE) continue;           // wall: filled by reflection
        int gi = xp * M + i, gj = yp * M + j;
        if (periodic) { gi = (gi + W) % W; gj = (gj + W) % W; }
        if (kind == FC_NB_SAME) {
            int q = en[1];
            int ci = gi - e.f.x[q] * M, cj = gj - e.f.y[q] * M;
            if ((unsigned)q >= (unsigned)e.n || (unsigned)ci >= (unsigned)M || (unsigned)cj >= (unsigned)M) {
                e.ctl->index_error = 1;
                continue;
            }
            int c = cj * M + ci;
            for (int f = 0; f < F; ++f) tile[f * PP + t] = cell_value(e, lb, q, f, c);
        } else if (kind == FC_NB_FINER) {
            int q = d < 2 ? (j < M / 2 ? en[1] : en[2]) : (d < 4 ? (i < M / 2 ? en[1] : en[2]) : en[1]);
            int fi = (unsigned)q < (unsigned)e.n ? 2 * gi - e.f.x[q] * M : -1;
            int fj = (unsigned)q < (unsigned)e.n ? 2 * gj - e.f.y[q] * M : -1;
            if ((unsigned)fi >= (unsigned)(M - 1) || (unsigned)fj >= (unsigned)(M - 1)) {
                e.ctl->index_error = 1;
                continue;
            }
            int c00 = fj * M + fi;
            for (int f = 0; f < F; ++f) {
                T a00 = cell_value(e, lb, q, f, c00), a10 = cell_value(e, lb, q, f, c00 + 1);
                T a01 = cell_value(e, lb, q, f, c00 + M), a11 = cell_value(e, lb, q, f, c00 + M + 1);
                tile[f * PP + t] = T(0.25) * ((a00 + a10) + (a01 + a11));
            }
        } else {                                    // coarser: limited linear interpolation
            int q = en[1];
            int slot = (unsigned)q < (unsigned)e.n ? (e.grslot ? e.grslot[q] : q) : -1;
            int ci = slot >= 0 ? (gi >> 1) - e.f.x[q] * M : -1, cj = slot >= 0 ? (gj >> 1) - e.f.y[q] * M : -1;
            if ((unsigned)ci >= (unsigned)M || (unsigned)cj >= (unsigned)M) {
                e.ctl->index_error = 1;
                continue;
            }
            T sgx = (gi & 1) ? T(0.25) : T(-0.25), sgy = (gj & 1) ? T(0.25) : T(-0.25);
            const T *ct = e.gr + (size_t)slot * F * PP;
            for (int f = 0; f < F; ++f) {
                const T *A = ct + f * PP;
                T qc = A[tix<M>(ci, cj)];
                T sx = minmod(A[tix<M>(ci + 1, cj)] - qc, qc - A[tix<M>(ci - 1, cj)]);
                T sy = minmod(A[tix<M>(ci, cj + 1)] - qc, qc - A[tix<M>(ci, cj - 1)]);
                tile[f * PP + t] = radd(radd(qc, rmul(sgx, sx)), rmul(sgy, sy));
            }
        }
    }
    __syncthreads();
    if (e.conn != FC_CONN_SQUARE) return;
    const int last = (1 << lp) - 1;
    const bool wx = xp == 0 || xp == last, wy = yp == 0 || yp == last;
    if (wx) {   // x walls over the full padded height, normal momentum negated
        for (int t = threadIdx.x; t < P * 2 * F; t += blockDim.x) {
            int j = t % P - 2, k = (t / P) % 2, f = t / (2 * P);
            T sg = (F == 3 && f == 1) ? T(-1) : T(1);
            T *A = tile + f * PP;
            if (xp == 0) A[tix<M>(-1 - k, j)] = sg * A[tix<M>(k, j)];
            if (xp == last) A[tix<M>(M + k, j)] = sg * A[tix<M>(M - 1 - k, j)];
        }
        __syncthreads();
    }
    if (wy) {
        for (int t = threadIdx.x; t < P * 2 * F; t += blockDim.x) {
            int i = t % P - 2, k = (t / P) % 2, f = t / (2 * P);
            T sg = (F == 3 && f == 2) ? T(-1) : T(1);
            T *A = tile + f * PP;
            if (yp == 0) A[tix<M>(i, -1 - k)] = sg * A[tix<M>(i, k)];
            if (yp == last) A[tix<M>(i, M + k)] = sg * A[tix<M>(i, M - 1 - k)];
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void load_nbr(const Env<T> &e, int p, int *nb)
{
    if (threadIdx.x < 32) nb[threadIdx.x] = e.f.nbr[(size_t)p * 32 + threadIdx.x];
}

// ---------------------------------------------------------------------------
// edge solvers in the edge frame (h, normal momentum, transverse momentum)
//
// shallow water, Roe linearisation: u_hat, v_hat sqrt(h)-weighted averages,
// c_hat = sqrt(g (hL + hR)/2); waves a_p r_p with r1 = (1, u - c, v),
// r2 = (0, 0, 1), r3 = (1, u + c, v) and speeds u - c, u, u + c.
// Record layout: {a1, a2, a3, u_hat, v_hat, c_hat}.
template <typename T>
__device__ __forceinline__ void swe_wave(const T *rec, int p, T *w, T *s)
{
    T u = rec[3], v = rec[4], c = rec[5];
    if (p == 0) { w[0] = rec[0]; w[1] = rec[0] * (u - c); w[2] = rec[0] * v; *s = u - c; }
    else if (p == 1) { w[0] = T(0); w[1] = T(0); w[2] = rec[1]; *s = u; }
    else { w[0] = rec[2]; w[1] = rec[2] * (u + c); w[2] = rec[2] * v; *s = u + c; }
}

// fluctuations amdq, apdq of an edge record (edge frame)
template <typename T>
__device__ __forceinline__ void swe_fluct(const T *rec, T *am, T *ap)
{
    for (int k = 0; k < 3; ++k) { am[k] = T(0); ap[k] = T(0); }
    for (int p = 0; p < 3; ++p) {
        T w[3], s;
        swe_wave(rec, p, w, &s);
        T sm = tmin(s, T(0)), sp = tmax(s, T(0));
        for (int k = 0; k < 3; ++k) { am[k] += sm * w[k]; ap[k] += sp * w[k]; }
    }
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

// MC-limited own correction of an edge (edge frame), times 0.5
template <typename T, int EQ>
__device__ __forceinline__ void own_correction(const T *rec, const T *recL, const T *recR, T dtdx, T *out)
{
    if constexpr (EQ == FC_EQ_SWE) {
        T acc[3] = {T(0), T(0), T(0)};
        for (int p = 0; p < 3; ++p) {
            T w[3], s, wu[3], su;
            swe_wave(rec, p, w, &s);
            swe_wave(s >= T(0) ? recL : recR, p, wu, &su);
            T ww = (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2];
            T wup = (wu[0] * w[0] + wu[1] * w[1]) + wu[2] * w[2];
            T phi = T(0);
            if (ww != T(0)) {
                T th = fdiv(wup, ww);
                phi = tmax(T(0), tmin(tmin(T(0.5) * (T(1) + th), T(2)), T(2) * th));
            }
            T as = fabs(s);
            T cc = as * (T(1) - dtdx * as);
            for (int k = 0; k < 3; ++k) acc[k] += cc * (phi * w[k]);
        }
        for (int k = 0; k < 3; ++k) out[k] = T(0.5) * acc[k];
    } else {
        T w = rec[0], s = rec[1];
        T wu = (s >= T(0) ? recL : recR)[0];
        T phi = T(0);
        if (w * w != T(0)) {
            T th = fdiv(wu * w, w * w);
            phi = tmax(T(0), tmin(tmin(T(0.5) * (T(1) + th), T(2)), T(2) * th));
        }
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

template <typename T>
__device__ __forceinline__ T level_dt(const Env<T> &e, int level)
{
    double dt = e.ctl->dt;
    if (e.subcycle) dt = dt / (double)(1 << (level - e.lmin));
    return (T)dt;
}

// ---------------------------------------------------------------------------
// fused update: ghost fill + Riemann solves + limited corrections + transverse
// propagation + conservative update + CFL maximum + coarse-fine registers
template <int M> struct UpdCfg {
    static constexpr int NT = M == 8 ? 128 : (M == 16 ? 256 : 512);
};

template <typename T, int M, int EQ>
struct UpdLayout {
    static constexpr int F = EQ == FC_EQ_SWE ? 3 : 1;
    static constexpr int P = M + 4, PP = P * P;
    static constexpr int ER = EQ == FC_EQ_SWE ? 6 : 2;     // edge record length
    static constexpr int NXE = (M + 2) * (M + 3);           // x-edges rows -1..M, i -1..M+1
    static constexpr int NYE = (M + 3) * (M + 2);           // y-edges rows -1..M+1, i -1..M
    static constexpr int NF = (M + 1) * M;                  // corrected edges per direction
    static constexpr int DER = EQ == FC_EQ_SWE ? 3 * PP : 0;
    static constexpr int SLOTS = 2 * 4 * F * NF;
    static constexpr int ALIAS = SLOTS > DER ? SLOTS : DER;
    static constexpr size_t elems = (size_t)F * PP + ER * (NXE + NYE) + ALIAS + 2 * F * NF;
    static constexpr size_t bytes = elems * sizeof(T) + 32 * sizeof(int) + sizeof(LvBufs) + 64 * sizeof(double);
};

template <typename T, int M, int EQ>
__global__ void __launch_bounds__(UpdCfg<M>::NT)
k_update(Env<T> e, const int *list, int count, int ksub, int fine_acc)
{
    using L = UpdLayout<T, M, EQ>;
    constexpr int NT = UpdCfg<M>::NT, F = L::F, P = L::P, PP = L::PP, ER = L::ER;
    constexpr int NXE = L::NXE, NYE = L::NYE, NF = L::NF;
    extern __shared__ __align__(16) unsigned char smem[];
    double *red = (double *)smem;                   // 64 doubles
    LvBufs *lb = (LvBufs *)(red + 64);
    int *nb = (int *)(lb + 1);                      // 32 ints
    T *tile = (T *)(nb + 32);
    T *ex = tile + F * PP;
    T *ey = ex + ER * NXE;
    T *alias = ey + ER * NYE;
    T *der = alias;                     // u, v, sqrt(h) per padded cell (P1-P2)
    T *s2x = alias;                     // transverse parts into x-edges (P3-P4)
    T *s2y = alias + 4 * F * NF;        // transverse parts into y-edges (P3-P4)
    T *Ft = alias + L::ALIAS;
    T *Gt = Ft + F * NF;

    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    const int b = blockIdx.x;
    if (b >= count) return;
    const int p = list ? list[b] : b;
    const int lev = e.f.level[p];
    // level step and mesh ratio, computed once per CTA in FP64
    __shared__ T s_dt[2];
    if (threadIdx.x == 0) {
        double dtd = e.ctl->dt;
        if (e.subcycle) dtd = dtd / (double)(1 << (lev - e.lmin));
        s_dt[0] = (T)dtd;
        s_dt[1] = (T)(dtd / level_dx(lev, M));
    }
    resolve_levels(e, lb);
    load_nbr(e, p, nb);
    __syncthreads();
    const T dtl = s_dt[0];
    const T dtdx = s_dt[1];            // square cells: dt/dx = dt/dy
    // P0: patch plus two ghost layers
    fill_tile<T, M, F>(e, *lb, p, nb, tile);

    // P1: per-cell velocities and sqrt(h); dry-state check
    if constexpr (EQ == FC_EQ_SWE) {
        int dry = 0;
        for (int t = threadIdx.x; t < PP; t += NT) {
            T h = tile[t];
            if (!(h > T(0))) dry = 1;
            T ih = fdiv(T(1), h);
            der[t] = tile[PP + t] * ih;
            der[PP + t] = tile[2 * PP + t] * ih;
            der[2 * PP + t] = fsqrt(h);
        }
        if (__syncthreads_or(dry)) {
            if (threadIdx.x == 0) e.ctl->dry_error = 1;
            return;
        }
    }

    // P2: Riemann problem at every x- and y-edge of the staged tile
    T smax = T(0);
    for (int w = threadIdx.x; w < NXE + NYE; w += NT) {
        bool isx = w < NXE;
        int q = isx ? w : w - NXE;
        int cols = isx ? M + 3 : M + 2;
        int jr = q / cols, ic = q % cols;
        int iL, iR;
        bool inner;
        if (isx) { iL = (jr + 1) * P + ic; iR = iL + 1; inner = ic >= 1 && ic <= M + 1 && jr >= 1 && jr <= M; }
        else { iL = jr * P + ic + 1; iR = iL + P; inner = ic >= 1 && ic <= M && jr >= 1 && jr <= M + 1; }
        T *rec = (isx ? ex : ey) + q;    // record component k at rec[k * count]
        if constexpr (EQ == FC_EQ_SWE) {
            const int nf = isx ? 1 : 2, tf = isx ? 2 : 1;
            const T *un = der + (isx ? 0 : PP), *ut = der + (isx ? PP : 0);
            T r[6];
            swe_roe(tile[iL], tile[nf * PP + iL], tile[tf * PP + iL], un[iL], ut[iL], der[2 * PP + iL],
                    tile[iR], tile[nf * PP + iR], tile[tf * PP + iR], un[iR], ut[iR], der[2 * PP + iR], e.g, r);
            int stride = isx ? NXE : NYE;
            for (int k = 0; k < 6; ++k) rec[k * stride] = r[k];
            if (inner) smax = tmax(smax, fabs(r[3]) + r[5]);
        } else {
            int stride = isx ? NXE : NYE;
            T s = isx ? e.adv_u : e.adv_v;
            rec[0] = tile[iR] - tile[iL];
            rec[stride] = s;
            if (inner) smax = tmax(smax, (T)fabs(s));
        }
    }
    __syncthreads();

    // P3: transverse parts.  y-edge (i, j) [i -1..M, j 0..M] feeds the x-edges
    // around cells (i, j) (its up-going part) and (i, j-1) (down-going part);
    // x-edge (i, j) [i 0..M, j -1..M] feeds the y-edges around cells (i, j)
    // (right-going part) and (i-1, j) (left-going part).  Slot order:
    // 0 below-left, 1 below-right, 2 above-left, 3 above-right.
    {
        constexpr int NY2X = (M + 2) * (M + 1), NX2Y = (M + 1) * (M + 2);
        for (int w = threadIdx.x; w < NY2X + NX2Y; w += NT) {
            bool fromy = w < NY2X;
            int q = fromy ? w : w - NY2X;
            T am[3], ap[3], am_m[3], am_p[3], ap_m[3], ap_p[3];   // edge frame
            int i, j;
            if (fromy) { i = q % (M + 2) - 1; j = q / (M + 2); }
            else { i = q % (M + 1); j = q / (M + 1) - 1; }
            if constexpr (EQ == FC_EQ_SWE) {
                T r[6];
                const T *src = fromy ? ey + (j + 1) * (M + 2) + (i + 1) : ex + (j + 1) * (M + 3) + (i + 1);
                int stride = fromy ? NYE : NXE;
                for (int k = 0; k < 6; ++k) r[k] = src[k * stride];
                swe_fluct(r, am, ap);
                swe_trans(r, am, am_m, am_p);
                swe_trans(r, ap, ap_m, ap_p);
            } else {
                const T *src = fromy ? ey + (j + 1) * (M + 2) + (i + 1) : ex + (j + 1) * (M + 3) + (i + 1);
                int stride = fromy ? NYE : NXE;
                T wv = src[0], s = src[stride];
                am[0] = tmin(s, T(0)) * wv; ap[0] = tmax(s, T(0)) * wv;
                T vt = fromy ? e.adv_u : e.adv_v;     // constant transverse speed
                am_m[0] = tmin(vt, T(0)) * am[0]; am_p[0] = tmax(vt, T(0)) * am[0];
                ap_m[0] = tmin(vt, T(0)) * ap[0]; ap_p[0] = tmax(vt, T(0)) * ap[0];
            }
            // to global components (h, hu, hv)
            auto put = [&](T *slot, int sidx, const T *v) {
                if constexpr (F == 3) {
                    slot[(sidx * 3 + 0) * NF] = v[0];
                    slot[(sidx * 3 + 1) * NF] = fromy ? v[2] : v[1];
                    slot[(sidx * 3 + 2) * NF] = fromy ? v[1] : v[2];
                } else slot[sidx * NF] = v[0];
            };
            if (fromy) {
                // up-going ap enters cell (i, j): -x part -> x-edge (i, j) slot BR,
                // +x part -> x-edge (i+1, j) slot BL; down-going am enters (i, j-1):
                // -x part -> x-edge (i, j-1) slot AR, +x part -> (i+1, j-1) slot AL
                if (j < M) {
                    if (i >= 0) put(s2x + j * (M + 1) + i, 1, ap_m);
                    if (i + 1 <= M) put(s2x + j * (M + 1) + i + 1, 0, ap_p);
                }
                if (j >= 1) {
                    if (i >= 0) put(s2x + (j - 1) * (M + 1) + i, 3, am_m);
                    if (i + 1 <= M) put(s2x + (j - 1) * (M + 1) + i + 1, 2, am_p);
                }
            } else {
                // right-going ap enters cell (i, j): +y part -> y-edge (i, j+1) slot BL,
                // -y part -> y-edge (i, j) slot AL; left-going am enters (i-1, j):
                // +y part -> y-edge (i-1, j+1) slot BR, -y part -> (i-1, j) slot AR
                if (i < M) {
                    if (j + 1 <= M) put(s2y + (j + 1) * M + i, 0, ap_p);
                    if (j >= 0) put(s2y + j * M + i, 2, ap_m);
                }
                if (i >= 1) {
                    if (j + 1 <= M) put(s2y + (j + 1) * M + i - 1, 1, am_p);
                    if (j >= 0) put(s2y + j * M + i - 1, 3, am_m);
                }
            }
        }
    }
    __syncthreads();

    // P4: correction fluxes F~ (x-edges i 0..M, j 0..M-1) and G~ (y-edges
    // i 0..M-1, j 0..M): own limited correction, then the four transverse
    // parts in the order below-left, below-right, above-left, above-right
    {
        const T kk = T(0.5) * dtdx;
        for (int w = threadIdx.x; w < 2 * NF; w += NT) {
            bool isx = w < NF;
            int q = isx ? w : w - NF;
            T r[ER], rl[ER], rr[ER], own[3];
            if (isx) {
                int i = q % (M + 1), j = q / (M + 1);
                int base = (j + 1) * (M + 3) + (i + 1);
                for (int k = 0; k < ER; ++k) {
                    r[k] = ex[k * NXE + base]; rl[k] = ex[k * NXE + base - 1]; rr[k] = ex[k * NXE + base + 1];
                }
            } else {
                int i = q % M, j = q / M;
                int base = (j + 1) * (M + 2) + (i + 1);
                for (int k = 0; k < ER; ++k) {
                    r[k] = ey[k * NYE + base]; rl[k] = ey[k * NYE + base - (M + 2)]; rr[k] = ey[k * NYE + base + (M + 2)];
                }
            }
            own_correction<T, EQ>(r, rl, rr, dtdx, own);
            const T *sl = isx ? s2x : s2y;
            T *out = isx ? Ft : Gt;
            for (int f = 0; f < F; ++f) {
                int fe = F == 3 ? (isx ? f : (f == 0 ? 0 : 3 - f)) : 0;   // edge-frame index of global f
                T v = own[fe];
                for (int s = 0; s < 4; ++s) v -= kk * sl[(s * F + f) * NF + q];
                out[f * NF + q] = v;
            }
        }
    }
    __syncthreads();

    // P5: conservative update of the interior, CFL maximum, registers
    {
        const int ks = (e.kdone[lev] + 1);
        T *qout = qbuf(e, buf_out(e.ctl->start_buf[lev], ks));
        (void)ksub;
        int bad = 0;
        for (int c = threadIdx.x; c < M * M; c += NT) {
            int i = c % M, j = c / M;
            T X[3], Y[3];
            T amx[3], apx[3], amx2[3], apx2[3], amy[3], apy[3], amy2[3], apy2[3];
            int xl = (j + 1) * (M + 3) + (i + 1), yb = (j + 1) * (M + 2) + (i + 1);
            if constexpr (EQ == FC_EQ_SWE) {
                T r[6];
                for (int k = 0; k < 6; ++k) r[k] = ex[k * NXE + xl];
                swe_fluct(r, amx, apx);
                for (int k = 0; k < 6; ++k) r[k] = ex[k * NXE + xl + 1];
                swe_fluct(r, amx2, apx2);
                for (int k = 0; k < 6; ++k) r[k] = ey[k * NYE + yb];
                swe_fluct(r, amy, apy);
                for (int k = 0; k < 6; ++k) r[k] = ey[k * NYE + yb + (M + 2)];
                swe_fluct(r, amy2, apy2);
            } else {
                T w0 = ex[xl], s0 = ex[NXE + xl], w1 = ex[xl + 1], s1 = ex[NXE + xl + 1];
                amx[0] = tmin(s0, T(0)) * w0; apx[0] = tmax(s0, T(0)) * w0;
                amx2[0] = tmin(s1, T(0)) * w1; apx2[0] = tmax(s1, T(0)) * w1;
                T v0 = ey[yb], t0 = ey[NYE + yb], v1 = ey[yb + M + 2], t1 = ey[NYE + yb + M + 2];
                amy[0] = tmin(t0, T(0)) * v0; apy[0] = tmax(t0, T(0)) * v0;
                amy2[0] = tmin(t1, T(0)) * v1; apy2[0] = tmax(t1, T(0)) * v1;
            }
            int fx = j * (M + 1) + i, gy = j * M + i;
            for (int f = 0; f < F; ++f) {
                // edge-frame component of global field f for x- and y-edges
                int fxe = f, fye = F == 3 ? (f == 0 ? 0 : 3 - f) : 0;
                X[f] = (apx[fxe] + amx2[fxe]) + (Ft[f * NF + fx + 1] - Ft[f * NF + fx]);
                Y[f] = (apy[fye] + amy2[fye]) + (Gt[f * NF + gy + M] - Gt[f * NF + gy]);
                T qn = (tile[f * PP + tix<M>(i, j)] - dtdx * X[f]) - dtdx * Y[f];
                if (!isfinite(qn)) bad = 1;
                qout[((size_t)f * e.n + p) * (M * M) + c] = qn;
            }
            // effective fluxes through coarse-fine sides, times dt (FP64)
            if (e.cfslot && (i == 0 || i == M - 1 || j == 0 || j == M - 1)) {
                for (int side = 0; side < 4; ++side) {
                    bool on = side == 0 ? i == 0 : side == 1 ? i == M - 1 : side == 2 ? j == 0 : j == M - 1;
                    if (!on) continue;
                    int slot = e.cfslot[p * 4 + side];
                    if (slot < 0) continue;
                    int kind = nb[4 * side];
                    bool acc = kind == FC_NB_COARSER && fine_acc;
                    int along = side < 2 ? j : i;
                    double *rg = e.reg + ((size_t)slot * M + along) * F;
                    T qc[3];
                    for (int f = 0; f < F; ++f) qc[f] = tile[f * PP + tix<M>(i, j)];
                    for (int f = 0; f < F; ++f) {
                        T fl;
                        int fe;
                        if (side < 2) {          // x-direction flux
                            fe = f;
                            if constexpr (EQ == FC_EQ_SWE) {
                                T u = qc[1] / qc[0], v = qc[2] / qc[0];
                                fl = f == 0 ? qc[1] : (f == 1 ? qc[1] * u + T(0.5) * e.g * qc[0] * qc[0] : qc[1] * v);
                            } else fl = e.adv_u * qc[0];
                        } else {
                            fe = F == 3 ? (f == 0 ? 0 : 3 - f) : 0;
                            if constexpr (EQ == FC_EQ_SWE) {
                                T u = qc[1] / qc[0], v = qc[2] / qc[0];
                                fl = f == 0 ? qc[2] : (f == 2 ? qc[2] * v + T(0.5) * e.g * qc[0] * qc[0] : qc[2] * u);
                            } else fl = e.adv_v * qc[0];
                        }
                        T val;
                        if (side == 0) val = (fl - apx[fe]) + Ft[f * NF + fx];
                        else if (side == 1) val = (fl + amx2[fe]) + Ft[f * NF + fx + 1];
                        else if (side == 2) val = (fl - apy[fe]) + Gt[f * NF + gy];
                        else val = (fl + amy2[fe]) + Gt[f * NF + gy + M];
                        double r = (double)dtl * (double)val;
                        rg[f] = acc ? rg[f] + r : r;
                    }
                }
            }
        }
        T bm = block_max<NT, T>(smax, (T *)red);
        if (threadIdx.x == 0) atomic_max_nonneg(&e.ctl->smax_bits[lev], (double)bm);
        if (__syncthreads_or(bad) && threadIdx.x == 0) e.ctl->nonfinite_error = 1;
    }
}

// ---------------------------------------------------------------------------
// complete tiles (interior + ghosts) of listed patches, written to e.gr
template <typename T, int M, int F>
__global__ void k_fill_tiles(Env<T> e, const int *list, int count)
{
    constexpr int P = M + 4, PP = P * P;
    extern __shared__ __align__(16) unsigned char smem[];
    T *tile = (T *)smem;
    int *nb = (int *)(tile + F * PP);
    LvBufs *lb = (LvBufs *)(nb + 32);
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    int b = blockIdx.x;
    if (b >= count) return;
    int p = list ? list[b] : b;
    resolve_levels(e, lb);
    load_nbr(e, p, nb);
    __syncthreads();
    fill_tile<T, M, F>(e, *lb, p, nb, tile);
    T *dst = e.gr + (size_t)(e.grslot ? e.grslot[p] : p) * F * PP;
    for (int t = threadIdx.x; t < F * PP; t += blockDim.x) dst[t] = tile[t];
}

// ---------------------------------------------------------------------------
// coarse-fine correction of coarse boundary cells (Sec. 4): the coarse cell
// takes the average of the two fine effective fluxes in place of its own.  One
// thread per boundary cell of a listed coarse patch applies the sides it
// touches in the order -x, +x, -y, +y, so corner cells are never written by
// two threads.
template <typename T, int M, int F>
__global__ void k_reflux(Env<T> e, const int *patches, int count)
{
    constexpr int NB = 4 * M - 4;
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count * NB) return;
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    int p = patches[g / NB], b = g % NB;
    int i, j;
    if (b < M) { i = b; j = 0; }
    else if (b < 2 * M) { i = b - M; j = M - 1; }
    else if (b < 3 * M - 2) { i = 0; j = b - 2 * M + 1; }
    else { i = M - 1; j = b - (3 * M - 2) + 1; }
    int lev = e.f.level[p];
    double dx = level_dx(lev, M);
    int s = e.ctl->start_buf[lev];
    T *q = qbuf(e, e.kdone[lev] == 0 ? s : buf_out(s, e.kdone[lev]));
    const int *nbp = e.f.nbr + (size_t)p * 32;
    for (int side = 0; side < 4; ++side) {
        bool on = side == 0 ? i == 0 : side == 1 ? i == M - 1 : side == 2 ? j == 0 : j == M - 1;
        if (!on || nbp[4 * side] != FC_NB_FINER) continue;
        int c = side < 2 ? j : i;
        int fine = c < M / 2 ? nbp[4 * side + 1] : nbp[4 * side + 2];
        if ((unsigned)fine >= (unsigned)e.n) { e.ctl->index_error = 1; return; }
        int sc = e.cfslot[p * 4 + side], sf = e.cfslot[fine * 4 + (side ^ 1)];
        if (sc < 0 || sf < 0) { e.ctl->index_error = 1; return; }
        int kf = 2 * (c % (M / 2));
        double sg = (side & 1) ? 1.0 : -1.0;
        for (int f = 0; f < F; ++f) {
            double rc = e.reg[((size_t)sc * M + c) * F + f];
            double r0 = e.reg[((size_t)sf * M + kf) * F + f];
            double r1 = e.reg[((size_t)sf * M + kf + 1) * F + f];
            double corr = (rc - 0.5 * (r0 + r1)) / dx;
            size_t o = ((size_t)f * e.n + p) * (M * M) + j * M + i;
            q[o] = (T)((double)q[o] + sg * corr);
        }
    }
}

// ---------------------------------------------------------------------------
// step control: Courant number, accept / retake, next dt (single thread)
struct DxTab { double dx[kMaxLevels]; int nsub[kMaxLevels]; };

__global__ void k_step_ctl(StepCtl *c, int lmin, int lmax, int subcycle, DxTab tab)
{
    if (threadIdx.x | blockIdx.x) return;
    if (c->dry_error | c->nonfinite_error | c->index_error) return;
    double rate = 0.0;
    for (int l = lmin; l <= lmax; ++l) {
        double s = __longlong_as_double((long long)c->smax_bits[l]);
        rate = fmax(rate, s / tab.dx[subcycle ? lmin : l]);
        c->smax_bits[l] = 0ULL;
    }
    double dt = c->dt, nu = dt * rate;
    bool accept = nu <= 1.0 || c->dt_fixed > 0.0 || c->attempts == 3;
    if (accept) {
        c->t += dt;
        c->last_dt = dt;
        c->last_courant = nu;
        c->accepted += 1;
        for (int l = lmin; l <= lmax; ++l)
            if (tab.nsub[l] > 0) c->start_buf[l] = buf_out(c->start_buf[l], tab.nsub[l]);
        if (nu > 1.0) c->cfl_error = 1;
        c->attempts = 0;
        // the Courant step is kept even under a fixed step, for a later switch
        c->next_dt = rate > 0.0 ? c->cfl / rate : c->next_dt;
        c->dt = c->dt_fixed > 0.0 ? c->dt_fixed : c->next_dt;
    } else {
        c->attempts += 1;
        c->retries += 1;
        c->dt = 0.9 * dt * (c->cfl / nu);
    }
}

// R10 first-step rule: largest cell characteristic speed per level
template <typename T, int F>
__global__ void k_cell_speed(Env<T> e)
{
    __shared__ double red[32];
    int p = blockIdx.x;
    if (p >= e.n) return;
    int lev = e.f.level[p];
    int s = e.ctl->start_buf[lev];
    const T *q = qbuf(e, s);
    int mm = e.m * e.m;
    double v = 0.0;
    for (int c = threadIdx.x; c < mm; c += blockDim.x) {
        if constexpr (F == 3) {
            double h = (double)q[((size_t)0 * e.n + p) * mm + c];
            double u = (double)q[((size_t)1 * e.n + p) * mm + c] / h;
            double w = (double)q[((size_t)2 * e.n + p) * mm + c] / h;
            double cc = sqrt((double)e.g * h);
            v = fmax(v, fmax(fabs(u) + cc, fabs(w) + cc));
        } else {
            v = fmax(v, fmax(fabs((double)e.adv_u), fabs((double)e.adv_v)));
        }
    }
    double bm = block_max<256, double>(v, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&e.ctl->smax_bits[lev], bm);
}

__global__ void k_dt_from_next(StepCtl *c)
{
    if (threadIdx.x | blockIdx.x) return;
    if (c->next_dt > 0.0) c->dt = c->next_dt;
}

int launch_dt_from_next(StepCtl *ctl, cudaStream_t s)
{
    k_dt_from_next<<<1, 32, 0, s>>>(ctl);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

__global__ void k_dt_from_cells(StepCtl *c, int lmin, int lmax, int subcycle, DxTab tab)
{
    if (threadIdx.x | blockIdx.x) return;
    double rate = 0.0;
    for (int l = lmin; l <= lmax; ++l) {
        double s = __longlong_as_double((long long)c->smax_bits[l]);
        rate = fmax(rate, s / tab.dx[subcycle ? lmin : l]);
        c->smax_bits[l] = 0ULL;
    }
    if (rate > 0.0) c->dt = c->cfl / rate;
    c->next_dt = c->dt;
}

// ---------------------------------------------------------------------------
// initial data: point samples at cell centres of the square
template <typename T, int F>
__global__ void k_init(Env<T> e, int kind, const double *pr, int np)
{
    int p = blockIdx.x;
    if (p >= e.n) return;
    int m = e.m, mm = m * m, lev = e.f.level[p];
    double dx = level_dx(lev, m);
    T *q = qbuf(e, e.ctl->start_buf[lev]);
    for (int c = threadIdx.x; c < mm; c += blockDim.x) {
        int i = c % m, j = c / m;
        double x = (((double)e.f.x[p] * m + i) + 0.5) * dx;
        double y = (((double)e.f.y[p] * m + j) + 0.5) * dx;
        double v0 = 0.0;
        if (kind == FC_INIT_DAMBREAK) {
            double ax = x - pr[0], ay = y - pr[1];
            v0 = __dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)) < pr[2] ? pr[3] : pr[4];
        } else if (kind == FC_INIT_HUMPS) {
            double h = pr[0];
            for (int b = 0; b < (np - 1) / 4; ++b) {
                const double *hp = pr + 1 + 4 * b;
                double ax = x - hp[2], ay = y - hp[3];
                double r2 = __dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay));
                h = __dadd_rn(h, __dmul_rn(hp[0], exp(-(r2 / __dmul_rn(hp[1], hp[1])))));
            }
            v0 = h;
        } else if (kind == FC_INIT_ADV_BOX) {
            v0 = (x >= pr[0] && x < pr[1] && y >= pr[2] && y < pr[3]) ? pr[4] : pr[5];
        } else {
            v0 = pr[0] + pr[1] * sin(2.0 * 3.14159265358979323846 * (pr[2] * x + pr[3] * y));
        }
        q[(size_t)p * mm + c] = (T)v0;
        if (F == 3) {
            q[((size_t)1 * e.n + p) * mm + c] = T(0);
            q[((size_t)2 * e.n + p) * mm + c] = T(0);
        }
    }
}

// ---------------------------------------------------------------------------
// conservation sums: per-patch partials, then one block in fixed order
template <typename T, int F>
__global__ void k_sum_patches(Env<T> e, double *part)
{
    __shared__ double red[F][32];
    int p = blockIdx.x;
    if (p >= e.n) return;
    int mm = e.m * e.m, lev = e.f.level[p];
    const T *q = qbuf(e, e.ctl->start_buf[lev]);
    double acc[F];
    for (int f = 0; f < F; ++f) acc[f] = 0.0;
    for (int c = threadIdx.x; c < mm; c += blockDim.x)
        for (int f = 0; f < F; ++f) acc[f] += (double)q[((size_t)f * e.n + p) * mm + c];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int f = 0; f < F; ++f) {
        double v = acc[f];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[f][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < F) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[threadIdx.x][k];
        double dx = level_dx(lev, e.m);
        part[(size_t)p * F + threadIdx.x] = v * (dx * dx);
    }
}

template <int F>
__global__ void k_sum_final(const double *part, int n, double *out)
{
    __shared__ double red[F][1024];
    for (int f = 0; f < F; ++f) {
        double v = 0.0;
        for (int p = threadIdx.x; p < n; p += blockDim.x) v += part[(size_t)p * F + f];
        red[f][threadIdx.x] = v;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int f = 0; f < F; ++f) red[f][threadIdx.x] += red[f][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < F) out[threadIdx.x] = red[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// tagging (Sec. 5): criterion on the ghost-filled patch, decided with
// explicitly rounded arithmetic
template <typename T>
__device__ __forceinline__ T grad_norm(T l, T r, T b, T t)
{
    T gx = rmul(rsub(r, l), T(0.5));
    T gy = rmul(rsub(t, b), T(0.5));
    return sqrt(radd(rmul(gx, gx), rmul(gy, gy)));
}

template <typename T, int M, int F>
__global__ void k_tag(Env<T> e, int crit, double thr, int8_t *flags)
{
    constexpr int P = M + 4, PP = P * P;
    extern __shared__ __align__(16) unsigned char smem[];
    T *tile = (T *)smem;
    int *nb = (int *)(tile + F * PP);
    LvBufs *lb = (LvBufs *)(nb + 32);
    __shared__ int hit;
    int p = blockIdx.x;
    if (p >= e.n) return;
    resolve_levels(e, lb);
    load_nbr(e, p, nb);
    if (threadIdx.x == 0) hit = 0;
    __syncthreads();
    fill_tile<T, M, F>(e, *lb, p, nb, tile);
    T th = (T)thr;
    int loc = 0;
    if (crit == FC_TAG_GRAD) {
        for (int c = threadIdx.x; c < M * M; c += blockDim.x) {
            int i = c % M, j = c / M;
            T g = grad_norm(tile[tix<M>(i - 1, j)], tile[tix<M>(i + 1, j)], tile[tix<M>(i, j - 1)],
                            tile[tix<M>(i, j + 1)]);
            if (g > th) loc = 1;
        }
    } else {
        __shared__ T mn[32], mx[32];
        T lo = tile[tix<M>(0, 0)], hi = lo;
        for (int c = threadIdx.x; c < M * M; c += blockDim.x) {
            T v = tile[tix<M>(c % M, c / M)];
            lo = tmin(lo, v); hi = tmax(hi, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = tmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = tmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) { mn[threadIdx.x >> 5] = lo; mx[threadIdx.x >> 5] = hi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { lo = tmin(lo, mn[k]); hi = tmax(hi, mx[k]); }
            if (rsub(tmax(hi, mx[0]), tmin(lo, mn[0])) > th) loc = 1;
        }
    }
    if (loc) atomicOr(&hit, 1);
    __syncthreads();
    if (threadIdx.x == 0) flags[p] = hit ? 1 : 0;
}

// families of four sibling leaves whose averaged parent fails the criterion
template <typename T, int M>
__global__ void k_tag_family(Env<T> e, int crit, double thr, int min_level, int8_t *flags)
{
    __shared__ T par[M * M];
    __shared__ int fam, hit;
    int k = blockIdx.x;
    if (k + 3 >= e.n) return;
    const ForestDev &f = e.f;
    if (threadIdx.x == 0) {
        int ok = f.level[k] > min_level && (f.x[k] & 1) == 0 && (f.y[k] & 1) == 0;
        for (int c = 1; c < 4 && ok; ++c)
            ok = f.tree[k + c] == f.tree[k] && f.level[k + c] == f.level[k] && f.x[k + c] == f.x[k] + (c & 1) &&
                 f.y[k + c] == f.y[k] + (c >> 1);
        fam = ok;
        hit = 0;
    }
    __syncthreads();
    if (!fam) return;
    constexpr int H = M / 2;
    int mm = M * M;
    for (int c = threadIdx.x; c < mm; c += blockDim.x) {
        int i = c % M, j = c / M;
        int ch = k + (i >= H) + 2 * (j >= H);
        const T *q = qbuf(e, e.ctl->start_buf[f.level[ch]]) + (size_t)ch * mm;
        int fi = 2 * (i % H), fj = 2 * (j % H);
        par[c] = T(0.25) * ((q[fj * M + fi] + q[fj * M + fi + 1]) + (q[(fj + 1) * M + fi] + q[(fj + 1) * M + fi + 1]));
    }
    __syncthreads();
    T th = (T)thr;
    int loc = 0;
    if (crit == FC_TAG_GRAD) {
        for (int c = threadIdx.x; c < mm; c += blockDim.x) {
            int i = c % M, j = c / M;
            if (i < 1 || i > M - 2 || j < 1 || j > M - 2) continue;
            T g = grad_norm(par[c - 1], par[c + 1], par[c - M], par[c + M]);
            if (g > th) loc = 1;
        }
    } else if (threadIdx.x == 0) {
        T lo = par[0], hi = par[0];
        for (int c = 1; c < mm; ++c) { lo = tmin(lo, par[c]); hi = tmax(hi, par[c]); }
        if (rsub(hi, lo) > th) loc = 1;
    }
    if (loc) atomicOr(&hit, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !hit)
        for (int c = 0; c < 4; ++c)
            if (flags[k + c] == 0) flags[k + c] = -1;
}

// ---------------------------------------------------------------------------
// regrid transfer: new leaf k from its origin in the old forest
template <typename T, int M, int F>
__global__ void k_transfer(Env<T> eo, Env<T> en, const int *origin, const T *tiles_old, const int *old_x,
                           const int *old_y)
{
    constexpr int P = M + 4, PP = P * P, H = M / 2, MM = M * M;
    int k = blockIdx.x;
    if (k >= en.n) return;
    int kind = origin[3 * k], o = origin[3 * k + 1], dl = origin[3 * k + 2];
    T *qn = en.q[0];
    for (int c = threadIdx.x; c < MM; c += blockDim.x) {
        int i = c % M, j = c / M;
        for (int f = 0; f < F; ++f) {
            T v;
            if (kind == 0) {
                v = qbuf(eo, eo.ctl->start_buf[eo.f.level[o]])[((size_t)f * eo.n + o) * MM + c];
            } else if (kind == 1) {
                int r = 1 << dl;
                int gi = en.f.x[k] * M + i, gj = en.f.y[k] * M + j;
                int ci = gi / r - old_x[o] * M, cj = gj / r - old_y[o] * M;
                T sgx = (T)(((double)(gi % r) + 0.5) / r - 0.5);
                T sgy = (T)(((double)(gj % r) + 0.5) / r - 0.5);
                const T *A = tiles_old + ((size_t)o * F + f) * PP;
                T qc = A[tix<M>(ci, cj)];
                T sx = minmod(A[tix<M>(ci + 1, cj)] - qc, qc - A[tix<M>(ci - 1, cj)]);
                T sy = minmod(A[tix<M>(ci, cj + 1)] - qc, qc - A[tix<M>(ci, cj - 1)]);
                v = radd(radd(qc, rmul(sgx, sx)), rmul(sgy, sy));
            } else {
                int ch = o + (i >= H) + 2 * (j >= H);
                const T *a = qbuf(eo, eo.ctl->start_buf[eo.f.level[ch]]) + ((size_t)f * eo.n + ch) * MM;
                int fi = 2 * (i % H), fj = 2 * (j % H);
                v = T(0.25) * ((a[fj * M + fi] + a[fj * M + fi + 1]) + (a[(fj + 1) * M + fi] + a[(fj + 1) * M + fi + 1]));
            }
            qn[((size_t)f * en.n + k) * MM + c] = v;
        }
    }
}

// layout conversion between [F][n][mm] (inside) and [n][F][mm] (caller)
template <typename T>
__global__ void k_read(Env<T> e, int field, T *dst)
{
    int p = blockIdx.x;
    if (p >= e.n) return;
    int mm = e.m * e.m;
    const T *q = qbuf(e, e.ctl->start_buf[e.f.level[p]]);
    int f0 = field < 0 ? 0 : field, f1 = field < 0 ? e.F : field + 1, nf = f1 - f0;
    for (int f = f0; f < f1; ++f)
        for (int c = threadIdx.x; c < mm; c += blockDim.x)
            dst[((size_t)p * nf + (f - f0)) * mm + c] = q[((size_t)f * e.n + p) * mm + c];
}

template <typename T>
__global__ void k_write(Env<T> e, const T *src)
{
    int p = blockIdx.x;
    if (p >= e.n) return;
    int mm = e.m * e.m;
    T *q = qbuf(e, e.ctl->start_buf[e.f.level[p]]);
    for (int f = 0; f < e.F; ++f)
        for (int c = threadIdx.x; c < mm; c += blockDim.x)
            q[((size_t)f * e.n + p) * mm + c] = src[((size_t)p * e.F + f) * mm + c];
}

// ---------------------------------------------------------------------------
// launchers
static inline int blocks_of(long long n, int b) { return (int)((n + b - 1) / b); }

template <typename T, int M, int EQ>
static int launch_update_t(const Env<T> &e, List l, int ksub, int fine_acc, cudaStream_t s)
{
    using Lay = UpdLayout<T, M, EQ>;
    constexpr int NT = UpdCfg<M>::NT;
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(k_update<T, M, EQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Lay::bytes);
        if (err != cudaSuccess) return cuda_status(err, "cudaFuncSetAttribute(k_update)");
        configured = true;
    }
    if (l.count <= 0) return FC_OK;
    k_update<T, M, EQ><<<l.count, NT, Lay::bytes, s>>>(e, l.idx, l.count, ksub, fine_acc);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_update(const Env<T> &e, List l, int ksub, int fine_acc, cudaStream_t s)
{
    if (e.eq == FC_EQ_SWE) {
        if (e.m == 8) return launch_update_t<T, 8, FC_EQ_SWE>(e, l, ksub, fine_acc, s);
        if (e.m == 16) return launch_update_t<T, 16, FC_EQ_SWE>(e, l, ksub, fine_acc, s);
        if (e.m == 32 && sizeof(T) == 4) return launch_update_t<T, 32, FC_EQ_SWE>(e, l, ksub, fine_acc, s);
    } else {
        if (e.m == 8) return launch_update_t<T, 8, FC_EQ_ADV>(e, l, ksub, fine_acc, s);
        if (e.m == 16) return launch_update_t<T, 16, FC_EQ_ADV>(e, l, ksub, fine_acc, s);
        if (e.m == 32) return launch_update_t<T, 32, FC_EQ_ADV>(e, l, ksub, fine_acc, s);
    }
    set_error("unsupported patch size %d for this precision / equation", e.m);
    return FC_ERR_UNIMPLEMENTED;
}

template <typename T, int M, int F>
static size_t tile_smem() { return (size_t)F * (M + 4) * (M + 4) * sizeof(T) + 32 * sizeof(int) + sizeof(LvBufs) + 16; }

#define FC_DISPATCH_MF(e, CALL)                                                           \
    do {                                                                                  \
        if ((e).F == 3) {                                                                 \
            if ((e).m == 8) { constexpr int M = 8, F = 3; CALL; }                          \
            else if ((e).m == 16) { constexpr int M = 16, F = 3; CALL; }                   \
            else if ((e).m == 32) { constexpr int M = 32, F = 3; CALL; }                   \
        } else {                                                                          \
            if ((e).m == 8) { constexpr int M = 8, F = 1; CALL; }                          \
            else if ((e).m == 16) { constexpr int M = 16, F = 1; CALL; }                   \
            else if ((e).m == 32) { constexpr int M = 32, F = 1; CALL; }                   \
        }                                                                                 \
    } while (0)

template <typename T>
int launch_fill_tiles(const Env<T> &e, List l, cudaStream_t s)
{
    if (l.count <= 0) return FC_OK;
    FC_DISPATCH_MF(e, (k_fill_tiles<T, M, F><<<l.count, 256, tile_smem<T, M, F>(), s>>>(e, l.idx, l.count)));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_reflux(const Env<T> &e, List patches, cudaStream_t s)
{
    if (patches.count <= 0) return FC_OK;
    FC_DISPATCH_MF(e, (k_reflux<T, M, F><<<blocks_of((long long)patches.count * (4 * M - 4), 128), 128, 0, s>>>(
                          e, patches.idx, patches.count)));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

int launch_step_ctl(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, const int *nsub,
                    cudaStream_t s)
{
    DxTab tab;
    for (int l = 0; l < kMaxLevels; ++l) { tab.dx[l] = dx[l]; tab.nsub[l] = nsub[l]; }
    k_step_ctl<<<1, 32, 0, s>>>(ctl, lmin, lmax, subcycle, tab);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_cell_rate(const Env<T> &e, cudaStream_t s)
{
    if (e.F == 3) k_cell_speed<T, 3><<<e.n, 256, 0, s>>>(e);
    else k_cell_speed<T, 1><<<e.n, 256, 0, s>>>(e);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

int launch_dt_from_cells(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, cudaStream_t s)
{
    DxTab tab;
    for (int l = 0; l < kMaxLevels; ++l) { tab.dx[l] = dx[l]; tab.nsub[l] = 0; }
    k_dt_from_cells<<<1, 32, 0, s>>>(ctl, lmin, lmax, subcycle, tab);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_init(const Env<T> &e, int kind, const double *d_p, int np, cudaStream_t s)
{
    if (e.F == 3) k_init<T, 3><<<e.n, 256, 0, s>>>(e, kind, d_p, np);
    else k_init<T, 1><<<e.n, 256, 0, s>>>(e, kind, d_p, np);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_sums(const Env<T> &e, double *d_part, double *d_out, cudaStream_t s)
{
    if (e.F == 3) {
        k_sum_patches<T, 3><<<e.n, 256, 0, s>>>(e, d_part);
        k_sum_final<3><<<1, 1024, 0, s>>>(d_part, e.n, d_out);
    } else {
        k_sum_patches<T, 1><<<e.n, 256, 0, s>>>(e, d_part);
        k_sum_final<1><<<1, 1024, 0, s>>>(d_part, e.n, d_out);
    }
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_tag(const Env<T> &e, int crit, double thr, int min_level, int8_t *d_flags, cudaStream_t s)
{
    FC_DISPATCH_MF(e, (k_tag<T, M, F><<<e.n, 256, tile_smem<T, M, F>(), s>>>(e, crit, thr, d_flags)));
    FC_CUDA(cudaGetLastError());
    if (e.m == 8) k_tag_family<T, 8><<<e.n, 256, 0, s>>>(e, crit, thr, min_level, d_flags);
    else if (e.m == 16) k_tag_family<T, 16><<<e.n, 256, 0, s>>>(e, crit, thr, min_level, d_flags);
    else k_tag_family<T, 32><<<e.n, 256, 0, s>>>(e, crit, thr, min_level, d_flags);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_transfer(const Env<T> &eold, const Env<T> &enew, const int *origin, const T *tiles_old,
                    const int *old_x, const int *old_y, cudaStream_t s)
{
    FC_DISPATCH_MF(enew, (k_transfer<T, M, F><<<enew.n, 256, 0, s>>>(eold, enew, origin, tiles_old, old_x, old_y)));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_read(const Env<T> &e, int field, T *dst, cudaStream_t s)
{
    k_read<T><<<e.n, 256, 0, s>>>(e, field, dst);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_write(const Env<T> &e, const T *src, cudaStream_t s)
{
    k_write<T><<<e.n, 256, 0, s>>>(e, src);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

#define FC_INSTANTIATE(T)                                                                                     \
    template int launch_update<T>(const Env<T> &, List, int, int, cudaStream_t);                              \
    template int launch_fill_tiles<T>(const Env<T> &, List, cudaStream_t);                                    \
    template int launch_reflux<T>(const Env<T> &, List, cudaStream_t);                                        \
    template int launch_cell_rate<T>(const Env<T> &, cudaStream_t);                                           \
    template int launch_init<T>(const Env<T> &, int, const double *, int, cudaStream_t);                      \
    template int launch_sums<T>(const Env<T> &, double *, double *, cudaStream_t);                            \
    template int launch_tag<T>(const Env<T> &, int, double, int, int8_t *, cudaStream_t);                     \
    template int launch_transfer<T>(const Env<T> &, const Env<T> &, const int *, const T *, const int *,      \
                                    const int *, cudaStream_t);                                               \
    template int launch_read<T>(const Env<T> &, int, T *, cudaStream_t);                                      \
    template int launch_write<T>(const Env<T> &, const T *, cudaStream_t);

FC_INSTANTIATE(float)
FC_INSTANTIATE(double)

}  // namespace fc
