// fc3_kernels.cuh -- sm_103a kernels of the three-dimensional patch solver
// (octree of M^3 patches, periodic unit cube, scalar advection with a
// constant velocity; arXiv:1308.1472 Sec. 2-4 for d = 3, Eq. (1) of Sec. 5).
//
// Layout in HBM (one context):
//   leaves   int32 level[n], x[n], y[n], z[n]            (Morton order)
//   nb       int32 [n][26][5] {kind, id0..id3} per direction (dx,dy,dz) in
//            x-fastest order with (0,0,0) left out; kind 1 same level, 2
//            coarser, 3 finer (ids of the finer leaves next to the patch,
//            indexed by their position bits along the axes where the
//            direction is 0, in axis order)
//   q        T [n][M^3] ([k][j][i]), two buffers (state, next state)
//   gr       T [ntile][(M+4)^3] complete tiles of the patches next to a
//            finer patch (sources of coarse-to-fine interpolation)
//   flux     T [nrec][6][M^2] face fluxes through the boundary cells of
//            patches next to a patch of another level (coarse-fine
//            correction), side 2d + (upper), cells [b][a] over the two
//            other axes in increasing order
//
// Work decomposition: one CTA per patch.  The CTA gathers the patch and
// two ghost layers into shared memory (same-level copy, 2x2x2 mean of finer
// cells, limited linear interpolation from a coarser neighbour's complete
// tile), then in three barrier-separated phases computes (1) the
// fluctuation entering every cell of a one-cell band, (2) the correction
// flux of every face of the patch's cells: its own MC-limited term, then the
// transverse and corner parts gathered from the band in a fixed order, and
// (3) the update of each cell and the flux through its boundary faces.  With
// a constant velocity each cell receives exactly one fluctuation per
// direction, A_d = u_d (Q_c - Q_{c-1}) for u_d >= 0, u_d (Q_{c+1} - Q_c)
// otherwise, and a face of direction t whose upwind cell (along t) is b
// takes
//   F_t = own_t - dt/(2dx) u_t sum_{d != t} A_d(b)
//              + dt^2/(6dx^2) u_t sum_{d != t} |u_e| (A_d(b) - A_d(b - sgn(u_e) e)),
// e the third direction: the transverse parts of the fluctuations entering
// b and the corner parts of those entering b and its upwind neighbour along
// e (the gathered form of splitting each fluctuation in the two
// perpendicular directions and each transverse part again in the third).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fc_internal.cuh"

namespace fc3 {

constexpr int kMaxLevel = 10;

template <typename T>
struct Env3 {
    int n;
    const int *level, *x, *y, *z;
    const int *nb;         // [n][26][5]
    const int *tslot;      // [n] complete-tile slot or -1
    const int *fslot;      // [n] flux-record slot or -1
    const T *q;            // state (the newer state of each level)
    const T *qold;         // older state of each level (sub-cycling), or q
    T *qo;                 // where the update writes
    T *gr;                 // complete tiles
    T *flux;               // coarse-fine records: dt * face flux
    T vel[3];
    T k[kMaxLevel + 1];    // dt_l / dx_l per level
    T dtl[kMaxLevel + 1];  // step of each level
    T idx[kMaxLevel + 1];  // 1 / dx_l
    T alpha[kMaxLevel + 1];// weight of the newer state per level at this launch's time
    const int *list;       // patches updated by this launch (null: all)
    int count;
    int ksub;              // 0: records of sides facing a coarser leaf are set, else added
    int limiter, transverse;
    int *err;              // set to 1 when a table entry points nowhere (nothing read then)
};

// value c of leaf r at the launch's time: its level's older and newer states
// blended with that level's weight a (1: newer, 0: older)
template <typename T, int M>
__device__ __forceinline__ T lval(const Env3<T> &e, T a, int r, int c)
{
    const size_t o = (size_t)r * (M * M * M) + c;
    if (a == T(1)) return e.q[o];
    if (a == T(0)) return e.qold[o];
    return (T(1) - a) * e.qold[o] + a * e.q[o];
}

template <int M> __host__ __device__ constexpr int P3() { return (M + 4) * (M + 4) * (M + 4); }
template <int M> __device__ __forceinline__ int tix3(int i, int j, int k)
{
    return (i + 2) + (M + 4) * ((j + 2) + (M + 4) * (k + 2));
}

template <typename T> __device__ __forceinline__ T mm3(T a, T b)
{
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

template <int M> struct Log2M;
template <> struct Log2M<4> { static constexpr int v = 2; };
template <> struct Log2M<8> { static constexpr int v = 3; };

// complete tile of patch p into shared memory (all threads of the CTA; the
// CTA's 26 x 5 neighbour entries are staged in nbs): the interior, then the
// 26 ghost regions (2 or M cells along each axis), one warp per region
template <typename T, int M>
__device__ void gather3(const Env3<T> &e, int p, T *tile, int *nbs)
{
    constexpr int P = M + 4, MM = M * M * M, LM = Log2M<M>::v;
    const int l = e.level[p];
    const int N = M << l;
    const int org[3] = {e.x[p] * M, e.y[p] * M, e.z[p] * M};
    for (int t = threadIdx.x; t < 26 * 5; t += blockDim.x) nbs[t] = e.nb[(size_t)p * 26 * 5 + t];
    const T a_same = e.alpha[l], a_fine = e.alpha[l < kMaxLevel ? l + 1 : l];
    // the interior: every load of the thread issued before its first store
    // (the sources are generic pointers, a store in between would order them)
    constexpr int NI = 2;                       // MM / blockDim (256 threads, m = 8; m = 4 needs 1)
    T iv[NI];
    #pragma unroll
    for (int it = 0; it < NI; ++it) {
        const int c = threadIdx.x + it * blockDim.x;
        if (c < MM) iv[it] = lval<T, M>(e, a_same, p, c);
    }
    #pragma unroll
    for (int it = 0; it < NI; ++it) {
        const int c = threadIdx.x + it * blockDim.x;
        if (c < MM) {
            const int i = c & (M - 1), j = (c >> LM) & (M - 1), k = c >> (2 * LM);
            tile[(i + 2) + P * ((j + 2) + P * (k + 2))] = iv[it];
        }
    }
    for (int c = threadIdx.x + NI * blockDim.x; c < MM; c += blockDim.x) {
        const int i = c & (M - 1), j = (c >> LM) & (M - 1), k = c >> (2 * LM);
        tile[(i + 2) + P * ((j + 2) + P * (k + 2))] = lval<T, M>(e, a_same, p, c);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < 26; r += nw) {
        const int d26 = r < 13 ? r : r + 1;
        const int dir[3] = {d26 % 3 - 1, (d26 / 3) % 3 - 1, d26 / 9 - 1};
        const int lg[3] = {dir[0] ? 1 : LM, dir[1] ? 1 : LM, dir[2] ? 1 : LM};
        const int cnt = 1 << (lg[0] + lg[1] + lg[2]);
        const int *en = nbs + r * 5;
        const int kind = en[0];
        if (kind == 1 && en[1] >= 0 && cnt <= 128) {
            // same level (the common case): a lane's (up to 4) loads first, then its stores
            T sv[4];
            int st_[4];
            #pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int c = lane + 32 * it;
                st_[it] = -1;
                if (c < cnt) {
                    const int a[3] = {c & ((1 << lg[0]) - 1), (c >> lg[0]) & ((1 << lg[1]) - 1), c >> (lg[0] + lg[1])};
                    int li[3];
                    #pragma unroll
                    for (int q = 0; q < 3; ++q) li[q] = dir[q] < 0 ? a[q] - 2 : (dir[q] > 0 ? M + a[q] : a[q]);
                    sv[it] = lval<T, M>(e, a_same, en[1], (li[0] & (M - 1)) + M * ((li[1] & (M - 1)) + M * (li[2] & (M - 1))));
                    st_[it] = (li[0] + 2) + P * ((li[1] + 2) + P * (li[2] + 2));
                }
            }
            #pragma unroll
            for (int it = 0; it < 4; ++it)
                if (st_[it] >= 0) tile[st_[it]] = sv[it];
            continue;
        }
        for (int c = lane; c < cnt; c += 32) {
            const int a[3] = {c & ((1 << lg[0]) - 1), (c >> lg[0]) & ((1 << lg[1]) - 1), c >> (lg[0] + lg[1])};
            int li[3];
            #pragma unroll
            for (int q = 0; q < 3; ++q) li[q] = dir[q] < 0 ? a[q] - 2 : (dir[q] > 0 ? M + a[q] : a[q]);
            T v = T(0);
            if (kind == 1 && en[1] >= 0) {
                v = lval<T, M>(e, a_same, en[1], (li[0] & (M - 1)) + M * ((li[1] & (M - 1)) + M * (li[2] & (M - 1))));
            } else {
                int g[3];
                #pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int w = org[q] + li[q];
                    g[q] = w < 0 ? w + N : (w >= N ? w - N : w);
                }
                if (kind == 2) {
                    const int ts = en[1] >= 0 ? e.tslot[en[1]] : -1;
                    if (ts < 0) { *e.err = 1; }
                    else {
                        const T *A = e.gr + (size_t)ts * P3<M>();
                        const int ci = (g[0] >> 1) & (M - 1), cj = (g[1] >> 1) & (M - 1), ck = (g[2] >> 1) & (M - 1);
                        const T qc = A[tix3<M>(ci, cj, ck)];
                        const T sx = mm3(A[tix3<M>(ci + 1, cj, ck)] - qc, qc - A[tix3<M>(ci - 1, cj, ck)]);
                        const T sy = mm3(A[tix3<M>(ci, cj + 1, ck)] - qc, qc - A[tix3<M>(ci, cj - 1, ck)]);
                        const T sz = mm3(A[tix3<M>(ci, cj, ck + 1)] - qc, qc - A[tix3<M>(ci, cj, ck - 1)]);
                        const T ox = (g[0] & 1) ? T(0.25) : T(-0.25), oy = (g[1] & 1) ? T(0.25) : T(-0.25),
                                oz = (g[2] & 1) ? T(0.25) : T(-0.25);
                        v = ((qc + ox * sx) + oy * sy) + oz * sz;
                    }
                } else {
                    int sub = 0, nbits = 0;
                    #pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (dir[q] == 0) { sub |= (((2 * g[q]) >> LM) & 1) << nbits; ++nbits; }
                    const int fr = kind == 3 ? en[1 + sub] : -1;
                    if (fr < 0) { *e.err = 1; }
                    else {
                        const int fi = (2 * g[0]) & (M - 1), fj = (2 * g[1]) & (M - 1), fk = (2 * g[2]) & (M - 1);
                        auto at = [&](int x, int y, int z) { return lval<T, M>(e, a_fine, fr, (fi + x) + M * ((fj + y) + M * (fk + z))); };
                        const T s0 = at(0, 0, 0) + at(1, 0, 0), s1 = at(0, 1, 0) + at(1, 1, 0);
                        const T s2 = at(0, 0, 1) + at(1, 0, 1), s3 = at(0, 1, 1) + at(1, 1, 1);
                        v = T(0.125) * ((s0 + s1) + (s2 + s3));
                    }
                }
            }
            tile[(li[0] + 2) + P * ((li[1] + 2) + P * (li[2] + 2))] = v;
        }
    }
}

// complete tiles of the listed patches (one level per launch, coarsest first)
template <typename T, int M>
__global__ void k3_fill_tiles(Env3<T> e, const int *list, int count)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int nbs[26 * 5];
    T *tile = reinterpret_cast<T *>(smem);
    if (blockIdx.x >= count) return;
    const int p = list[blockIdx.x];
    gather3<T, M>(e, p, tile, nbs);
    __syncthreads();
    T *dst = e.gr + (size_t)e.tslot[p] * P3<M>();
    for (int c = threadIdx.x; c < P3<M>(); c += blockDim.x) dst[c] = tile[c];
}

// older state of the listed patches := their newer state
template <typename T, int M>
__global__ void k3_copy_old(Env3<T> e, const int *list, int count)
{
    constexpr int MM = M * M * M;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)count * MM) return;
    const size_t o = (size_t)list[g / MM] * MM + (size_t)(g % MM);
    const_cast<T *>(e.qold)[o] = e.q[o];
}

template <typename T, int M>
struct Upd3Layout {
    static constexpr int P = M + 4, B = M + 2, NF = (M + 1) * M * M;
    static constexpr size_t tile = 0;
    static constexpr size_t A = tile + (size_t)P * P * P * sizeof(T);
    static constexpr size_t F = A + (size_t)3 * B * B * B * sizeof(T);
    static constexpr size_t bytes = F + (size_t)3 * NF * sizeof(T);
};

// MC limiter
template <typename T> __device__ __forceinline__ T mc3(T th)
{
    T a = (T(1) + th) / T(2), r = a < T(2) ? a : T(2);
    r = r < T(2) * th ? r : T(2) * th;
    return r > T(0) ? r : T(0);
}

template <typename T, int M>
__global__ void k3_update(Env3<T> e)
{
    using L = Upd3Layout<T, M>;
    constexpr int P = M + 4, B = M + 2, BB = B * B, BBB = BB * B, NF = L::NF, MM = M * M * M, LM = Log2M<M>::v;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int nbs[26 * 5];
    T *tile = reinterpret_cast<T *>(smem + L::tile);
    T *A = reinterpret_cast<T *>(smem + L::A);
    T *F = reinterpret_cast<T *>(smem + L::F);
    if ((int)blockIdx.x >= e.count) return;
    const int p = e.list ? e.list[blockIdx.x] : (int)blockIdx.x;
    const int l = e.level[p];
    const T k = e.k[l];
    gather3<T, M>(e, p, tile, nbs);
    __syncthreads();
    const int st[3] = {1, P, P * P};          // tile strides
    const int sa[3] = {1, B, BB};             // band strides
    // (1) fluctuation entering each cell of the band -1 .. M, per direction;
    // a thread sweeps one (i, j) column of the band along z
    for (int q = threadIdx.x; q < 3 * BB; q += blockDim.x) {
        const int d = q / BB, ij = q - d * BB;
        const int i = ij % B - 1, j = ij / B - 1;
        const T s = e.vel[d];
        const int sd = st[d];
        int t = tix3<M>(i, j, -1), a = d * BBB + ij;
        if (s >= T(0)) {
            for (int kk = -1; kk <= M; ++kk, t += P * P, a += BB) A[a] = s * (tile[t] - tile[t - sd]);
        } else {
            for (int kk = -1; kk <= M; ++kk, t += P * P, a += BB) A[a] = s * (tile[t + sd] - tile[t]);
        }
    }
    __syncthreads();
    // (2) correction flux of every face of the patch's cells; a thread sweeps
    // the faces of direction t along t for one column of the other two axes
    // (face index 0 .. M: face c of cells c-1 | c)
    const T k6 = k * k / T(6);
    for (int q = threadIdx.x; q < 3 * M * M; q += blockDim.x) {
        const int t = q >> (2 * LM), rest = q & (M * M - 1);
        const int a1 = t == 0 ? 1 : 0, a2 = t == 2 ? 1 : 2;
        int cc[3];
        cc[a1] = rest & (M - 1);
        cc[a2] = rest >> LM;
        cc[t] = 0;
        const T s = e.vel[t], as = s < T(0) ? -s : s;
        const int stt = st[t], sat = sa[t];
        int ft = tix3<M>(cc[0], cc[1], cc[2]);
        // band index of the upwind cell b of face 0 (b_t = -1 for s > 0, 0 otherwise)
        int bi = (cc[0] + 1) + B * ((cc[1] + 1) + B * (cc[2] + 1)) - (s > T(0) ? sat : 0);
        int fi = t * NF + (M + 1) * rest;
        // the two other directions (d) with their third direction (ee) and corner offset
        const int d0 = a1, d1 = a2;
        const T se0 = e.vel[a2], se1 = e.vel[a1];       // ee of d0 is a2, of d1 is a1
        const T ase0 = se0 < T(0) ? -se0 : se0, ase1 = se1 < T(0) ? -se1 : se1;
        const int off0 = se0 > T(0) ? -sa[a2] : sa[a2], off1 = se1 > T(0) ? -sa[a1] : sa[a1];
        const T kt = T(0.5) * k * s, kc = k6 * s;
        const T kl = T(0.5) * as * (T(1) - k * as);
        for (int ct = 0; ct <= M; ++ct, ft += stt, bi += sat, ++fi) {
            T f = T(0);
            if (e.limiter) {
                const T w = tile[ft] - tile[ft - stt];
                if (w != T(0)) {
                    const T wu = s >= T(0) ? tile[ft - stt] - tile[ft - 2 * stt] : tile[ft + stt] - tile[ft];
                    f = kl * mc3(wu / w) * w;
                }
            }
            if (e.transverse) {
                const T A0 = A[d0 * BBB + bi], A1 = A[d1 * BBB + bi];
                f -= kt * A0;
                f -= kt * A1;
                if (e.transverse == 2) {
                    if (se0 != T(0)) f += kc * ase0 * (A0 - A[d0 * BBB + bi + off0]);
                    if (se1 != T(0)) f += kc * ase1 * (A1 - A[d1 * BBB + bi + off1]);
                }
            }
            F[fi] = f;
        }
    }
    __syncthreads();
    // (3) update and boundary face fluxes
    const int rs = e.fslot[p];
    // side kinds (1 same, 2 coarser, 3 finer): face direction entries of the table
    int skind[6];
    #pragma unroll
    for (int side = 0; side < 6; ++side) {
        const int d26 = 13 + ((side & 1) ? 1 : -1) * (side < 2 ? 1 : (side < 4 ? 3 : 9));
        skind[side] = nbs[(d26 < 13 ? d26 : d26 - 1) * 5];
    }
    const T dtr = e.dtl[l];
    for (int c = threadIdx.x; c < MM; c += blockDim.x) {
        const int i = c & (M - 1), j = (c >> LM) & (M - 1), kk = c >> (2 * LM);
        const int tc = tix3<M>(i, j, kk), ac = (i + 1) + B * ((j + 1) + B * (kk + 1));
        const int cc[3] = {i, j, kk};
        // faces of the cell: direction d, index cc_d (lower) and cc_d + 1 (upper)
        const int f0 = 0 * NF + i + (M + 1) * (j + M * kk);
        const int f1 = 1 * NF + j + (M + 1) * (i + M * kk);
        const int f2 = 2 * NF + kk + (M + 1) * (i + M * j);
        const int fl[3] = {f0, f1, f2};
        T v = tile[tc];
        #pragma unroll
        for (int d = 0; d < 3; ++d) v = v - k * (A[d * BBB + ac] + (F[fl[d] + 1] - F[fl[d]]));
        e.qo[(size_t)p * MM + c] = v;
        if (rs >= 0) {
            // records: dt * flux through the boundary face, set on sides
            // facing a finer leaf, summed over the substeps on sides facing a
            // coarser one (set at the first)
            T *rec = e.flux + (size_t)rs * 6 * M * M;
            #pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
                const T s = e.vel[d], sq = s * tile[tc];
                #pragma unroll
                for (int hi = 0; hi < 2; ++hi) {
                    if (cc[d] != (hi ? M - 1 : 0)) continue;
                    const int kind = skind[2 * d + hi];
                    if (kind != 2 && kind != 3) continue;
                    const T fx = hi ? sq + (s < T(0) ? A[d * BBB + ac] : T(0)) + F[fl[d] + 1]
                                    : sq - (s > T(0) ? A[d * BBB + ac] : T(0)) + F[fl[d]];
                    T *r = rec + (2 * d + hi) * M * M + cc[a2] * M + cc[a1];
                    *r = (kind == 2 && e.ksub > 0) ? *r + dtr * fx : dtr * fx;
                }
            }
        }
    }
}

// coarse-fine correction: one thread per boundary cell of a listed patch;
// the sides of the cell in order 0..5, each next to finer patches taking
// the mean of the four fine face fluxes in place of its own
template <typename T, int M>
__global__ void k3_reflux(Env3<T> e, const int *list, int count)
{
    constexpr int MM = M * M * M, NB = MM - (M - 2) * (M - 2) * (M - 2);
    static_assert(2 * M * M + (M - 2) * 4 * (M - 1) == NB, "boundary cell count");
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)count * NB) return;
    const int p = list[g / NB];
    int r = (int)(g % NB);
    // r-th boundary cell: the bottom layer, the perimeters of the middle
    // layers (row j = 0, row j = M-1, then the two end cells of each row), the top layer
    int i, j, kk;
    constexpr int RING = 4 * (M - 1);
    if (r < M * M) { kk = 0; j = r / M; i = r % M; }
    else if (r < M * M + (M - 2) * RING) {
        r -= M * M;
        kk = 1 + r / RING;
        const int s = r % RING;
        if (s < M) { j = 0; i = s; }
        else if (s < 2 * M) { j = M - 1; i = s - M; }
        else { j = 1 + (s - 2 * M) / 2; i = ((s - 2 * M) & 1) ? M - 1 : 0; }
    } else { r -= M * M + (M - 2) * RING; kk = M - 1; j = r / M; i = r % M; }
    const int l = e.level[p];
    const T k = e.idx[l];                       // records carry dt: (R_c - mean R_f) / dx
    const int cc[3] = {i, j, kk};
    const int N = M << l;
    const int org[3] = {e.x[p] * M, e.y[p] * M, e.z[p] * M};
    T v = e.qo[(size_t)p * MM + i + M * (j + M * kk)];
    for (int side = 0; side < 6; ++side) {
        const int d = side >> 1, hi = side & 1;
        if (cc[d] != (hi ? M - 1 : 0)) continue;
        int dir[3] = {0, 0, 0};
        dir[d] = hi ? 1 : -1;
        int t = (dir[0] + 1) + 3 * (dir[1] + 1) + 9 * (dir[2] + 1);
        t = t < 13 ? t : t - 1;
        const int *en = e.nb + ((size_t)p * 26 + t) * 5;
        if (en[0] != 3) continue;
        const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
        // the cell across and its 2x2 fine face cells
        int gg[3];
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            int vv = org[a] + cc[a] + (a == d ? (hi ? 1 : -1) : 0);
            gg[a] = vv < 0 ? vv + N : (vv >= N ? vv - N : vv);
        }
        const int sub = (((2 * gg[a1]) / M) & 1) | ((((2 * gg[a2]) / M) & 1) << 1);
        const int fr = en[1 + sub];
        if (fr < 0 || e.fslot[fr] < 0 || e.fslot[p] < 0) { *e.err = 1; continue; }
        const T *fx = e.flux + (size_t)e.fslot[fr] * 6 * M * M + (size_t)(2 * d + (hi ? 0 : 1)) * M * M;
        const int fa = (2 * gg[a1]) % M, fb = (2 * gg[a2]) % M;
        const T f0 = fx[fb * M + fa], f1 = fx[fb * M + fa + 1], f2 = fx[(fb + 1) * M + fa],
                f3 = fx[(fb + 1) * M + fa + 1];
        const T fc = e.flux[(size_t)e.fslot[p] * 6 * M * M + (size_t)side * M * M + cc[a2] * M + cc[a1]];
        const T mean = T(0.25) * ((f0 + f1) + (f2 + f3));
        const T delta = k * (fc - mean);
        v = hi ? v + delta : v - delta;
    }
    e.qo[(size_t)p * MM + i + M * (j + M * kk)] = v;
}

}  // namespace fc3
