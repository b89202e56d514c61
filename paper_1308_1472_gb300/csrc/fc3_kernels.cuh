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
    const T *q;            // state
    T *qo;                 // next state
    T *gr;                 // complete tiles
    T *flux;               // face-flux records
    T vel[3];
    T k[kMaxLevel + 1];    // dt / dx per level
    int limiter, transverse;
    int *err;              // set to 1 when a table entry points nowhere (nothing read then)
};

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

// value of cell (i, j, k) of patch p (any of -2 .. M+1; not interior)
template <typename T, int M>
__device__ T ghost3(const Env3<T> &e, int p, int l, int i, int j, int k)
{
    constexpr int MM = M * M * M;
    const int N = M << l;
    const int li[3] = {i, j, k};
    const int org[3] = {e.x[p] * M, e.y[p] * M, e.z[p] * M};
    int g[3], dir[3];
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = org[a] + li[a];
        g[a] = v < 0 ? v + N : (v >= N ? v - N : v);
        dir[a] = li[a] < 0 ? -1 : (li[a] >= M ? 1 : 0);
    }
    int t = (dir[0] + 1) + 3 * (dir[1] + 1) + 9 * (dir[2] + 1);
    t = t < 13 ? t : t - 1;
    const int *en = e.nb + ((size_t)p * 26 + t) * 5;
    const int kind = en[0];
    if (kind == 1) {
        if (en[1] < 0) { *e.err = 1; return T(0); }
        const T *Q = e.q + (size_t)en[1] * MM;
        return Q[(g[0] % M) + M * ((g[1] % M) + M * (g[2] % M))];
    }
    if (kind == 2) {
        const int ts = en[1] >= 0 ? e.tslot[en[1]] : -1;
        if (ts < 0) { *e.err = 1; return T(0); }
        const T *A = e.gr + (size_t)ts * P3<M>();
        const int ci = (g[0] >> 1) % M, cj = (g[1] >> 1) % M, ck = (g[2] >> 1) % M;
        const T qc = A[tix3<M>(ci, cj, ck)];
        const T sx = mm3(A[tix3<M>(ci + 1, cj, ck)] - qc, qc - A[tix3<M>(ci - 1, cj, ck)]);
        const T sy = mm3(A[tix3<M>(ci, cj + 1, ck)] - qc, qc - A[tix3<M>(ci, cj - 1, ck)]);
        const T sz = mm3(A[tix3<M>(ci, cj, ck + 1)] - qc, qc - A[tix3<M>(ci, cj, ck - 1)]);
        const T ox = (g[0] & 1) ? T(0.25) : T(-0.25), oy = (g[1] & 1) ? T(0.25) : T(-0.25),
                oz = (g[2] & 1) ? T(0.25) : T(-0.25);
        return ((qc + ox * sx) + oy * sy) + oz * sz;
    }
    // finer: the 2x2x2 cells 2g + {0,1}^3 of the finer leaf beside the patch
    int sub = 0, nbits = 0;
    #pragma unroll
    for (int a = 0; a < 3; ++a)
        if (dir[a] == 0) { sub |= (((2 * g[a]) / M) & 1) << nbits; ++nbits; }
    if (kind != 3 || en[1 + sub] < 0) { *e.err = 1; return T(0); }
    const T *Q = e.q + (size_t)en[1 + sub] * MM;
    const int fi = (2 * g[0]) % M, fj = (2 * g[1]) % M, fk = (2 * g[2]) % M;
    auto at = [&](int a, int b, int c) { return Q[(fi + a) + M * ((fj + b) + M * (fk + c))]; };
    const T s0 = at(0, 0, 0) + at(1, 0, 0), s1 = at(0, 1, 0) + at(1, 1, 0);
    const T s2 = at(0, 0, 1) + at(1, 0, 1), s3 = at(0, 1, 1) + at(1, 1, 1);
    return T(0.125) * ((s0 + s1) + (s2 + s3));
}

// complete tile of patch p into shared memory (all threads of the CTA)
template <typename T, int M>
__device__ void gather3(const Env3<T> &e, int p, T *tile)
{
    constexpr int P = M + 4, PPP = P * P * P, MM = M * M * M;
    const int l = e.level[p];
    const T *Q = e.q + (size_t)p * MM;
    for (int c = threadIdx.x; c < PPP; c += blockDim.x) {
        const int i = c % P - 2, j = (c / P) % P - 2, k = c / (P * P) - 2;
        T v;
        if (i >= 0 && i < M && j >= 0 && j < M && k >= 0 && k < M) v = Q[i + M * (j + M * k)];
        else v = ghost3<T, M>(e, p, l, i, j, k);
        tile[c] = v;
    }
}

// complete tiles of the listed patches (one level per launch, coarsest first)
template <typename T, int M>
__global__ void k3_fill_tiles(Env3<T> e, const int *list, int count)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *tile = reinterpret_cast<T *>(smem);
    if (blockIdx.x >= count) return;
    const int p = list[blockIdx.x];
    gather3<T, M>(e, p, tile);
    __syncthreads();
    T *dst = e.gr + (size_t)e.tslot[p] * P3<M>();
    for (int c = threadIdx.x; c < P3<M>(); c += blockDim.x) dst[c] = tile[c];
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
    constexpr int P = M + 4, B = M + 2, BBB = B * B * B, NF = L::NF, MM = M * M * M;
    extern __shared__ __align__(16) unsigned char smem[];
    T *tile = reinterpret_cast<T *>(smem + L::tile);
    T *A = reinterpret_cast<T *>(smem + L::A);
    T *F = reinterpret_cast<T *>(smem + L::F);
    const int p = blockIdx.x;
    if (p >= e.n) return;
    const int l = e.level[p];
    const T k = e.k[l];
    gather3<T, M>(e, p, tile);
    __syncthreads();
    const int st[3] = {1, P, P * P};
    // (1) fluctuation entering each cell of the band -1 .. M, per direction
    for (int c = threadIdx.x; c < 3 * BBB; c += blockDim.x) {
        const int d = c / BBB, r = c - d * BBB;
        const int i = r % B - 1, j = (r / B) % B - 1, kk = r / (B * B) - 1;
        const int t = tix3<M>(i, j, kk);
        const T s = e.vel[d];
        A[c] = s >= T(0) ? s * (tile[t] - tile[t - st[d]]) : s * (tile[t + st[d]] - tile[t]);
    }
    __syncthreads();
    // (2) correction flux of every face of the patch's cells: face index
    // 0 .. M along its direction (face z of cells z-1 | z), 0 .. M-1 across
    auto aix = [](int i, int j, int kk) { return (i + 1) + B * ((j + 1) + B * (kk + 1)); };
    for (int c = threadIdx.x; c < 3 * NF; c += blockDim.x) {
        const int t = c / NF, r = c - t * NF;
        int cc[3];
        cc[t] = r % (M + 1);
        const int rest = r / (M + 1);
        const int a1 = t == 0 ? 1 : 0, a2 = t == 2 ? 1 : 2;
        cc[a1] = rest % M;
        cc[a2] = rest / M;
        const T s = e.vel[t];
        const int ft = tix3<M>(cc[0], cc[1], cc[2]);
        T f = T(0);
        if (e.limiter) {
            const T w = tile[ft] - tile[ft - st[t]];
            if (w != T(0)) {
                const T wu = s >= T(0) ? tile[ft - st[t]] - tile[ft - 2 * st[t]] : tile[ft + st[t]] - tile[ft];
                const T as = s < T(0) ? -s : s;
                f = T(0.5) * as * (T(1) - k * as) * mc3(wu / w) * w;
            }
        }
        if (e.transverse) {
            int b[3] = {cc[0], cc[1], cc[2]};
            if (s > T(0)) b[t] -= 1;                               // upwind cell along t
            const int bi = aix(b[0], b[1], b[2]);
            #pragma unroll
            for (int d = 0; d < 3; ++d)
                if (d != t) f -= T(0.5) * k * s * A[d * BBB + bi];
            if (e.transverse == 2) {
                #pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d == t) continue;
                    const int ee = 3 - d - t;
                    const T se = e.vel[ee];
                    if (se == T(0)) continue;
                    int b2[3] = {b[0], b[1], b[2]};
                    b2[ee] += se > T(0) ? -1 : 1;
                    const T ase = se < T(0) ? -se : se;
                    f += (k * k / T(6)) * s * ase * (A[d * BBB + bi] - A[d * BBB + aix(b2[0], b2[1], b2[2])]);
                }
            }
        }
        F[c] = f;
    }
    __syncthreads();
    // (3) update and boundary face fluxes
    auto fix = [](int t, int i, int j, int kk) {
        const int cc[3] = {i, j, kk};
        const int a1 = t == 0 ? 1 : 0, a2 = t == 2 ? 1 : 2;
        return t * NF + cc[t] + (M + 1) * (cc[a1] + M * cc[a2]);
    };
    const int rs = e.fslot[p];
    for (int c = threadIdx.x; c < MM; c += blockDim.x) {
        const int i = c % M, j = (c / M) % M, kk = c / (M * M);
        const int tc = tix3<M>(i, j, kk), ac = aix(i, j, kk);
        T v = tile[tc];
        const int cc[3] = {i, j, kk};
        #pragma unroll
        for (int d = 0; d < 3; ++d) {
            int up[3] = {i, j, kk};
            up[d] += 1;
            const T dF = F[fix(d, up[0], up[1], up[2])] - F[fix(d, i, j, kk)];
            v = v - k * (A[d * BBB + ac] + dF);
        }
        e.qo[(size_t)p * MM + c] = v;
        if (rs >= 0) {
            #pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
                const T s = e.vel[d], sq = s * tile[tc];
                T *rec = e.flux + (size_t)rs * 6 * M * M;
                if (cc[d] == 0)
                    rec[(2 * d) * M * M + cc[a2] * M + cc[a1]] =
                        sq - (s > T(0) ? A[d * BBB + ac] : T(0)) + F[fix(d, i, j, kk)];
                if (cc[d] == M - 1) {
                    int up[3] = {i, j, kk};
                    up[d] += 1;
                    rec[(2 * d + 1) * M * M + cc[a2] * M + cc[a1]] =
                        sq + (s < T(0) ? A[d * BBB + ac] : T(0)) + F[fix(d, up[0], up[1], up[2])];
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
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)count * NB) return;
    const int p = list[g / NB];
    int r = (int)(g % NB);
    // r-th boundary cell in [k][j][i] order
    int i = 0, j = 0, kk = 0;
    for (int c = 0, seen = 0; c < MM; ++c) {
        const int ci = c % M, cj = (c / M) % M, ck = c / (M * M);
        const bool bd = ci == 0 || ci == M - 1 || cj == 0 || cj == M - 1 || ck == 0 || ck == M - 1;
        if (!bd) continue;
        if (seen == r) { i = ci; j = cj; kk = ck; break; }
        ++seen;
    }
    const int l = e.level[p];
    const T k = e.k[l];
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
