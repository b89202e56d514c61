// fc_update.cuh -- the one-CTA-per-patch fused update (k_update), shared by
// fc_kernels.cu (the plain method) and fc_update_ext.cu (the same kernel with
// the optional T2 transverse variant and the entropy fix compiled in, EXT).
#pragma once
#include "fc_patch.cuh"

namespace fc {

// ---------------------------------------------------------------------------
// fused update: ghost fill + Riemann solves + limited corrections + transverse
// propagation + conservative update + CFL maximum + coarse-fine registers
// threads per CTA of the fused update: variant 0 / 1 per patch size (the
// autotuner picks one per context)
template <int M, int V> struct UpdCfg {
    static constexpr int NT = M == 8 ? (V ? 192 : 128) : (M == 16 ? (V ? 384 : 352) : (V ? 1024 : 512));
};

template <typename T, int M, int EQ>
struct UpdLayout {
    static constexpr int F = EQ == FC_EQ_SWE ? 3 : 1;
    static constexpr int P = M + 4, PP = P * P;
    static constexpr int ER = EQ == FC_EQ_SWE ? 6 : 2;     // edge record length
    static constexpr int NXE = (M + 2) * (M + 3);           // x-edges rows -1..M, i -1..M+1
    static constexpr int NYE = (M + 3) * (M + 2);           // y-edges rows -1..M+1, i -1..M
    static constexpr int NF = (M + 1) * M;                  // corrected edges per direction
    static constexpr int SLOTS = 2 * 4 * F * NF;            // transverse parts (P2-P3)
    static constexpr int LR = 4 * F * NF;                   // cell contributions (P3-P4), aliases SLOTS
    static constexpr int GEO = EQ == kEqSphere ? geo_size(M) : 0;   // staged patch geometry
    static constexpr size_t elems = (size_t)F * PP + ER * (NXE + NYE) + SLOTS + GEO;
    static constexpr size_t bytes = 64 * sizeof(double) + 9 * sizeof(NbMeta<T>) + 16 + elems * sizeof(T);
};

// Shallow-water edge: Roe record from the two staged cells (tile indices),
// in the edge frame (h, normal momentum, transverse momentum).
template <typename T>
__device__ __forceinline__ void roe_from_tile(const T *tile, int PP, int iL, int iR, int nf, int tf, T g, T *r)
{
    T hL = tile[iL], hR = tile[iR];
    T nL = tile[nf * PP + iL], nR = tile[nf * PP + iR];
    T tL = tile[tf * PP + iL], tR = tile[tf * PP + iR];
    T ihL = fdiv(T(1), hL), ihR = fdiv(T(1), hR);
    swe_roe(hL, nL, tL, nL * ihL, tL * ihL, fsqrt(hL), hR, nR, tR, nR * ihR, tR * ihR, fsqrt(hR), g, r);
}

// Fused update of one patch per CTA:
//  P0 gather patch + ghost ring into shared memory
//  P2 Riemann problem at every edge of the staged tile (records), CFL maximum,
//     and, for the edges whose fluctuations feed perpendicular corrections,
//     the four transverse parts into per-target slots
//  P3 per corrected edge: MC-limited own correction minus the four transverse
//     parts = F~; left/right cell contributions L = A+dQ - F~, R = A-dQ + F~
//  P4 per cell: q - dt/dx (L_x(i) + R_x(i+1)) - dt/dy (L_y(j) + R_y(j+1));
//     coarse-fine registers dt (f(q) -/+ contribution) on marked sides
// Phases P2-P4 of the fused update of patch p (tile filled, geometry staged):
// records, transverse slots, CFL maximum, corrections, update and registers.
template <typename T, int M, int EQ, int NT, bool EXT = false>
__device__ __forceinline__ void update_body(const Env<T> &e, int p, int lev, T dtl, T dtdx, const NbMeta<T> *meta,
                                            const T *tile, T *ex, T *ey, T *s2x, T *s2y, const T *sg, double *red,
                                            int ksub, int fine_acc)
{
    using L = UpdLayout<T, M, EQ>;
    constexpr int F = L::F, P = L::P, PP = L::PP, ER = L::ER;
    constexpr int NXE = L::NXE, NYE = L::NYE, NF = L::NF;
    constexpr bool SPH = EQ == kEqSphere;
    T *Lx = s2x, *Rx = Lx + F * NF, *Ly = Rx + F * NF, *Ry = Ly + F * NF;   // after P3
    (void)P; (void)meta; (void)sg;
    // P2
    T smax = T(0);
    // one body per edge orientation (compile-time), so only the warp that
    // straddles the x/y boundary diverges
    // MODE 0: record and transverse parts at once (T1); MODE 1: record only;
    // MODE 2: transverse parts from the stored record (T2 reads the records
    // of the neighbouring edges for the limited correction it splits)
    auto p2_edge = [&](auto isx_c, auto mode_c, int w) {
        constexpr bool isx = decltype(isx_c)::value;
        constexpr int MODE = decltype(mode_c)::value;
        int i, j, iL, iR;
        T *rec;
        int stride;
        if (isx) {
            int jr = w / (M + 3), ic = w - jr * (M + 3);
            i = ic - 1; j = jr - 1;
            iL = (jr + 1) * P + ic; iR = iL + 1;
            rec = ex + w; stride = NXE;
        } else {
            int q = w - NXE;
            int jr = q / (M + 2), ic = q - jr * (M + 2);
            i = ic - 1; j = jr - 1;
            iL = jr * P + ic + 1; iR = iL + P;
            rec = ey + q; stride = NYE;
        }
        const bool inner = isx ? (i >= 0 && i <= M && j >= 0 && j < M) : (i >= 0 && i < M && j >= 0 && j <= M);
        const bool trans = isx ? (i >= 0 && i <= M) : (j >= 0 && j <= M);
        T am[3], ap[3], am_m[3], am_p[3], ap_m[3], ap_p[3];
        (void)am; (void)ap; (void)am_m; (void)am_p; (void)ap_m; (void)ap_p;
        if constexpr (EQ == FC_EQ_SWE) {
            T r[6];
            if constexpr (MODE != 2) {
                roe_from_tile(tile, PP, iL, iR, isx ? 1 : 2, isx ? 2 : 1, e.g, r);
                for (int k = 0; k < 6; ++k) rec[k * stride] = r[k];
                if (inner) smax = tmax(smax, fabs(r[3]) + r[5]);
            } else {
                for (int k = 0; k < 6; ++k) r[k] = rec[k * stride];
            }
            if (MODE != 1 && trans) {
                // |u| < c and |v| < c at every edge of the warp: subsonic forms
                // (a warp-uniform branch; deciding per edge lets the compiler
                // evaluate both forms)
                bool sub = __all_sync(__activemask(), fabs(r[3]) < r[5] && fabs(r[4]) < r[5]);
                if (sub) swe_fluct_sub(r, am, ap);
                else swe_fluct(r, am, ap);
                if (EXT && e.efix) {
                    const int nf = isx ? 1 : 2;
                    swe_efix(r, tile[iL], tile[nf * PP + iL], tile[iR], tile[nf * PP + iR], e.g, am, ap);
                }
                if constexpr (MODE == 2) {
                    // T2: the fluctuations carry the edge's limited correction cq
                    // (twice the correction flux): A-dQ + cq, A+dQ - cq
                    const int nb = isx ? 1 : (M + 2);
                    T rl[6], rr[6], own[3];
                    for (int k = 0; k < 6; ++k) { rl[k] = rec[k * stride - nb]; rr[k] = rec[k * stride + nb]; }
                    own_correction<T, FC_EQ_SWE>(r, rl, rr, dtdx, own);
                    for (int k = 0; k < 3; ++k) { am[k] += T(2) * own[k]; ap[k] -= T(2) * own[k]; }
                }
                if (sub) {
                    swe_trans_sub(r, am, am_m, am_p);
                    swe_trans_sub(r, ap, ap_m, ap_p);
                } else {
                    swe_trans(r, am, am_m, am_p);
                    swe_trans(r, ap, ap_m, ap_p);
                }
            }
        } else if constexpr (SPH) {
            // capacity form: the edge's own speed; transverse parts take the
            // speed of the edge they cross and 1/kappa of the cell the
            // fluctuation enters (folded into the slot values here)
            T s = isx ? sg[geo_sx(M, i, j)] : sg[geo_sy(M, i, j)];
            T wv = tile[iR] - tile[iL];
            rec[0] = wv;
            rec[stride] = s;
            if (inner) {
                T ik = isx ? tmax(sg[geo_cap(M, i - 1, j)], sg[geo_cap(M, i, j)])
                           : tmax(sg[geo_cap(M, i, j - 1)], sg[geo_cap(M, i, j)]);
                smax = tmax(smax, (T)fabs(s) * ik);
            }
            if (trans) {
                T am0 = tmin(s, T(0)) * wv, ap0 = tmax(s, T(0)) * wv;
                if (!isx) {
                    if (j < M) {
                        T a = ap0 * sg[geo_cap(M, i, j)];
                        if (i >= 0) s2x[(1 * F) * NF + j * (M + 1) + i] = tmin(sg[geo_sx(M, i, j)], T(0)) * a;
                        if (i + 1 <= M) s2x[(0 * F) * NF + j * (M + 1) + i + 1] = tmax(sg[geo_sx(M, i + 1, j)], T(0)) * a;
                    }
                    if (j >= 1) {
                        T a = am0 * sg[geo_cap(M, i, j - 1)];
                        if (i >= 0) s2x[(3 * F) * NF + (j - 1) * (M + 1) + i] = tmin(sg[geo_sx(M, i, j - 1)], T(0)) * a;
                        if (i + 1 <= M)
                            s2x[(2 * F) * NF + (j - 1) * (M + 1) + i + 1] = tmax(sg[geo_sx(M, i + 1, j - 1)], T(0)) * a;
                    }
                } else {
                    if (i < M) {
                        T a = ap0 * sg[geo_cap(M, i, j)];
                        if (j + 1 <= M) s2y[(0 * F) * NF + (j + 1) * M + i] = tmax(sg[geo_sy(M, i, j + 1)], T(0)) * a;
                        if (j >= 0) s2y[(2 * F) * NF + j * M + i] = tmin(sg[geo_sy(M, i, j)], T(0)) * a;
                    }
                    if (i >= 1) {
                        T a = am0 * sg[geo_cap(M, i - 1, j)];
                        if (j + 1 <= M)
                            s2y[(1 * F) * NF + (j + 1) * M + i - 1] = tmax(sg[geo_sy(M, i - 1, j + 1)], T(0)) * a;
                        if (j >= 0) s2y[(3 * F) * NF + j * M + i - 1] = tmin(sg[geo_sy(M, i - 1, j)], T(0)) * a;
                    }
                }
            }
        } else {
            T s = isx ? e.adv_u : e.adv_v;
            T wv = tile[iR] - tile[iL];
            if constexpr (MODE != 2) {
                rec[0] = wv;
                rec[stride] = s;
                if (inner) smax = tmax(smax, (T)fabs(s));
            }
            if (MODE != 1 && trans) {
                am[0] = tmin(s, T(0)) * wv; ap[0] = tmax(s, T(0)) * wv;
                if constexpr (MODE == 2) {
                    const int nb = isx ? 1 : (M + 2);
                    const T r2[2] = {wv, s}, rl[2] = {rec[-nb], s}, rr[2] = {rec[nb], s};
                    T own[1];
                    own_correction<T, FC_EQ_ADV>(r2, rl, rr, dtdx, own);
                    am[0] += T(2) * own[0]; ap[0] -= T(2) * own[0];
                }
                T vt = isx ? e.adv_v : e.adv_u;       // constant transverse speed
                am_m[0] = tmin(vt, T(0)) * am[0]; am_p[0] = tmax(vt, T(0)) * am[0];
                ap_m[0] = tmin(vt, T(0)) * ap[0]; ap_p[0] = tmax(vt, T(0)) * ap[0];
            }
        }
        if constexpr (!SPH && MODE != 1) if (trans) {
            // edge frame -> global components (h, hu, hv): x-edges keep the
            // order, y-edges swap the two momenta
            auto put = [&](T *slot, int sidx, T v0, T v1, T v2) {
                if constexpr (F == 3) {
                    slot[(sidx * 3 + 0) * NF] = v0;
                    slot[(sidx * 3 + 1) * NF] = isx ? v1 : v2;
                    slot[(sidx * 3 + 2) * NF] = isx ? v2 : v1;
                } else slot[sidx * NF] = v0;
            };
#define FC_PUT(sl, k, v) put(sl, k, v[0], F == 3 ? v[1] : T(0), F == 3 ? v[2] : T(0))
            if (!isx) {
                // y-edge (i, j): up-going ap enters cell (i, j): -x part -> x-edge
                // (i, j) slot BR, +x part -> x-edge (i+1, j) slot BL; down-going
                // am enters (i, j-1): -x part -> x-edge (i, j-1) slot AR, +x part
                // -> (i+1, j-1) slot AL
                if (j < M) {
                    if (i >= 0) FC_PUT(s2x + j * (M + 1) + i, 1, ap_m);
                    if (i + 1 <= M) FC_PUT(s2x + j * (M + 1) + i + 1, 0, ap_p);
                }
                if (j >= 1) {
                    if (i >= 0) FC_PUT(s2x + (j - 1) * (M + 1) + i, 3, am_m);
                    if (i + 1 <= M) FC_PUT(s2x + (j - 1) * (M + 1) + i + 1, 2, am_p);
                }
            } else {
                // x-edge (i, j): right-going ap enters cell (i, j): +y part ->
                // y-edge (i, j+1) slot BL, -y part -> y-edge (i, j) slot AL;
                // left-going am enters (i-1, j): +y part -> y-edge (i-1, j+1)
                // slot BR, -y part -> (i-1, j) slot AR
                if (i < M) {
                    if (j + 1 <= M) FC_PUT(s2y + (j + 1) * M + i, 0, ap_p);
                    if (j >= 0) FC_PUT(s2y + j * M + i, 2, ap_m);
                }
                if (i >= 1) {
                    if (j + 1 <= M) FC_PUT(s2y + (j + 1) * M + i - 1, 1, am_p);
                    if (j >= 0) FC_PUT(s2y + j * M + i - 1, 3, am_m);
                }
            }
#undef FC_PUT
        }
    };
    using M0 = std::integral_constant<int, 0>;
    using M1 = std::integral_constant<int, 1>;
    using M2 = std::integral_constant<int, 2>;
    if (SPH || !EXT || !e.t2) {
        #pragma unroll
        for (int w = threadIdx.x; w < NXE + NYE; w += NT) {
            if (w < NXE) p2_edge(std::true_type{}, M0{}, w);
            else p2_edge(std::false_type{}, M0{}, w);
        }
    } else if constexpr (!SPH && EXT) {
        for (int w = threadIdx.x; w < NXE + NYE; w += NT) {
            if (w < NXE) p2_edge(std::true_type{}, M1{}, w);
            else p2_edge(std::false_type{}, M1{}, w);
        }
        __syncthreads();
        for (int w = threadIdx.x; w < NXE + NYE; w += NT) {
            if (w < NXE) p2_edge(std::true_type{}, M2{}, w);
            else p2_edge(std::false_type{}, M2{}, w);
        }
    }
    T bm = block_max<NT, T>(smax, (T *)red);          // contains a barrier
    if (threadIdx.x == 0) atomic_max_nonneg(&e.ctl->smax_bits[lev], (double)bm);

    // P3: correction fluxes and cell contributions of every corrected edge
    constexpr int NIT = (2 * NF + NT - 1) / NT;
    T cl[NIT][F], cr[NIT][F];
    {
        const T kk = T(0.5) * dtdx;
        // one body per edge orientation (compile-time)
        auto p3_edge = [&](auto isx_c, int w, T *clo, T *cro) {
            constexpr bool isx = decltype(isx_c)::value;
            int q = isx ? w : w - NF;
            T r[ER], rl[ER], rr[ER], own[3], am[3], ap[3];
            if (isx) {
                int j = q / (M + 1), i = q - j * (M + 1);
                int base = (j + 1) * (M + 3) + (i + 1);
                for (int k = 0; k < ER; ++k) {
                    r[k] = ex[k * NXE + base]; rl[k] = ex[k * NXE + base - 1]; rr[k] = ex[k * NXE + base + 1];
                }
            } else {
                int j = q / M, i = q - j * M;
                int base = (j + 1) * (M + 2) + (i + 1);
                for (int k = 0; k < ER; ++k) {
                    r[k] = ey[k * NYE + base]; rl[k] = ey[k * NYE + base - (M + 2)]; rr[k] = ey[k * NYE + base + (M + 2)];
                }
            }
            bool drop = false;          // sphere: patch-boundary edge ending at a cube corner
            if constexpr (SPH) {
                // the upwind cell's capacity scales the Courant factor
                int i, j;
                if (isx) { j = q / (M + 1); i = q - j * (M + 1); }
                else { j = q / M; i = q - j * M; }
                const bool up = r[1] >= T(0);
                const T ik = isx ? sg[geo_cap(M, up ? i - 1 : i, j)] : sg[geo_cap(M, i, up ? j - 1 : j)];
                own_correction<T, FC_EQ_ADV>(r, rl, rr, dtdx * ik, own);
                // cube corners (no diagonal neighbour; on the square a missing
                // corner neighbour is a wall, which has ghost cells)
                // on the two-tree sphere every tree corner is such a point
                // (two cells meet there), found by the patch's position
                const int last = (1 << e.f.level[meta[8].id[0]]) - 1, px = meta[8].x[0], py = meta[8].y[0];
                const int cc = e.conn == FC_CONN_PILLOW
                                   ? (px == 0 && py == 0) | (px == last && py == 0) << 1 |
                                         (px == 0 && py == last) << 2 | (px == last && py == last) << 3
                               : e.conn != FC_CONN_SPHERE ? 0 :
                               (meta[4].kind == FC_NB_NONE) | (meta[5].kind == FC_NB_NONE) << 1 |
                               (meta[6].kind == FC_NB_NONE) << 2 | (meta[7].kind == FC_NB_NONE) << 3;
                if (cc) {
                    if (isx)
                        drop = ((cc & 1) && i == 0 && j == 0) || ((cc & 2) && i == M && j == 0) ||
                               ((cc & 4) && i == 0 && j == M - 1) || ((cc & 8) && i == M && j == M - 1);
                    else
                        drop = ((cc & 1) && i == 0 && j == 0) || ((cc & 2) && i == M - 1 && j == 0) ||
                               ((cc & 4) && i == 0 && j == M) || ((cc & 8) && i == M - 1 && j == M);
                }
            } else {
                own_correction<T, EQ>(r, rl, rr, dtdx, own);
            }
            if constexpr (EQ == FC_EQ_SWE) {
                if (__all_sync(__activemask(), fabs(r[3]) < r[5])) swe_fluct_sub(r, am, ap);
                else swe_fluct(r, am, ap);
                if (EXT && e.efix) {
                    int i, j, iL, iR;
                    if (isx) { j = q / (M + 1); i = q - j * (M + 1); iL = tix<M>(i - 1, j); }
                    else { j = q / M; i = q - j * M; iL = tix<M>(i, j - 1); }
                    iR = tix<M>(i, j);
                    const int nf = isx ? 1 : 2;
                    swe_efix(r, tile[iL], tile[nf * PP + iL], tile[iR], tile[nf * PP + iR], e.g, am, ap);
                }
            }
            else { am[0] = tmin(r[1], T(0)) * r[0]; ap[0] = tmax(r[1], T(0)) * r[0]; }
            const T *sl = isx ? s2x : s2y;
            #pragma unroll
            for (int f = 0; f < F; ++f) {
                const int fe = F == 3 ? (isx ? f : (f == 0 ? 0 : 3 - f)) : 0;   // edge-frame index of global f
                T v = own[fe];
                if (!drop)
                    for (int k = 0; k < 4; ++k) v -= kk * sl[(k * F + f) * NF + q];
                clo[f] = ap[fe] - v;
                cro[f] = am[fe] + v;
            }
        };
        #pragma unroll
        for (int it = 0; it < NIT; ++it) {
            int w = threadIdx.x + it * NT;
            if (w < NF) p3_edge(std::true_type{}, w, cl[it], cr[it]);
            else if (w < 2 * NF) p3_edge(std::false_type{}, w, cl[it], cr[it]);
        }
        __syncthreads();                               // slots are dead from here
        #pragma unroll
        for (int it = 0; it < NIT; ++it) {
            int w = threadIdx.x + it * NT;
            if (w < 2 * NF) {
                bool isx = w < NF;
                int q = isx ? w : w - NF;
                T *Ld = isx ? Lx : Ly, *Rd = isx ? Rx : Ry;
                #pragma unroll
                for (int f = 0; f < F; ++f) { Ld[f * NF + q] = cl[it][f]; Rd[f * NF + q] = cr[it][f]; }
            }
        }
    }
    __syncthreads();

    // P4: conservative update, registers
    {
        const int ks = e.kdone[lev] + 1;
        T *qout = qbuf(e, buf_out(e.ctl->start_buf[lev], ks));
        (void)ksub;
        int bad = 0;
        const bool anycf = meta[0].cfslot >= 0 || meta[1].cfslot >= 0 || meta[2].cfslot >= 0 || meta[3].cfslot >= 0;
        #pragma unroll
        for (int c = threadIdx.x; c < M * M; c += NT) {
            int j = c / M, i = c - j * M;
            int fx = j * (M + 1) + i, gy = j * M + i;
            T qc[3];
            const T dtk = SPH ? dtdx * sg[geo_cap(M, i, j)] : dtdx;   // dt / (kappa dx)
            for (int f = 0; f < F; ++f) {
                qc[f] = tile[f * PP + tix<M>(i, j)];
                T X = Lx[f * NF + fx] + Rx[f * NF + fx + 1];
                T Y = Ly[f * NF + gy] + Ry[f * NF + gy + M];
                T qn = (qc[f] - dtk * X) - dtk * Y;
                if (!isfinite(qn)) bad = 1;
                qout[((size_t)f * e.n + p) * (M * M) + c] = qn;
            }
            // effective fluxes through coarse-fine sides, times dt (FP64)
            if (anycf && (i == 0 || i == M - 1 || j == 0 || j == M - 1)) {
                for (int side = 0; side < 4; ++side) {
                    bool on = side == 0 ? i == 0 : side == 1 ? i == M - 1 : side == 2 ? j == 0 : j == M - 1;
                    if (!on) continue;
                    int slot = meta[side].cfslot;
                    if (slot < 0) continue;
                    bool acc = meta[side].kind == FC_NB_COARSER && fine_acc;
                    int along = side < 2 ? j : i;
                    double *rg = e.reg + ((size_t)slot * M + along) * F;
                    for (int f = 0; f < F; ++f) {
                        T fl;
                        if constexpr (SPH) {      // the side edge's speed times the cell value
                            T se = side == 0 ? sg[geo_sx(M, 0, j)] : side == 1 ? sg[geo_sx(M, M, j)]
                                 : side == 2 ? sg[geo_sy(M, i, 0)] : sg[geo_sy(M, i, M)];
                            fl = se * qc[0];
                        } else if (side < 2) {    // x-direction flux of the cell state
                            if constexpr (EQ == FC_EQ_SWE) {
                                T u = qc[1] / qc[0], v = qc[2] / qc[0];
                                fl = f == 0 ? qc[1] : (f == 1 ? qc[1] * u + T(0.5) * e.g * qc[0] * qc[0] : qc[1] * v);
                            } else fl = e.adv_u * qc[0];
                        } else {
                            if constexpr (EQ == FC_EQ_SWE) {
                                T u = qc[1] / qc[0], v = qc[2] / qc[0];
                                fl = f == 0 ? qc[2] : (f == 2 ? qc[2] * v + T(0.5) * e.g * qc[0] * qc[0] : qc[2] * u);
                            } else fl = e.adv_v * qc[0];
                        }
                        T val;
                        if (side == 0) val = fl - Lx[f * NF + fx];
                        else if (side == 1) val = fl + Rx[f * NF + fx + 1];
                        else if (side == 2) val = fl - Ly[f * NF + gy];
                        else val = fl + Ry[f * NF + gy + M];
                        double r = (double)dtl * (double)val;
                        rg[f] = acc ? rg[f] + r : r;
                    }
                }
            }
        }
        if (bad) e.ctl->nonfinite_error = 1;          // every writer stores the same value
    }
}

template <typename T, int M, int EQ, int NT, bool EXT = false>
__global__ void __launch_bounds__(NT)
k_update(Env<T> e, const int *list, int count, int ksub, int fine_acc)
{
    pdl_begin();
    using L = UpdLayout<T, M, EQ>;
    constexpr int F = L::F, PP = L::PP, ER = L::ER;
    constexpr int NXE = L::NXE, NYE = L::NYE, NF = L::NF;
    extern __shared__ __align__(16) unsigned char smem[];
    double *red = (double *)smem;                       // 64 doubles
    NbMeta<T> *meta = (NbMeta<T> *)(red + 64);
    T *s_dt = (T *)(meta + 9);                          // 2 values (16 bytes reserved)
    T *tile = (T *)((unsigned char *)s_dt + 16);
    T *ex = tile + F * PP;
    T *ey = ex + ER * NXE;
    T *s2x = ey + ER * NYE;             // transverse parts into x-edges [4][F][NF]
    T *s2y = s2x + 4 * F * NF;          // transverse parts into y-edges [4][F][NF]
    T *Lx = s2x, *Rx = Lx + F * NF, *Ly = Rx + F * NF, *Ry = Ly + F * NF;   // after P3
    T *sg = s2y + 4 * F * NF;           // sphere: 1/kappa and edge speeds of the patch
    constexpr bool SPH = EQ == kEqSphere;

    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    const int b = blockIdx.x;
    if (b >= count) return;
    const int p = list ? list[b] : b;
    const int lev = e.f.level[p];
    load_meta(e, p, meta);
    if constexpr (SPH) {                // visible after the gather's barriers
        // 16-byte loads from the (256-byte aligned, 16-byte multiple) patch
        // record; element stores, as sg itself is only 8-byte aligned
        using V = typename Vec16<T>::type;
        constexpr int NV = Vec16<T>::n, G = geo_size(M);
        static_assert(G % NV == 0, "patch geometry is a whole number of 16-byte vectors");
        const V *src = reinterpret_cast<const V *>(e.geo + (size_t)p * G);
        for (int v = threadIdx.x; v < G / NV; v += NT) {
            V w = src[v];
            const T *ws = reinterpret_cast<const T *>(&w);
            for (int k = 0; k < NV; ++k) sg[v * NV + k] = ws[k];
        }
    }
    __syncthreads();
    // level step and mesh ratio of this attempt (square cells: dt/dx = dt/dy)
    const T dtl = sizeof(T) == 8 ? (T)e.ctl->dtl_d[lev] : (T)e.ctl->dtl_f[lev];
    const T dtdx = sizeof(T) == 8 ? (T)e.ctl->dtdx_d[lev] : (T)e.ctl->dtdx_f[lev];
    (void)s_dt;

    // P0
    // capacity form: cubed-sphere ghost rules, or those of the square when
    // the geometry is the square's (a swirl velocity field)
    int dry;
    if (SPH && is_sphere_conn(e.conn)) dry = gather_tile<T, M, F, true>(e, meta, tile);
    else dry = gather_tile<T, M, F, false>(e, meta, tile);
    if (dry) {
        if (threadIdx.x == 0) e.ctl->dry_error = 1;
        return;
    }

    update_body<T, M, EQ, NT, EXT>(e, p, lev, dtl, dtdx, meta, tile, ex, ey, s2x, s2y, sg, red, ksub, fine_acc);
}

}  // namespace fc
