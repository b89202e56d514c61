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
#include <type_traits>

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
template <typename T, int M, int EQ, int NT>
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
    auto p2_edge = [&](auto isx_c, int w) {
        constexpr bool isx = decltype(isx_c)::value;
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
            roe_from_tile(tile, PP, iL, iR, isx ? 1 : 2, isx ? 2 : 1, e.g, r);
            for (int k = 0; k < 6; ++k) rec[k * stride] = r[k];
            if (inner) smax = tmax(smax, fabs(r[3]) + r[5]);
            if (trans) {
                // |u| < c and |v| < c at every edge of the warp: subsonic forms
                // (a warp-uniform branch; deciding per edge lets the compiler
                // evaluate both forms)
                bool sub = __all_sync(__activemask(), fabs(r[3]) < r[5] && fabs(r[4]) < r[5]);
                if (sub) {
                    swe_fluct_sub(r, am, ap);
                    swe_trans_sub(r, am, am_m, am_p);
                    swe_trans_sub(r, ap, ap_m, ap_p);
                } else {
                    swe_fluct(r, am, ap);
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
            rec[0] = wv;
            rec[stride] = s;
            if (inner) smax = tmax(smax, (T)fabs(s));
            if (trans) {
                am[0] = tmin(s, T(0)) * wv; ap[0] = tmax(s, T(0)) * wv;
                T vt = isx ? e.adv_v : e.adv_u;       // constant transverse speed
                am_m[0] = tmin(vt, T(0)) * am[0]; am_p[0] = tmax(vt, T(0)) * am[0];
                ap_m[0] = tmin(vt, T(0)) * ap[0]; ap_p[0] = tmax(vt, T(0)) * ap[0];
            }
        }
        if constexpr (!SPH) if (trans) {
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
    #pragma unroll
    for (int w = threadIdx.x; w < NXE + NYE; w += NT) {
        if (w < NXE) p2_edge(std::true_type{}, w);
        else p2_edge(std::false_type{}, w);
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
                const int cc = (meta[4].kind == FC_NB_NONE) | (meta[5].kind == FC_NB_NONE) << 1 |
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

template <typename T, int M, int EQ, int NT>
__global__ void __launch_bounds__(NT)
k_update(Env<T> e, const int *list, int count, int ksub, int fine_acc)
{
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
    int dry = gather_tile<T, M, F, SPH>(e, meta, tile);
    if (dry) {
        if (threadIdx.x == 0) e.ctl->dry_error = 1;
        return;
    }

    update_body<T, M, EQ, NT>(e, p, lev, dtl, dtdx, meta, tile, ex, ey, s2x, s2y, sg, red, ksub, fine_acc);
}

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

// static neighbour record of every patch (rebuilt with the forest): entry d
// (0..7 directions, 8 = the patch) = {kind | level0 << 8 | level1 << 16, id0,
// id1, coarse-tile slot, x0 | y0 << 16, x1 | y1 << 16}
__global__ void k_nbrec(ForestDev f, const int *grslot, int *rec)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= f.n * 9) return;
    int p = g / 9, d = g - 9 * p;
    int kind, id[2];
    if (d == 8) { kind = FC_NB_SAME; id[0] = p; id[1] = -1; }
    else {
        const int *en = f.nbr + (size_t)p * 32 + 4 * d;
        kind = en[0]; id[0] = en[1]; id[1] = en[2];
    }
    int lv[2] = {0, 0}, xy[2] = {0, 0};
    for (int k = 0; k < 2; ++k)
        if ((unsigned)id[k] < (unsigned)f.n) { lv[k] = f.level[id[k]]; xy[k] = f.x[id[k]] | (f.y[id[k]] << 16); }
        else id[k] = -1;
    int *r = rec + (size_t)p * kRecInts + 6 * d;
    r[0] = kind | (lv[0] << 8) | (lv[1] << 16);
    r[1] = id[0]; r[2] = id[1];
    r[3] = (kind == FC_NB_COARSER && id[0] >= 0) ? (grslot ? grslot[id[0]] : id[0]) : -1;
    r[4] = xy[0]; r[5] = xy[1];
    if (d == 8) { r[6] = 0; r[7] = 0; }            // padding to kRecInts
}

int launch_nbrec(const ForestDev &f, const int *grslot, int *rec, cudaStream_t s)
{
    if (f.n <= 0) return FC_OK;
    k_nbrec<<<(f.n * 9 + 255) / 256, 256, 0, s>>>(f, grslot, rec);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

// ---------------------------------------------------------------------------
// complete tiles (interior + ghosts) of listed patches, written to e.gr
template <typename T, int M, int F, bool SG>
__global__ void k_fill_tiles(Env<T> e, const int *list, int count)
{
    constexpr int P = M + 4, PP = P * P;
    extern __shared__ __align__(16) unsigned char smem[];
    NbMeta<T> *meta = (NbMeta<T> *)smem;
    T *tile = (T *)(smem + ((9 * sizeof(NbMeta<T>) + 15) / 16) * 16);
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    int b = blockIdx.x;
    if (b >= count) return;
    int p = list ? list[b] : b;
    load_meta(e, p, meta);
    __syncthreads();
    gather_tile<T, M, F, SG>(e, meta, tile);
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
    if (e.conn == FC_CONN_SPHERE) {
        // the fine cells across each side are located by their centres; the
        // fine patch's side facing p and the index along it come from its
        // own tree, and both fluxes are compared as leaving the coarse cell
        constexpr int LM = Log2M<M>::v;
        const int sh = kMaxBits - lev - LM;
        const long long wc = 1LL << sh, wf = wc / 2;
        const double ik = (double)e.geo[(size_t)p * geo_size(M) + geo_cap(M, i, j)];
        const long long X0 = ((long long)e.f.x[p] * M + i) * wc, Y0 = ((long long)e.f.y[p] * M + j) * wc;
        for (int side = 0; side < 4; ++side) {
            bool on = side == 0 ? i == 0 : side == 1 ? i == M - 1 : side == 2 ? j == 0 : j == M - 1;
            if (!on || nbp[4 * side] != FC_NB_FINER) continue;
            int c = side < 2 ? j : i;
            int sc = e.cfslot[p * 4 + side];
            if (sc < 0) { e.ctl->index_error = 1; return; }
            double rin[F];
            for (int f = 0; f < F; ++f) rin[f] = 0.0;
            for (int h = 0; h < 2; ++h) {
                long long a = h == 0 ? wf / 2 : wf + wf / 2, X, Y, Xm, Ym;
                if (side == 0) { X = X0 - wf / 2; Y = Y0 + a; }
                else if (side == 1) { X = X0 + wc + wf / 2; Y = Y0 + a; }
                else if (side == 2) { X = X0 + a; Y = Y0 - wf / 2; }
                else { X = X0 + a; Y = Y0 + wc + wf / 2; }
                if (cube_map_point(e.f.tree[p], X, Y, &Xm, &Ym) < 0) { e.ctl->index_error = 1; return; }
                const int fx = (int)(Xm >> (sh - 1)), fy = (int)(Ym >> (sh - 1));
                int fine = -1;
                for (int k = 1; k <= 2; ++k) {
                    int cand = nbp[4 * side + k];
                    if ((unsigned)cand < (unsigned)e.n && e.f.x[cand] == (fx >> LM) && e.f.y[cand] == (fy >> LM))
                        fine = cand;
                }
                if (fine < 0) { e.ctl->index_error = 1; return; }
                int sf = -1;
                for (int d = 0; d < 4; ++d) {
                    const int *en = e.f.nbr + (size_t)fine * 32 + 4 * d;
                    if (en[0] == FC_NB_COARSER && en[1] == p) sf = d;
                }
                int slot = sf < 0 ? -1 : e.cfslot[fine * 4 + sf];
                if (slot < 0) { e.ctl->index_error = 1; return; }
                int along = sf < 2 ? fy - e.f.y[fine] * M : fx - e.f.x[fine] * M;
                double sgf = (sf & 1) ? -1.0 : 1.0;          // into the fine patch through side sf
                for (int f = 0; f < F; ++f) rin[f] += sgf * e.reg[((size_t)slot * M + along) * F + f];
            }
            double sgc = (side & 1) ? 1.0 : -1.0;
            for (int f = 0; f < F; ++f) {
                double rc = e.reg[((size_t)sc * M + c) * F + f];
                double corr = ((sgc * rc - 0.5 * rin[f]) / dx) * ik;
                size_t o = ((size_t)f * e.n + p) * (M * M) + j * M + i;
                q[o] = (T)((double)q[o] + corr);
            }
        }
        return;
    }
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
        } else if (e.conn != FC_CONN_SPHERE) {
            v = fmax(v, fmax(fabs((double)e.adv_u), fabs((double)e.adv_v)));
        }
    }
    if (e.conn == FC_CONN_SPHERE) {
        // edges touching the interior: |speed| over the smaller capacity
        const T *g = e.geo + (size_t)p * geo_size(e.m);
        const int m = e.m;
        for (int c = threadIdx.x; c < m * (m + 1); c += blockDim.x) {
            int j = c / (m + 1), i = c - j * (m + 1);
            double kx = fmax((double)g[geo_cap(m, i - 1, j)], (double)g[geo_cap(m, i, j)]);
            double ky = fmax((double)g[geo_cap(m, j, i - 1)], (double)g[geo_cap(m, j, i)]);
            v = fmax(v, fmax(fabs((double)g[geo_sx(m, i, j)]) * kx, fabs((double)g[geo_sy(m, j, i)]) * ky));
        }
    }
    double bm = block_max<256, double>(v, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&e.ctl->smax_bits[lev], bm);
}

// per-level step and dt/dx of the coming attempt (first node of every step)
__global__ void k_level_dt(StepCtl *c, int lmin, int lmax, int subcycle, DxTab tab)
{
    int l = threadIdx.x;
    if (blockIdx.x || l >= kMaxLevels) return;
    double dt = c->dt;
    if (subcycle && l >= lmin) dt = dt / (double)(1 << (l - lmin));
    double r = dt / tab.dx[l];
    c->dtl_d[l] = dt; c->dtdx_d[l] = r;
    c->dtl_f[l] = (float)dt; c->dtdx_f[l] = (float)r;
}

int launch_level_dt(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, cudaStream_t s)
{
    DxTab tab;
    for (int l = 0; l < kMaxLevels; ++l) { tab.dx[l] = dx[l]; tab.nsub[l] = 0; }
    k_level_dt<<<1, 32, 0, s>>>(ctl, lmin, lmax, subcycle, tab);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
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
        } else if (kind == FC_INIT_HILL) {
            // Gaussian of the great-circle distance to (lon0, lat0), at the
            // mapped cell centre
            const long long w2 = 2 * ((1LL << (kMaxBits - lev)) / m);
            const long long U = ((long long)e.f.x[p] * m + i) * w2 + w2 / 2 - kCubeN;
            const long long V = ((long long)e.f.y[p] * m + j) * w2 + w2 / 2 - kCubeN;
            double pt[3], ce[3] = {__dmul_rn(cos(pr[1]), cos(pr[0])), __dmul_rn(cos(pr[1]), sin(pr[0])), sin(pr[1])};
            sph_point(e.f.tree[p], U, V, pt);
            double d0 = pt[0] - ce[0], d1 = pt[1] - ce[1], d2 = pt[2] - ce[2];
            double ch = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
            double d = 2.0 * asin(ch < 2.0 ? 0.5 * ch : 1.0);
            v0 = exp(-(__dmul_rn(d, d) / __dmul_rn(pr[2], pr[2])));
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
    if (e.conn == FC_CONN_SPHERE) {   // capacity-weighted: kappa = 1 / (stored inverse)
        const T *g = e.geo + (size_t)p * geo_size(e.m);
        for (int c = threadIdx.x; c < mm; c += blockDim.x) {
            double kap = 1.0 / (double)g[geo_cap(e.m, c % e.m, c / e.m)];
            for (int f = 0; f < F; ++f) acc[f] += kap * (double)q[((size_t)f * e.n + p) * mm + c];
        }
    } else
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

template <typename T, int M, int F, bool SG>
__global__ void k_tag(Env<T> e, int crit, double thr, int8_t *flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    NbMeta<T> *meta = (NbMeta<T> *)smem;
    T *tile = (T *)(smem + ((9 * sizeof(NbMeta<T>) + 15) / 16) * 16);
    __shared__ int hit;
    int p = blockIdx.x;
    if (p >= e.n) return;
    load_meta(e, p, meta);
    if (threadIdx.x == 0) hit = 0;
    __syncthreads();
    gather_tile<T, M, F, SG>(e, meta, tile);
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

// cubed sphere (one field): capacity-weighted parent averages; children by
// limited interpolation, then shifted per old cell so that the new cells
// inside it carry its mass (kappa_old r^2 q_old) exactly in real arithmetic
// (an old cell lies inside one new leaf while r <= m; deeper refinement keeps
// the plain interpolation)
template <typename T, int M>
__global__ void k_transfer_sphere(Env<T> eo, Env<T> en, const int *origin, const T *tiles_old, const int *old_x,
                                  const int *old_y)
{
    constexpr int P = M + 4, PP = P * P, H = M / 2, MM = M * M, G = geo_size(M);
    int k = blockIdx.x;
    if (k >= en.n) return;
    int kind = origin[3 * k], o = origin[3 * k + 1], dl = origin[3 * k + 2];
    T *qn = en.q[0] + (size_t)k * MM;
    const T *gn = en.geo + (size_t)k * G;
    if (kind == 0) {
        const T *a = qbuf(eo, eo.ctl->start_buf[eo.f.level[o]]) + (size_t)o * MM;
        for (int c = threadIdx.x; c < MM; c += blockDim.x) qn[c] = a[c];
        return;
    }
    if (kind == 2) {
        for (int c = threadIdx.x; c < MM; c += blockDim.x) {
            int i = c % M, j = c / M;
            int ch = o + (i >= H) + 2 * (j >= H);
            const T *a = qbuf(eo, eo.ctl->start_buf[eo.f.level[ch]]) + (size_t)ch * MM;
            const T *go = eo.geo + (size_t)ch * G;
            int fi = 2 * (i % H), fj = 2 * (j % H);
            double k00 = 1.0 / (double)go[geo_cap(M, fi, fj)], k10 = 1.0 / (double)go[geo_cap(M, fi + 1, fj)];
            double k01 = 1.0 / (double)go[geo_cap(M, fi, fj + 1)], k11 = 1.0 / (double)go[geo_cap(M, fi + 1, fj + 1)];
            double ks = (k00 + k10) + (k01 + k11);
            double v = ((k00 * (double)a[fj * M + fi] + k10 * (double)a[fj * M + fi + 1]) +
                        (k01 * (double)a[(fj + 1) * M + fi] + k11 * (double)a[(fj + 1) * M + fi + 1])) / ks;
            qn[c] = (T)v;
        }
        return;
    }
    const int r = 1 << dl, rb = r < M ? r : M, nb = M / rb;
    const T *A = tiles_old + (size_t)o * PP;
    const T *go = eo.geo + (size_t)o * G;
    for (int bb = threadIdx.x; bb < nb * nb; bb += blockDim.x) {
        int bi = bb % nb, bj = bb / nb;
        int gi0 = en.f.x[k] * M + bi * rb, gj0 = en.f.y[k] * M + bj * rb;
        int ci = gi0 / r - old_x[o] * M, cj = gj0 / r - old_y[o] * M;
        T qc = A[tix<M>(ci, cj)];
        T sx = minmod(A[tix<M>(ci + 1, cj)] - qc, qc - A[tix<M>(ci - 1, cj)]);
        T sy = minmod(A[tix<M>(ci, cj + 1)] - qc, qc - A[tix<M>(ci, cj - 1)]);
        double ksum = 0.0, mass = 0.0;
        for (int jj = 0; jj < rb; ++jj)
            for (int ii = 0; ii < rb; ++ii) {
                int gi = gi0 + ii, gj = gj0 + jj;
                T sgx = (T)(((double)(gi % r) + 0.5) / r - 0.5);
                T sgy = (T)(((double)(gj % r) + 0.5) / r - 0.5);
                T v = radd(radd(qc, rmul(sgx, sx)), rmul(sgy, sy));
                int c = (bj * rb + jj) * M + bi * rb + ii;
                qn[c] = v;
                double kap = 1.0 / (double)gn[geo_cap(M, bi * rb + ii, bj * rb + jj)];
                ksum += kap;
                mass += kap * (double)v;
            }
        if (r > M) continue;
        double want = (1.0 / (double)go[geo_cap(M, ci, cj)]) * (double)(r * r) * (double)qc;
        double d = (want - mass) / ksum;
        for (int jj = 0; jj < rb; ++jj)
            for (int ii = 0; ii < rb; ++ii) {
                int c = (bj * rb + jj) * M + bi * rb + ii;
                qn[c] = (T)((double)qn[c] + d);
            }
    }
}

// cubed sphere: geometry of every patch (one block per patch)
template <typename T, int M>
__global__ void k_geometry(Env<T> e, double omega, double tilt, T *geo)
{
    int p = blockIdx.x;
    if (p >= e.n) return;
    const int lev = e.f.level[p], t = e.f.tree[p];
    const long long w2 = 2 * ((1LL << (kMaxBits - lev)) / M);
    const double dxi = level_dx(lev, M);
    const long long Ub = (long long)e.f.x[p] * M * w2 - kCubeN, Vb = (long long)e.f.y[p] * M * w2 - kCubeN;
    T *g = geo + (size_t)p * geo_size(M);
    for (int c = threadIdx.x; c < geo_size(M); c += blockDim.x) {
        double v, pa[3], pb[3];
        if (c < geo_ncap(M)) {
            int i = c % (M + 2) - 1, j = c / (M + 2) - 1;
            long long U0 = Ub + i * w2, V0 = Vb + j * w2;
            double kap = sph_cell_area(t, U0, U0 + w2, V0, V0 + w2) / __dmul_rn(dxi, dxi);
            v = 1.0 / kap;
        } else if (c < geo_ncap(M) + geo_nedge(M)) {   // x-edge: psi(top) - psi(bottom)
            int q = c - geo_ncap(M), i = q % (M + 3) - 1, j = q / (M + 3) - 1;
            long long U = Ub + i * w2, V0 = Vb + j * w2;
            sph_point(t, U, V0, pa);
            sph_point(t, U, V0 + w2, pb);
            v = __dadd_rn(sph_psi(omega, tilt, pb), -sph_psi(omega, tilt, pa)) / dxi;
        } else {                                         // y-edge: psi(left) - psi(right)
            int q = c - geo_ncap(M) - geo_nedge(M), i = q % (M + 2) - 1, j = q / (M + 2) - 1;
            long long U0 = Ub + i * w2, V = Vb + j * w2;
            sph_point(t, U0, V, pa);
            sph_point(t, U0 + w2, V, pb);
            v = __dadd_rn(sph_psi(omega, tilt, pa), -sph_psi(omega, tilt, pb)) / dxi;
        }
        g[c] = (T)v;
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
    k_update<T, M, EQ, NT><<<l.count, NT, Lay::bytes, s>>>(e, l.idx, l.count, ksub, fine_acc);
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
    k_update_pipe<T, M, EQ, NT><<<grid, NT, Lay::bytes, s>>>(e, l.idx, l.count, ksub, fine_acc);
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
    if (e.eq == FC_EQ_SWE) {
        if (e.m == 8) return launch_update_v<T, 8, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
        if (e.m == 16) return launch_update_v<T, 16, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
        if constexpr (sizeof(T) == 4)      // FP64 m = 32 shallow water does not fit shared memory
            if (e.m == 32) return launch_update_v<T, 32, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
    } else if (e.conn == FC_CONN_SPHERE) {
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

template <typename T, int M, int F>
static size_t tile_smem() { return ((9 * sizeof(NbMeta<T>) + 15) / 16) * 16 + (size_t)F * (M + 4) * (M + 4) * sizeof(T); }

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
    if (e.conn == FC_CONN_SPHERE) {
        if (e.m == 8) k_fill_tiles<T, 8, 1, true><<<l.count, 256, tile_smem<T, 8, 1>(), s>>>(e, l.idx, l.count);
        else if (e.m == 16) k_fill_tiles<T, 16, 1, true><<<l.count, 256, tile_smem<T, 16, 1>(), s>>>(e, l.idx, l.count);
        else k_fill_tiles<T, 32, 1, true><<<l.count, 256, tile_smem<T, 32, 1>(), s>>>(e, l.idx, l.count);
    } else
        FC_DISPATCH_MF(e, (k_fill_tiles<T, M, F, false><<<l.count, 256, tile_smem<T, M, F>(), s>>>(e, l.idx, l.count)));
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
    if (e.conn == FC_CONN_SPHERE) {
        if (e.m == 8) k_tag<T, 8, 1, true><<<e.n, 256, tile_smem<T, 8, 1>(), s>>>(e, crit, thr, d_flags);
        else if (e.m == 16) k_tag<T, 16, 1, true><<<e.n, 256, tile_smem<T, 16, 1>(), s>>>(e, crit, thr, d_flags);
        else k_tag<T, 32, 1, true><<<e.n, 256, tile_smem<T, 32, 1>(), s>>>(e, crit, thr, d_flags);
    } else
        FC_DISPATCH_MF(e, (k_tag<T, M, F, false><<<e.n, 256, tile_smem<T, M, F>(), s>>>(e, crit, thr, d_flags)));
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
    if (enew.conn == FC_CONN_SPHERE) {
        if (enew.m == 8) k_transfer_sphere<T, 8><<<enew.n, 256, 0, s>>>(eold, enew, origin, tiles_old, old_x, old_y);
        else if (enew.m == 16) k_transfer_sphere<T, 16><<<enew.n, 256, 0, s>>>(eold, enew, origin, tiles_old, old_x, old_y);
        else k_transfer_sphere<T, 32><<<enew.n, 256, 0, s>>>(eold, enew, origin, tiles_old, old_x, old_y);
    } else
    FC_DISPATCH_MF(enew, (k_transfer<T, M, F><<<enew.n, 256, 0, s>>>(eold, enew, origin, tiles_old, old_x, old_y)));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_geometry(const Env<T> &e, double omega, double tilt, T *geo, cudaStream_t s)
{
    if (e.n <= 0) return FC_OK;
    if (e.m == 8) k_geometry<T, 8><<<e.n, 256, 0, s>>>(e, omega, tilt, geo);
    else if (e.m == 16) k_geometry<T, 16><<<e.n, 256, 0, s>>>(e, omega, tilt, geo);
    else k_geometry<T, 32><<<e.n, 256, 0, s>>>(e, omega, tilt, geo);
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
    template int launch_update<T>(const Env<T> &, List, int, int, int, cudaStream_t);                         \
    template int launch_fill_tiles<T>(const Env<T> &, List, cudaStream_t);                                    \
    template int launch_reflux<T>(const Env<T> &, List, cudaStream_t);                                        \
    template int launch_cell_rate<T>(const Env<T> &, cudaStream_t);                                           \
    template int launch_init<T>(const Env<T> &, int, const double *, int, cudaStream_t);                      \
    template int launch_sums<T>(const Env<T> &, double *, double *, cudaStream_t);                            \
    template int launch_tag<T>(const Env<T> &, int, double, int, int8_t *, cudaStream_t);                     \
    template int launch_transfer<T>(const Env<T> &, const Env<T> &, const int *, const T *, const int *,      \
                                    const int *, cudaStream_t);                                               \
    template int launch_geometry<T>(const Env<T> &, double, double, T *, cudaStream_t);                       \
    template int launch_read<T>(const Env<T> &, int, T *, cudaStream_t);                                      \
    template int launch_write<T>(const Env<T> &, const T *, cudaStream_t);

FC_INSTANTIATE(float)
FC_INSTANTIATE(double)

}  // namespace fc
