// fc_kernels.cu -- sm_103a kernels of the patch method.
//
// Sec. 3 of the paper (LeVeque's wave propagation on an m x m patch with two
// ghost layers; ghost values by same-level copy, fine-to-coarse averaging and
// limited conservative coarse-to-fine interpolation, time-interpolated under
// sub-cycling; regrid by interpolation / averaging) and Sec. 4 (global or
// per-level dt, fine-to-coarse correction), Sec. 5 (per-patch tagging).
//
// The fused patch update and its launchers are in fc_update.cuh /
// fc_update_launch.cuh (instantiated in fc_update_f32.cu, fc_update_f64.cu);
// the row sweep in fc_sweep.cuh.
#include <cstdio>
#include <type_traits>

#include "fc_patch.cuh"

namespace fc {

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
// complete tiles (interior + ghosts) of listed patches, written to e.gr.
// Threads per CTA: 256 on the spheres; on the square 160 for FP32 shallow
// water with m = 16, held to 32 registers so that 12 CTAs fit on an SM (a launch over the tiles
// of one level then runs in one wave where it has up to 12 x the SM count of
// tiles), else 192: the interior (3 m^2 / 4 vectors for m = 16) and the ghost
// ring (8m + 16 cells) in one or two passes
template <typename T, int M, int F, bool SG>
struct FillShape {
    static constexpr bool kPacked = !SG && M == 16 && F == 3 && sizeof(T) == 4;
    static constexpr int threads = SG ? 256 : kPacked ? 160 : 192;
    static constexpr int min_blocks = kPacked ? 12 : 1;
};

template <typename T, int M, int F, bool SG>
__global__ void __launch_bounds__(FillShape<T, M, F, SG>::threads, FillShape<T, M, F, SG>::min_blocks)
k_fill_tiles(Env<T> e, const int *list, int count)
{
    pdl_trigger();
    constexpr int P = M + 4, PP = P * P;
    extern __shared__ __align__(16) unsigned char smem[];
    NbMeta<T> *meta = (NbMeta<T> *)smem;
    T *tile = (T *)(smem + ((9 * sizeof(NbMeta<T>) + 15) / 16) * 16);
    const int b = blockIdx.x;
    if (b >= count) return;
    // the forest's part first (list, tile slot, and on the square the
    // patch's static neighbour record), before the wait for the previous
    // kernel of the step
    const int p = list ? list[b] : b;
    const int slot = e.grslot ? e.grslot[p] : p;
    NbMeta<T> m;
    if constexpr (!SG)
        if (threadIdx.x < 9) meta_static(e, e.nbrec + (size_t)p * kRecInts + 6 * threadIdx.x, (int)threadIdx.x, m);
    pdl_wait();
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    if constexpr (SG) load_meta(e, p, meta);
    else if (threadIdx.x < 9) {
        meta_time(e, e.ctl->start_buf, m);
        meta[threadIdx.x] = m;
    }
    __syncthreads();
    gather_tile<T, M, F, SG>(e, meta, tile);
    // the tile is a whole number of 16-byte vectors, 16-byte aligned on both sides
    using V = int4;
    constexpr int NV = (int)(F * PP * sizeof(T) / sizeof(V));
    static_assert(F * PP * sizeof(T) % sizeof(V) == 0, "tile of whole vectors");
    V *dst = reinterpret_cast<V *>(e.gr + (size_t)slot * F * PP);
    const V *src = reinterpret_cast<const V *>(tile);
    for (int t = threadIdx.x; t < NV; t += blockDim.x) dst[t] = src[t];
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
    pdl_trigger();
    constexpr int NB = 4 * M - 4;
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count * NB) return;
    int p = patches[g / NB], b = g % NB;
    int i, j;
    if (b < M) { i = b; j = 0; }
    else if (b < 2 * M) { i = b - M; j = M - 1; }
    else if (b < 3 * M - 2) { i = 0; j = b - 2 * M + 1; }
    else { i = M - 1; j = b - (3 * M - 2) + 1; }
    const int lev = e.f.level[p];
    const double dx = level_dx(lev, M);
    const int *nbp = e.f.nbr + (size_t)p * 32;
    if (!is_sphere_conn(e.conn)) {
        // the forest's part before the wait for the previous kernel: the sides
        // of this cell that face finer leaves (at most two), the fine leaf
        // across each and both register slots
        int ns = 0, bad = 0, sd[2], scs[2], sfs[2];
        #pragma unroll
        for (int side = 0; side < 4; ++side) {
            const bool on = side == 0 ? i == 0 : side == 1 ? i == M - 1 : side == 2 ? j == 0 : j == M - 1;
            if (!on || nbp[4 * side] != FC_NB_FINER) continue;
            const int c = side < 2 ? j : i;
            const int fine = c < M / 2 ? nbp[4 * side + 1] : nbp[4 * side + 2];
            int sc = -1, sf = -1;
            if ((unsigned)fine < (unsigned)e.n) { sc = e.cfslot[p * 4 + side]; sf = e.cfslot[fine * 4 + (side ^ 1)]; }
            else bad = 1;
            if (ns < 2) { sd[ns] = side; scs[ns] = sc; sfs[ns] = sf; ++ns; }
        }
        pdl_wait();
        if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
        const int s = e.ctl->start_buf[lev];
        T *q = qbuf(e, e.kdone[lev] == 0 ? s : buf_out(s, e.kdone[lev]));
        for (int k = 0; k < ns; ++k) {
            const int side = sd[k], sc = scs[k], sf = sfs[k];
            if (bad || sc < 0 || sf < 0) { e.ctl->index_error = 1; return; }
            const int c = side < 2 ? j : i, kf = 2 * (c % (M / 2));
            const double sg = (side & 1) ? 1.0 : -1.0;
            for (int f = 0; f < F; ++f) {
                double rc = e.reg[((size_t)sc * M + c) * F + f];
                double r0 = e.reg[((size_t)sf * M + kf) * F + f];
                double r1 = e.reg[((size_t)sf * M + kf + 1) * F + f];
                double corr = (rc - 0.5 * (r0 + r1)) / dx;
                size_t o = ((size_t)f * e.n + p) * (M * M) + j * M + i;
                q[o] = (T)((double)q[o] + sg * corr);
            }
        }
        return;
    }
    pdl_wait();
    if (e.ctl->dry_error | e.ctl->nonfinite_error | e.ctl->index_error) return;
    int s = e.ctl->start_buf[lev];
    T *q = qbuf(e, e.kdone[lev] == 0 ? s : buf_out(s, e.kdone[lev]));
    {
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
                if (sphere_map_point(e.conn, e.f.tree[p], X, Y, &Xm, &Ym) < 0) { e.ctl->index_error = 1; return; }
                const int fx = (int)(Xm >> (sh - 1)), fy = (int)(Ym >> (sh - 1));
                int fine = -1;
                for (int k = 1; k <= 2; ++k) {
                    int cand = nbp[4 * side + k];
                    if ((unsigned)cand < (unsigned)e.n && e.f.x[cand] == (fx >> LM) && e.f.y[cand] == (fy >> LM))
                        fine = cand;
                }
                if (fine < 0) { e.ctl->index_error = 1; return; }
                // the fine side facing p: outward normal opposite to the
                // image of this side's outward normal (a fine corner patch of
                // the two-tree sphere faces p across two of its sides)
                long long Xn, Yn;
                if (sphere_map_point(e.conn, e.f.tree[p], X + (side == 0 ? -1 : side == 1 ? 1 : 0),
                                     Y + (side == 2 ? -1 : side == 3 ? 1 : 0), &Xn, &Yn) < 0) {
                    e.ctl->index_error = 1;
                    return;
                }
                const int sf = Xn > Xm ? 0 : Xn < Xm ? 1 : Yn > Ym ? 2 : 3;
                const int *en = e.f.nbr + (size_t)fine * 32 + 4 * sf;
                int slot = en[0] == FC_NB_COARSER && en[1] == p ? e.cfslot[fine * 4 + sf] : -1;
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
    }
}

// ---------------------------------------------------------------------------
// step control: Courant number, accept / retake, next dt (one warp: a lane
// per level for the wave-speed maxima and the per-level steps, lane 0 for the
// decision)
struct DxTab { double dx[kMaxLevels]; int nsub[kMaxLevels]; };

__global__ void k_step_ctl(StepCtl *c, int lmin, int lmax, int subcycle, DxTab tab)
{
    pdl_begin();
    const int l = threadIdx.x;
    if (blockIdx.x || l >= 32) return;
    const int err = l == 0 ? (c->dry_error | c->nonfinite_error | c->index_error) : 0;
    if (__shfl_sync(0xffffffffu, err, 0)) return;       // the whole warp
    double rate = 0.0;
    if (l >= lmin && l <= lmax) {
        rate = fmax(rate, __longlong_as_double((long long)c->smax_bits[l]) / tab.dx[subcycle ? lmin : l]);
        c->smax_bits[l] = 0ULL;
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    double dt_next = 0.0;
    if (l == 0) {
        double dt = c->dt, nu = dt * rate;
        bool accept = nu <= 1.0 || c->dt_fixed > 0.0 || c->attempts == 3;
        if (accept) {
            c->t += dt;
            c->last_dt = dt;
            c->last_courant = nu;
            c->accepted += 1;
            for (int k = lmin; k <= lmax; ++k)
                if (tab.nsub[k] > 0) c->start_buf[k] = buf_out(c->start_buf[k], tab.nsub[k]);
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
        dt_next = c->dt;
    }
    dt_next = __shfl_sync(0xffffffffu, dt_next, 0);
    // per-level step and dt/dx of the next attempt (as k_level_dt)
    if (l < kMaxLevels) {
        double dl = dt_next;
        if (subcycle && l >= lmin) dl = dl / (double)(1 << (l - lmin));
        const double r = dl / tab.dx[l];
        c->dtl_d[l] = dl; c->dtdx_d[l] = r;
        c->dtl_f[l] = (float)dl; c->dtdx_f[l] = (float)r;
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
            // in the state's precision (GB300's FP64 rate is a small fraction
            // of its FP32 rate); the maximum is kept in FP64
            const T h = q[((size_t)0 * e.n + p) * mm + c];
            const T u = q[((size_t)1 * e.n + p) * mm + c] / h;
            const T w = q[((size_t)2 * e.n + p) * mm + c] / h;
            const T cc = sqrt(e.g * h);
            v = fmax(v, (double)tmax(fabs(u) + cc, fabs(w) + cc));
        } else if (!e.geo) {
            v = fmax(v, fmax(fabs((double)e.adv_u), fabs((double)e.adv_v)));
        }
    }
    if (F == 1 && e.geo) {
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

// per-level step and dt/dx of the coming attempt (after the host sets the
// step size; k_step_ctl sets them for the attempts that follow a step)
__global__ void k_level_dt(StepCtl *c, int lmin, int lmax, int subcycle, DxTab tab)
{
    pdl_begin();
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
    FC_CUDA(launch_pdl(k_level_dt, 1, 32, 0, s, ctl, lmin, lmax, subcycle, tab));
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
            if (e.conn == FC_CONN_PILLOW) pil_point(e.f.tree[p], U, V, pt);
            else sph_point(e.f.tree[p], U, V, pt);
            double d0 = pt[0] - ce[0], d1 = pt[1] - ce[1], d2 = pt[2] - ce[2];
            double ch = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
            double d = 2.0 * asin(ch < 2.0 ? 0.5 * ch : 1.0);
            v0 = exp(-(__dmul_rn(d, d) / __dmul_rn(pr[2], pr[2])));
        } else if (kind == FC_INIT_HALF) {
            // Example 2: 1 on the half of the sphere facing (lon, lat), else 0
            const long long w2 = 2 * ((1LL << (kMaxBits - lev)) / m);
            const long long U = ((long long)e.f.x[p] * m + i) * w2 + w2 / 2 - kCubeN;
            const long long V = ((long long)e.f.y[p] * m + j) * w2 + w2 / 2 - kCubeN;
            double pt[3], ce[3] = {__dmul_rn(cos(pr[1]), cos(pr[0])), __dmul_rn(cos(pr[1]), sin(pr[0])), sin(pr[1])};
            if (e.conn == FC_CONN_PILLOW) pil_point(e.f.tree[p], U, V, pt);
            else sph_point(e.f.tree[p], U, V, pt);
            v0 = __dadd_rn(__dadd_rn(__dmul_rn(pt[0], ce[0]), __dmul_rn(pt[1], ce[1])), __dmul_rn(pt[2], ce[2])) > 0.0
                     ? 1.0 : 0.0;
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
    if (is_sphere_conn(e.conn)) {   // capacity-weighted: kappa = 1 / (stored inverse)
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
    if (!is_sphere_conn(e.conn)) {
        // square, swirl (stream function amplitude sin^2(pi x) sin^2(pi y) / pi,
        // amplitude e.adv_u): capacity 1, normal velocity of an edge =
        // difference of the stream function between its ends / edge length.
        // The stream function is a product of one factor per axis, evaluated
        // once per node column and row of the patch (nodes -1 .. M+2).
        __shared__ double sx2[M + 4], sy2[M + 4];
        const double dx = level_dx(e.f.level[p], M), amp = (double)e.adv_u;
        const long long i0 = (long long)e.f.x[p] * M, j0 = (long long)e.f.y[p] * M;
        for (int k = threadIdx.x; k < 2 * (M + 4); k += blockDim.x) {
            const int a = k < M + 4 ? k : k - (M + 4);
            const double sn = sin(M_PI * ((double)((k < M + 4 ? i0 : j0) + a - 1) * dx));
            (k < M + 4 ? sx2 : sy2)[a] = sn * sn;
        }
        __syncthreads();
        auto psi = [&](int i, int j) { return amp * (sx2[i + 1] * sy2[j + 1]) / M_PI; };   // node (i, j)
        T *g = geo + (size_t)p * geo_size(M);
        for (int c = threadIdx.x; c < geo_size(M); c += blockDim.x) {
            double v;
            if (c < geo_ncap(M)) v = 1.0;
            else if (c < geo_ncap(M) + geo_nedge(M)) {          // x-edge: psi(top) - psi(bottom)
                int q = c - geo_ncap(M), i = q % (M + 3) - 1, j = q / (M + 3) - 1;
                v = (psi(i, j + 1) - psi(i, j)) / dx;
            } else {                                            // y-edge: psi(left) - psi(right)
                int q = c - geo_ncap(M) - geo_nedge(M), i = q % (M + 2) - 1, j = q / (M + 2) - 1;
                v = (psi(i, j) - psi(i + 1, j)) / dx;
            }
            g[c] = (T)v;
        }
        return;
    }
    const int lev = e.f.level[p], t = e.f.tree[p];
    const long long w2 = 2 * ((1LL << (kMaxBits - lev)) / M);
    const double dxi = level_dx(lev, M);
    const bool pil = e.conn == FC_CONN_PILLOW;
    __shared__ double glx[kGl], glw[kGl];          // quadrature of the two-tree sphere's areas
    if (pil && threadIdx.x < kGl) gl_node(threadIdx.x, &glx[threadIdx.x], &glw[threadIdx.x]);
    __syncthreads();
    const long long Ub = (long long)e.f.x[p] * M * w2 - kCubeN, Vb = (long long)e.f.y[p] * M * w2 - kCubeN;
    T *g = geo + (size_t)p * geo_size(M);
    for (int c = threadIdx.x; c < geo_size(M); c += blockDim.x) {
        double v, pa[3], pb[3];
        if (c < geo_ncap(M)) {
            int i = c % (M + 2) - 1, j = c / (M + 2) - 1;
            long long U0 = Ub + i * w2, V0 = Vb + j * w2;
            double kap = (pil ? pil_cell_area(glx, glw, t, U0, U0 + w2, V0, V0 + w2)
                              : sph_cell_area(t, U0, U0 + w2, V0, V0 + w2)) / __dmul_rn(dxi, dxi);
            v = 1.0 / kap;
        } else if (c < geo_ncap(M) + geo_nedge(M)) {   // x-edge: psi(top) - psi(bottom)
            int q = c - geo_ncap(M), i = q % (M + 3) - 1, j = q / (M + 3) - 1;
            long long U = Ub + i * w2, V0 = Vb + j * w2;
            if (pil) { pil_point(t, U, V0, pa); pil_point(t, U, V0 + w2, pb); }
            else { sph_point(t, U, V0, pa); sph_point(t, U, V0 + w2, pb); }
            v = __dadd_rn(sph_psi(omega, tilt, pb), -sph_psi(omega, tilt, pa)) / dxi;
        } else {                                         // y-edge: psi(left) - psi(right)
            int q = c - geo_ncap(M) - geo_nedge(M), i = q % (M + 2) - 1, j = q / (M + 2) - 1;
            long long U0 = Ub + i * w2, V = Vb + j * w2;
            if (pil) { pil_point(t, U0, V, pa); pil_point(t, U0 + w2, V, pb); }
            else { sph_point(t, U0, V, pa); sph_point(t, U0 + w2, V, pb); }
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

// k_write for shallow water, with each patch's largest cell speed
// max(|u| + c, |v| + c) folded into its level's maximum as k_cell_speed does
// (the same expression in the state's precision, the same loop and block
// reduction), so that the first step after a written state needs no separate
// pass over the cells for its step size
template <typename T>
__global__ void k_write_swe(Env<T> e, const T *src)
{
    __shared__ double red[32];
    int p = blockIdx.x;
    if (p >= e.n) return;
    int mm = e.m * e.m, lev = e.f.level[p];
    T *q = qbuf(e, e.ctl->start_buf[lev]);
    double v = 0.0;
    for (int c = threadIdx.x; c < mm; c += blockDim.x) {
        const T h = src[((size_t)p * 3 + 0) * mm + c], hu = src[((size_t)p * 3 + 1) * mm + c],
                hv = src[((size_t)p * 3 + 2) * mm + c];
        q[((size_t)0 * e.n + p) * mm + c] = h;
        q[((size_t)1 * e.n + p) * mm + c] = hu;
        q[((size_t)2 * e.n + p) * mm + c] = hv;
        const T u = hu / h, w = hv / h;
        const T cc = sqrt(e.g * h);
        v = fmax(v, (double)tmax(fabs(u) + cc, fabs(w) + cc));
    }
    double bm = block_max<256, double>(v, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&e.ctl->smax_bits[lev], bm);
}

// ---------------------------------------------------------------------------
// launchers
static inline int blocks_of(long long n, int b) { return (int)((n + b - 1) / b); }

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
    if (is_sphere_conn(e.conn)) {
        if (e.m == 8) FC_CUDA(launch_pdl(k_fill_tiles<T, 8, 1, true>, l.count, 256, tile_smem<T, 8, 1>(), s, e, l.idx, l.count));
        else if (e.m == 16) FC_CUDA(launch_pdl(k_fill_tiles<T, 16, 1, true>, l.count, 256, tile_smem<T, 16, 1>(), s, e, l.idx, l.count));
        else FC_CUDA(launch_pdl(k_fill_tiles<T, 32, 1, true>, l.count, 256, tile_smem<T, 32, 1>(), s, e, l.idx, l.count));
    } else
        FC_DISPATCH_MF(e, FC_CUDA(launch_pdl(k_fill_tiles<T, M, F, false>, l.count, FillShape<T, M, F, false>::threads,
                                             tile_smem<T, M, F>(), s, e, l.idx, l.count)));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T>
int launch_reflux(const Env<T> &e, List patches, cudaStream_t s)
{
    if (patches.count <= 0) return FC_OK;
    FC_DISPATCH_MF(e, FC_CUDA(launch_pdl(k_reflux<T, M, F>, blocks_of((long long)patches.count * (4 * M - 4), 128), 128,
                                         0, s, e, patches.idx, patches.count)));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

int launch_step_ctl(StepCtl *ctl, int lmin, int lmax, int subcycle, const double *dx, const int *nsub,
                    cudaStream_t s)
{
    DxTab tab;
    for (int l = 0; l < kMaxLevels; ++l) { tab.dx[l] = dx[l]; tab.nsub[l] = nsub[l]; }
    FC_CUDA(launch_pdl(k_step_ctl, 1, 32, 0, s, ctl, lmin, lmax, subcycle, tab));
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
    if (is_sphere_conn(e.conn)) {
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
    if (is_sphere_conn(enew.conn)) {
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

template <typename T>
int launch_write_speed(const Env<T> &e, const T *src, cudaStream_t s)
{
    if (e.F != 3) { set_error("launch_write_speed: shallow water only"); return FC_ERR_INVALID_ARG; }
    if (e.n > 0) k_write_swe<T><<<e.n, 256, 0, s>>>(e, src);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

#define FC_INSTANTIATE(T)                                                                                     \
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
    template int launch_write<T>(const Env<T> &, const T *, cudaStream_t);                                    \
    template int launch_write_speed<T>(const Env<T> &, const T *, cudaStream_t);

FC_INSTANTIATE(float)
FC_INSTANTIATE(double)

}  // namespace fc
