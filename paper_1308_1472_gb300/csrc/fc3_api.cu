// fc3_api.cu -- context, octree and step plan of the three-dimensional patch
// solver (include/fc3.h).  The octree lives on the host (balance, neighbour
// tables and regrid maps are rebuilt when it changes and uploaded); fields,
// ghost fill, update, coarse-fine correction, tagging reductions and regrid
// transfer run in the kernels of fc3_kernels.cuh and of this file.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "../../include/fc3.h"
#include "fc3_kernels.cuh"
#include "fc_forest.cuh"

namespace fc3 {

using fc::cuda_status;
using fc::set_error;

// ---------------------------------------------------------------------------
// Morton keys of (x, y, z), 20 bits per axis, x in the lowest bit
constexpr int kBits = 20;
static uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}
static uint64_t key3(int l, int x, int y, int z)
{
    const int s = kBits - l;
    return spread3((uint32_t)x << s) | (spread3((uint32_t)y << s) << 1) | (spread3((uint32_t)z << s) << 2);
}
static uint64_t span3(int l) { return (uint64_t)1 << (3 * (kBits - l)); }
static int wrapi(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

struct Leaf3 {
    uint64_t key;
    int l, x, y, z;
};

struct Forest3 {
    std::vector<Leaf3> L;
    std::unordered_map<uint64_t, int> H;     // (level, Morton key) of every leaf -> its index
    int n() const { return (int)L.size(); }
    static uint64_t hkey(int l, int x, int y, int z) { return ((uint64_t)l << 60) | key3(l, x, y, z); }
    // rebuild the index after L changed (every function here that changes L calls it)
    void index()
    {
        H.clear();
        H.reserve(L.size() * 2);
        for (int i = 0; i < n(); ++i) H.emplace(hkey(L[i].l, L[i].x, L[i].y, L[i].z), i);
    }
    void sort()
    {
        std::sort(L.begin(), L.end(), [](const Leaf3 &a, const Leaf3 &b) { return a.key < b.key; });
        index();
    }
    // leaf containing the level-g block (a, b, c), or the first leaf inside it
    // (the leaf holding its lower corner): hash lookups at level g, g - 1,
    // then finer levels at the corner, then the remaining coarser levels
    int locate(int g, int a, int b, int c) const
    {
        auto at = [&](int l) -> int {
            const int x = l <= g ? a >> (g - l) : a << (l - g), y = l <= g ? b >> (g - l) : b << (l - g),
                      z = l <= g ? c >> (g - l) : c << (l - g);
            auto it = H.find(hkey(l, x, y, z));
            return it == H.end() ? -1 : it->second;
        };
        int r = at(g);
        if (r >= 0) return r;
        if (g > 0 && (r = at(g - 1)) >= 0) return r;
        for (int l = g + 1; l <= kMaxLevel; ++l)
            if ((r = at(l)) >= 0) return r;
        for (int l = g - 2; l >= 0; --l)
            if ((r = at(l)) >= 0) return r;
        return -1;
    }
    bool covers() const
    {
        uint64_t at = 0;
        for (const Leaf3 &f : L) {
            if (f.key != at) return false;
            at += span3(f.l);
        }
        return at == span3(0);
    }
    // coarsest leaf touching leaf i in direction (dx, dy, dz), -1 if finer leaves cover that side
    int touching(int i, int dx, int dy, int dz) const
    {
        const Leaf3 &f = L[i];
        const int w = 1 << f.l;
        const int j = locate(f.l, wrapi(f.x + dx, w), wrapi(f.y + dy, w), wrapi(f.z + dz, w));
        return (j < 0 || L[j].l > f.l) ? -1 : j;
    }
    bool balanced() const
    {
        for (int i = 0; i < n(); ++i)
            for (int d = 0; d < 27; ++d) {
                if (d == 13) continue;
                const int j = touching(i, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1);
                if (j >= 0 && L[j].l < L[i].l - 1) return false;
            }
        return true;
    }
    void refine(const std::vector<char> &mark)
    {
        std::vector<Leaf3> out;
        out.reserve(L.size() + 7 * std::count(mark.begin(), mark.end(), 1));
        for (int i = 0; i < n(); ++i) {
            if (!mark[i]) { out.push_back(L[i]); continue; }
            for (int c = 0; c < 8; ++c) {
                Leaf3 f{0, L[i].l + 1, 2 * L[i].x + (c & 1), 2 * L[i].y + ((c >> 1) & 1), 2 * L[i].z + (c >> 2)};
                f.key = key3(f.l, f.x, f.y, f.z);
                out.push_back(f);
            }
        }
        L.swap(out);           // children replace their parent in place: the order stays Morton
        index();
    }
    int balance(int max_level)
    {
        for (;;) {
            std::vector<char> mark(n(), 0);
            bool any = false;
            for (int i = 0; i < n(); ++i)
                for (int d = 0; d < 27; ++d) {
                    if (d == 13) continue;
                    const int j = touching(i, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1);
                    if (j >= 0 && L[j].l < L[i].l - 1) { mark[j] = 1; any = true; }
                }
            if (!any) return FC_OK;
            for (int i = 0; i < n(); ++i)
                if (mark[i] && L[i].l >= max_level) {
                    set_error("2:1 balance needs a level above max_level");
                    return FC_ERR_INVALID_ARG;
                }
            refine(mark);
        }
    }
    bool is_family(int i) const
    {
        if (i + 8 > n() || L[i].l == 0) return false;
        const Leaf3 &f = L[i];
        if ((f.x & 1) || (f.y & 1) || (f.z & 1)) return false;
        for (int c = 0; c < 8; ++c) {
            const Leaf3 &g = L[i + c];
            if (g.l != f.l || g.x != f.x + (c & 1) || g.y != f.y + ((c >> 1) & 1) || g.z != f.z + (c >> 2)) return false;
        }
        return true;
    }
};

// neighbour table, tile slots, record slots and lists of a forest
struct Tables {
    std::vector<int> nb, tslot, fslot, fill, fill_off, reflux;
    std::vector<int> lvl, lvl_off, rfl, rfl_off;     // patches and correction lists by level
    int ntile = 0, nrec = 0;
};

static int build_tables(const Forest3 &F, Tables &T)
{
    const int n = F.n();
    T.nb.assign((size_t)n * 26 * 5, -1);
    T.tslot.assign(n, -1);
    T.fslot.assign(n, -1);
    std::vector<char> has_finer(n, 0), face_other(n, 0), face_finer(n, 0);
    for (int i = 0; i < n; ++i) {
        const Leaf3 &f = F.L[i];
        const int w = 1 << f.l;
        int t = 0;
        for (int d = 0; d < 27; ++d) {
            if (d == 13) continue;
            const int dir[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
            const bool face = std::abs(dir[0]) + std::abs(dir[1]) + std::abs(dir[2]) == 1;
            const int b[3] = {wrapi(f.x + dir[0], w), wrapi(f.y + dir[1], w), wrapi(f.z + dir[2], w)};
            int *en = &T.nb[((size_t)i * 26 + t) * 5];
            const int r = F.locate(f.l, b[0], b[1], b[2]);
            if (r < 0) { set_error("neighbour search failed"); return FC_ERR_INVALID_ARG; }
            const int lr = F.L[r].l;
            if (lr == f.l) { en[0] = 1; en[1] = r; }
            else if (lr == f.l - 1) { en[0] = 2; en[1] = r; if (face) face_other[i] = 1; }
            else if (lr > f.l) {                 // finer leaves cover the block (the first may lie
                en[0] = 3;                          // on its far side, two levels finer)
                has_finer[i] = 1;
                if (face) { face_other[i] = 1; face_finer[i] = 1; }
                int free_ax[3], nf = 0;
                for (int a = 0; a < 3; ++a) if (dir[a] == 0) free_ax[nf++] = a;
                for (int s = 0; s < (1 << nf); ++s) {
                    int c[3];
                    for (int a = 0; a < 3; ++a) c[a] = 2 * b[a] + (dir[a] > 0 ? 0 : 1);
                    for (int q = 0; q < nf; ++q) c[free_ax[q]] = 2 * b[free_ax[q]] + ((s >> q) & 1);
                    const int fr = F.locate(f.l + 1, c[0], c[1], c[2]);
                    if (fr < 0 || F.L[fr].l != f.l + 1) { set_error("forest is not 2:1 balanced"); return FC_ERR_UNBALANCED; }
                    en[1 + s] = fr;
                }
            } else {
                set_error("forest is not 2:1 balanced");
                return FC_ERR_UNBALANCED;
            }
            ++t;
        }
    }
    // complete tiles of the patches next to a finer patch, by level; records
    // of the patches next (by a face) to another level; correction list
    T.fill.clear();
    T.fill_off.assign(kMaxLevel + 2, 0);
    T.ntile = 0;
    for (int l = 0; l <= kMaxLevel; ++l) {
        T.fill_off[l] = (int)T.fill.size();
        for (int i = 0; i < n; ++i)
            if (F.L[i].l == l && has_finer[i]) { T.tslot[i] = T.ntile++; T.fill.push_back(i); }
    }
    T.fill_off[kMaxLevel + 1] = (int)T.fill.size();
    T.nrec = 0;
    T.reflux.clear();
    for (int i = 0; i < n; ++i) {
        if (face_other[i]) T.fslot[i] = T.nrec++;
        if (face_finer[i]) T.reflux.push_back(i);
    }
    T.lvl.clear(); T.rfl.clear();
    T.lvl_off.assign(kMaxLevel + 2, 0);
    T.rfl_off.assign(kMaxLevel + 2, 0);
    for (int l = 0; l <= kMaxLevel; ++l) {
        T.lvl_off[l] = (int)T.lvl.size();
        T.rfl_off[l] = (int)T.rfl.size();
        for (int i = 0; i < n; ++i)
            if (F.L[i].l == l) {
                T.lvl.push_back(i);
                if (face_finer[i]) T.rfl.push_back(i);
            }
    }
    T.lvl_off[kMaxLevel + 1] = (int)T.lvl.size();
    T.rfl_off[kMaxLevel + 1] = (int)T.rfl.size();
    return FC_OK;
}

// ---------------------------------------------------------------------------
// kernels of this file
template <typename T, int M>
__global__ void k3_init(int n, const int *lv, const int *x, const int *y, const int *z, int kind, const double *a, T *q)
{
    constexpr int MM = M * M * M;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)n * MM) return;
    const int p = (int)(g / MM), c = (int)(g % MM);
    const int i = c % M, j = (c / M) % M, k = c / (M * M);
    const double dx = 1.0 / ((double)M * (double)(1 << lv[p]));
    const double xc = ((double)x[p] * M + i + 0.5) * dx, yc = ((double)y[p] * M + j + 0.5) * dx,
                 zc = ((double)z[p] * M + k + 0.5) * dx;
    double v;
    if (kind == FC3_INIT_BOX) v = (xc >= a[0] && xc < a[1] && yc >= a[2] && yc < a[3] && zc >= a[4] && zc < a[5]) ? a[6] : a[7];
    else if (kind == FC3_INIT_SINE) v = a[0] + a[1] * sin(2.0 * M_PI * (a[2] * xc + a[3] * yc + a[4] * zc));
    else {
        const double ex = xc - a[2], ey = yc - a[3], ez = zc - a[4];
        v = a[0] + a[1] * exp(-(ex * ex + ey * ey + ez * ez) / (a[5] * a[5]));
    }
    q[g] = (T)v;
}

// per patch: sum of q dx^3 (FP64) and max - min
template <typename T, int M>
__global__ void k3_patch_stats(int n, const int *lv, const T *q, double *sum, T *range)
{
    constexpr int MM = M * M * M;
    __shared__ double ss[256];
    __shared__ T smin[256], smax[256];
    const int p = blockIdx.x;
    if (p >= n) return;
    const T *Q = q + (size_t)p * MM;
    double s = 0.0;
    T lo = Q[0], hi = Q[0];
    for (int c = threadIdx.x; c < MM; c += blockDim.x) {
        const T v = Q[c];
        s += (double)v;
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    ss[threadIdx.x] = s; smin[threadIdx.x] = lo; smax[threadIdx.x] = hi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            smin[threadIdx.x] = smin[threadIdx.x + w] < smin[threadIdx.x] ? smin[threadIdx.x + w] : smin[threadIdx.x];
            smax[threadIdx.x] = smax[threadIdx.x + w] > smax[threadIdx.x] ? smax[threadIdx.x + w] : smax[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double dx = 1.0 / ((double)M * (double)(1 << lv[p]));
        if (sum) sum[p] = ss[0] * (dx * dx * dx);
        if (range) range[p] = smax[0] - smin[0];
    }
}

// max - min of the parent of each listed family (8 leaves from list[f]):
// parent cells are the means of 2x2x2 children, paired as in the ghost fill
template <typename T, int M>
__global__ void k3_family_range(const int *list, int count, const T *q, T *range)
{
    constexpr int MM = M * M * M, H = M / 2;
    __shared__ T smin[256], smax[256];
    const int f = blockIdx.x;
    if (f >= count) return;
    const int i0 = list[f];
    T lo = T(0), hi = T(0);
    bool first = true;
    for (int c = threadIdx.x; c < MM; c += blockDim.x) {
        const int I = c % M, J = (c / M) % M, K = c / (M * M);
        const int ch = (I >= H) + 2 * (J >= H) + 4 * (K >= H);
        const T *Q = q + (size_t)(i0 + ch) * MM;
        const int fi = 2 * (I % H), fj = 2 * (J % H), fk = 2 * (K % H);
        auto at = [&](int a, int b, int d) { return Q[(fi + a) + M * ((fj + b) + M * (fk + d))]; };
        const T s0 = at(0, 0, 0) + at(1, 0, 0), s1 = at(0, 1, 0) + at(1, 1, 0);
        const T s2 = at(0, 0, 1) + at(1, 0, 1), s3 = at(0, 1, 1) + at(1, 1, 1);
        const T v = T(0.125) * ((s0 + s1) + (s2 + s3));
        if (first) { lo = hi = v; first = false; }
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    smin[threadIdx.x] = lo; smax[threadIdx.x] = hi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            smin[threadIdx.x] = smin[threadIdx.x + w] < smin[threadIdx.x] ? smin[threadIdx.x + w] : smin[threadIdx.x];
            smax[threadIdx.x] = smax[threadIdx.x + w] > smax[threadIdx.x] ? smax[threadIdx.x + w] : smax[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) range[f] = smax[0] - smin[0];
}

// regrid transfer: new leaf p from old leaf src[p] with rel[p] = 0 copy,
// 1 limited linear interpolation from the parent's complete tile, 2 mean of
// the 2x2x2 children of the family starting at src[p]
template <typename T, int M>
__global__ void k3_transfer(int n, const int *lv, const int *x, const int *y, const int *z, const int *src,
                            const int *rel, const int *otslot, const int *ox, const int *oy, const int *oz,
                            const T *qold, const T *gold, T *q)
{
    constexpr int MM = M * M * M, H = M / 2;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)n * MM) return;
    const int p = (int)(g / MM), c = (int)(g % MM);
    const int i = c % M, j = (c / M) % M, k = c / (M * M);
    const int r = src[p];
    T v;
    if (rel[p] == 0) {
        v = qold[(size_t)r * MM + c];
    } else if (rel[p] == 1) {
        const long long gi = (long long)x[p] * M + i, gj = (long long)y[p] * M + j, gk = (long long)z[p] * M + k;
        const int ci = (int)((gi >> 1) - (long long)ox[r] * M), cj = (int)((gj >> 1) - (long long)oy[r] * M),
                  ck = (int)((gk >> 1) - (long long)oz[r] * M);
        const T *A = gold + (size_t)otslot[r] * P3<M>();
        const T qc = A[tix3<M>(ci, cj, ck)];
        const T sx = mm3(A[tix3<M>(ci + 1, cj, ck)] - qc, qc - A[tix3<M>(ci - 1, cj, ck)]);
        const T sy = mm3(A[tix3<M>(ci, cj + 1, ck)] - qc, qc - A[tix3<M>(ci, cj - 1, ck)]);
        const T sz = mm3(A[tix3<M>(ci, cj, ck + 1)] - qc, qc - A[tix3<M>(ci, cj, ck - 1)]);
        const T ofx = (gi & 1) ? T(0.25) : T(-0.25), ofy = (gj & 1) ? T(0.25) : T(-0.25), ofz = (gk & 1) ? T(0.25) : T(-0.25);
        v = ((qc + ofx * sx) + ofy * sy) + ofz * sz;
    } else {
        const int ch = (i >= H) + 2 * (j >= H) + 4 * (k >= H);
        const T *Q = qold + (size_t)(r + ch) * MM;
        const int fi = 2 * (i % H), fj = 2 * (j % H), fk = 2 * (k % H);
        auto at = [&](int a, int b, int d) { return Q[(fi + a) + M * ((fj + b) + M * (fk + d))]; };
        const T s0 = at(0, 0, 0) + at(1, 0, 0), s1 = at(0, 1, 0) + at(1, 1, 0);
        const T s2 = at(0, 0, 1) + at(1, 0, 1), s3 = at(0, 1, 1) + at(1, 1, 1);
        v = T(0.125) * ((s0 + s1) + (s2 + s3));
    }
    q[g] = v;
}

// ---------------------------------------------------------------------------
// device copy of a forest and its tables
struct DevForest {
    fc::DBuf<int> lv, x, y, z, nb, tslot, fslot, fill, reflux, lvl, rfl;
    int n = 0;
    Tables T;
};

}  // namespace fc3

struct fc3_ctx {
    fc3_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    fc3::Forest3 F;
    fc3::DevForest D;
    fc::DBuf<char> q[2], gr, flux, scratch;
    fc::DBuf<double> dsum;
    fc::DBuf<int> err;        // device error flag of the kernels
    int cur = 0;
    double t = 0.0, cell_updates = 0.0;
    size_t tsize = 8;
    // step graphs (one per state buffer), valid for plan_dt
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    double plan_dt = -1.0;
};

namespace fc3 {

static int check_err(fc3_ctx *c);
static bool fp32(const fc3_ctx *c) { return c->p.precision == FC_FP32; }

static void drop_graphs(fc3_ctx *c)
{
    for (int b = 0; b < 2; ++b) {
        if (c->gexec[b]) cudaGraphExecDestroy(c->gexec[b]);
        if (c->graph[b]) cudaGraphDestroy(c->graph[b]);
        c->gexec[b] = nullptr;
        c->graph[b] = nullptr;
    }
    c->plan_dt = -1.0;
}

template <typename V>
static int upload(fc::DBuf<V> &d, const std::vector<V> &h, cudaStream_t s)
{
    FC_TRY(d.alloc(h.size(), s));
    if (!h.empty()) FC_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
    return FC_OK;
}

// tables of c->F into c->D; fields reallocated (contents kept only by the caller)
static int install_forest(fc3_ctx *c)
{
    Tables T;
    FC_TRY(build_tables(c->F, T));
    const int n = c->F.n();
    std::vector<int> lv(n), x(n), y(n), z(n);
    for (int i = 0; i < n; ++i) { lv[i] = c->F.L[i].l; x[i] = c->F.L[i].x; y[i] = c->F.L[i].y; z[i] = c->F.L[i].z; }
    cudaStream_t s = c->stream;
    FC_TRY(upload(c->D.lv, lv, s)); FC_TRY(upload(c->D.x, x, s)); FC_TRY(upload(c->D.y, y, s)); FC_TRY(upload(c->D.z, z, s));
    FC_TRY(upload(c->D.nb, T.nb, s)); FC_TRY(upload(c->D.tslot, T.tslot, s)); FC_TRY(upload(c->D.fslot, T.fslot, s));
    FC_TRY(upload(c->D.fill, T.fill, s)); FC_TRY(upload(c->D.reflux, T.reflux, s));
    FC_TRY(upload(c->D.lvl, T.lvl, s)); FC_TRY(upload(c->D.rfl, T.rfl, s));
    const int m = c->p.m;
    const size_t mm = (size_t)m * m * m, p3 = (size_t)(m + 4) * (m + 4) * (m + 4);
    for (int b = 0; b < 2; ++b) FC_TRY(c->q[b].alloc((size_t)n * mm * c->tsize, s));
    FC_TRY(c->gr.alloc((size_t)std::max(T.ntile, 1) * p3 * c->tsize, s));
    FC_TRY(c->flux.alloc((size_t)std::max(T.nrec, 1) * 6 * m * m * c->tsize, s));
    c->D.n = n;
    c->D.T = std::move(T);
    drop_graphs(c);
    return FC_OK;
}

template <typename T>
static Env3<T> make_env(const fc3_ctx *c, int in, double dt)
{
    Env3<T> e{};
    e.n = c->D.n;
    e.level = c->D.lv.p; e.x = c->D.x.p; e.y = c->D.y.p; e.z = c->D.z.p;
    e.nb = c->D.nb.p; e.tslot = c->D.tslot.p; e.fslot = c->D.fslot.p;
    e.q = reinterpret_cast<const T *>(c->q[in].p);
    e.qold = e.q;
    e.qo = reinterpret_cast<T *>(c->q[1 - in].p);
    e.gr = reinterpret_cast<T *>(c->gr.p);
    e.flux = reinterpret_cast<T *>(c->flux.p);
    e.vel[0] = (T)c->p.u; e.vel[1] = (T)c->p.v; e.vel[2] = (T)c->p.w;
    for (int l = 0; l <= kMaxLevel; ++l) {
        const double idx = (double)c->p.m * (double)(1 << l);
        e.k[l] = (T)(dt * idx);
        e.dtl[l] = (T)dt;
        e.idx[l] = (T)idx;
        e.alpha[l] = T(1);
    }
    e.list = nullptr;
    e.count = c->D.n;
    e.ksub = 0;
    e.limiter = c->p.limiter;
    e.transverse = c->p.transverse;
    e.err = c->err.p;
    return e;
}

template <typename T, int M>
static int fill_levels(const fc3_ctx *c, const Env3<T> &e, const DevForest &D, cudaStream_t s)
{
    const size_t smem = (size_t)P3<M>() * sizeof(T);
    for (int l = 0; l <= kMaxLevel; ++l) {
        const int a = D.T.fill_off[l], b = D.T.fill_off[l + 1];
        if (b > a) k3_fill_tiles<T, M><<<b - a, 256, smem, s>>>(e, D.fill.p + a, b - a);
    }
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T, int M>
static int launch_step(fc3_ctx *c, int in, double dt)
{
    const Env3<T> e = make_env<T>(c, in, dt);
    cudaStream_t s = c->stream;
    FC_TRY((fill_levels<T, M>(c, e, c->D, s)));
    using L = Upd3Layout<T, M>;
    k3_update<T, M><<<e.n, M >= 8 ? 256 : 128, L::bytes, s>>>(e);
    const int nr = (int)c->D.T.reflux.size();
    if (c->p.refluxing && nr > 0) {
        constexpr int NB = M * M * M - (M - 2) * (M - 2) * (M - 2);
        const long long th = (long long)nr * NB;
        k3_reflux<T, M><<<(int)((th + 127) / 128), 128, 0, s>>>(e, c->D.reflux.p, nr);
    }
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

// shared-memory limits of the update kernels, set once outside any capture
template <typename T, int M>
static int configure_t()
{
    static bool done = false;
    if (!done) {
        FC_CUDA(cudaFuncSetAttribute(k3_update<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Upd3Layout<T, M>::bytes));
        done = true;
    }
    return FC_OK;
}
static int configure(const fc3_ctx *c)
{
    if (c->p.precision == FC_FP32) return c->p.m == 4 ? configure_t<float, 4>() : configure_t<float, 8>();
    return c->p.m == 4 ? configure_t<double, 4>() : configure_t<double, 8>();
}

// one sub-cycled coarse step (Sec. 4), the state updated in place in
// q[in] with q[1 - in] holding each level's older state: level lev takes
// its substep (older state := newer, coarser tiles at the substep's time,
// update), then for a level with finer leaves the two substeps of the next
// level and the correction of lev's coarse cells
template <typename T, int M>
struct SubPlan {
    fc3_ctx *c;
    Env3<T> base;
    int lo, hi, in;
    long long told[kMaxLevel + 1], tnew[kMaxLevel + 1];
    double dtc;
    int advance(int lev, int ksub)
    {
        const Tables &Tb = c->D.T;
        const double dt = dtc / (double)(1LL << (lev - lo));
        const long long T0 = tnew[lev], ticks = 1LL << (hi - lev);
        Env3<T> e = base;
        for (int l = 0; l <= kMaxLevel; ++l) {
            const long long a = told[l], b = tnew[l];
            e.alpha[l] = (b == a) ? T(1) : (T)((double)(T0 - a) / (double)(b - a));
            const double idx = (double)M * (double)(1 << l);
            const double dl = dtc / (double)(1LL << (l > lo ? l - lo : 0));
            e.dtl[l] = (T)dl;
            e.k[l] = (T)(dl * idx);
        }
        e.alpha[lev] = T(0);                // the level's own state is read from its copy
        cudaStream_t s = c->stream;
        const int a0 = Tb.lvl_off[lev], n0 = Tb.lvl_off[lev + 1] - a0;
        if (n0 > 0) {
            const long long th = (long long)n0 * M * M * M;
            k3_copy_old<T, M><<<(int)((th + 255) / 256), 256, 0, s>>>(e, c->D.lvl.p + a0, n0);
        }
        const size_t smem = (size_t)P3<M>() * sizeof(T);
        for (int l = lo; l < lev; ++l) {
            const int a = Tb.fill_off[l], b = Tb.fill_off[l + 1];
            if (b > a) k3_fill_tiles<T, M><<<b - a, 256, smem, s>>>(e, c->D.fill.p + a, b - a);
        }
        if (n0 > 0) {
            e.list = c->D.lvl.p + a0;
            e.count = n0;
            e.ksub = ksub;
            k3_update<T, M><<<n0, M >= 8 ? 256 : 128, Upd3Layout<T, M>::bytes, s>>>(e);
        }
        FC_CUDA(cudaGetLastError());
        told[lev] = T0;
        tnew[lev] = T0 + ticks;
        if (lev < hi) {
            FC_TRY(advance(lev + 1, 0));
            FC_TRY(advance(lev + 1, 1));
            const int r0 = Tb.rfl_off[lev], nr = Tb.rfl_off[lev + 1] - r0;
            if (c->p.refluxing && nr > 0) {
                constexpr int NB = M * M * M - (M - 2) * (M - 2) * (M - 2);
                const long long th = (long long)nr * NB;
                k3_reflux<T, M><<<(int)((th + 127) / 128), 128, 0, s>>>(base, c->D.rfl.p + r0, nr);
            }
            FC_CUDA(cudaGetLastError());
        }
        return FC_OK;
    }
};

template <typename T, int M>
static int launch_subcycled(fc3_ctx *c, int in, double dt)
{
    SubPlan<T, M> P;
    P.c = c;
    P.in = in;
    P.base = make_env<T>(c, in, dt);
    P.base.qold = reinterpret_cast<const T *>(c->q[1 - in].p);
    P.base.qo = reinterpret_cast<T *>(c->q[in].p);
    P.lo = kMaxLevel; P.hi = 0;
    for (const Leaf3 &f : c->F.L) { P.lo = std::min(P.lo, f.l); P.hi = std::max(P.hi, f.l); }
    for (int l = 0; l <= kMaxLevel; ++l) P.told[l] = P.tnew[l] = 0;
    P.dtc = dt;
    return P.advance(P.lo, 0);
}

static int step_launch(fc3_ctx *c, int in, double dt)
{
    if (c->p.subcycle) {
        if (fp32(c)) return c->p.m == 4 ? launch_subcycled<float, 4>(c, in, dt) : launch_subcycled<float, 8>(c, in, dt);
        return c->p.m == 4 ? launch_subcycled<double, 4>(c, in, dt) : launch_subcycled<double, 8>(c, in, dt);
    }
    if (fp32(c)) return c->p.m == 4 ? launch_step<float, 4>(c, in, dt) : launch_step<float, 8>(c, in, dt);
    return c->p.m == 4 ? launch_step<double, 4>(c, in, dt) : launch_step<double, 8>(c, in, dt);
}

// one step as a graph per state buffer, captured once per forest and dt
static int ensure_graphs(fc3_ctx *c, double dt)
{
    if (c->plan_dt == dt && (c->p.subcycle ? c->gexec[c->cur] != nullptr : (c->gexec[0] && c->gexec[1]))) return FC_OK;
    drop_graphs(c);
    FC_TRY(configure(c));
    for (int b = 0; b < 2; ++b) {
        if (c->p.subcycle && b != c->cur) continue;     // in place: one graph, for the current buffer
        FC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = step_launch(c, b, dt);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e2 != cudaSuccess) return cuda_status(e2, "cudaStreamEndCapture");
        c->graph[b] = g;
        FC_CUDA(cudaGraphInstantiate(&c->gexec[b], g, 0));
    }
    c->plan_dt = dt;
    return FC_OK;
}

static int finest(const fc3_ctx *c)
{
    int l = 0;
    for (const Leaf3 &f : c->F.L) l = std::max(l, f.l);
    return l;
}
static double smax(const fc3_ctx *c) { return std::max(std::fabs(c->p.u), std::max(std::fabs(c->p.v), std::fabs(c->p.w))); }
static int coarsest(const fc3_ctx *c)
{
    int l = kMaxLevel;
    for (const Leaf3 &f : c->F.L) l = std::min(l, f.l);
    return l;
}
// level whose cells set the Courant number: the finest under one global dt,
// the coarsest under sub-cycling (every level then at the same number)
static int cfl_level(const fc3_ctx *c) { return c->p.subcycle ? coarsest(c) : finest(c); }
static double next_dt(const fc3_ctx *c)
{
    const double s = smax(c);
    return s > 0.0 ? c->p.cfl * (1.0 / ((double)c->p.m * (double)(1 << cfl_level(c)))) / s : 0.0;
}

template <typename T>
static int patch_stats(fc3_ctx *c, std::vector<double> *sums, std::vector<double> *ranges)
{
    const int n = c->D.n, m = c->p.m;
    FC_TRY(c->dsum.alloc((size_t)n, c->stream));
    FC_TRY(c->scratch.alloc((size_t)n * sizeof(T), c->stream));
    const T *q = reinterpret_cast<const T *>(c->q[c->cur].p);
    T *rg = reinterpret_cast<T *>(c->scratch.p);
    if (m == 4) k3_patch_stats<T, 4><<<n, 64, 0, c->stream>>>(n, c->D.lv.p, q, c->dsum.p, rg);
    else k3_patch_stats<T, 8><<<n, 256, 0, c->stream>>>(n, c->D.lv.p, q, c->dsum.p, rg);
    FC_CUDA(cudaGetLastError());
    if (sums) {
        sums->resize(n);
        FC_CUDA(cudaMemcpyAsync(sums->data(), c->dsum.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    std::vector<T> r(n);
    FC_CUDA(cudaMemcpyAsync(r.data(), rg, n * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    if (ranges) ranges->assign(r.begin(), r.end());
    return FC_OK;
}

template <typename T>
static int family_ranges(fc3_ctx *c, const std::vector<int> &fam, std::vector<double> &out)
{
    out.clear();
    if (fam.empty()) return FC_OK;
    fc::DBuf<int> dl;
    FC_TRY(upload(dl, fam, c->stream));
    fc::DBuf<T> dr;
    FC_TRY(dr.alloc(fam.size(), c->stream));
    const T *q = reinterpret_cast<const T *>(c->q[c->cur].p);
    if (c->p.m == 4) k3_family_range<T, 4><<<(int)fam.size(), 64, 0, c->stream>>>(dl.p, (int)fam.size(), q, dr.p);
    else k3_family_range<T, 8><<<(int)fam.size(), 256, 0, c->stream>>>(dl.p, (int)fam.size(), q, dr.p);
    FC_CUDA(cudaGetLastError());
    std::vector<T> h(fam.size());
    FC_CUDA(cudaMemcpyAsync(h.data(), dr.p, fam.size() * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    out.assign(h.begin(), h.end());
    return FC_OK;
}

static int tag(fc3_ctx *c, std::vector<int8_t> &flags)
{
    const int n = c->D.n;
    std::vector<double> rng;
    FC_TRY(fp32(c) ? patch_stats<float>(c, nullptr, &rng) : patch_stats<double>(c, nullptr, &rng));
    const double thr = c->p.tag_threshold;
    flags.assign(n, 0);
    for (int i = 0; i < n; ++i) flags[i] = (rng[i] > thr && c->F.L[i].l < c->p.max_level) ? 1 : 0;
    std::vector<int> fam;
    for (int i = 0; i + 8 <= n; ++i) {
        if (!c->F.is_family(i) || c->F.L[i].l <= c->p.min_level) continue;
        bool any = false;
        for (int k = 0; k < 8; ++k) any |= flags[i + k] != 0 || rng[i + k] > thr;
        if (!any) fam.push_back(i);
        i += 7;
    }
    std::vector<double> fr;
    FC_TRY(fp32(c) ? family_ranges<float>(c, fam, fr) : family_ranges<double>(c, fam, fr));
    for (size_t f = 0; f < fam.size(); ++f)
        if (!(fr[f] > thr))
            for (int k = 0; k < 8; ++k) flags[fam[f] + k] = -1;
    return FC_OK;
}

template <typename T, int M>
static int transfer(fc3_ctx *c, const Forest3 &old, DevForest &OD, fc::DBuf<char> &qold, fc::DBuf<char> &gold,
                    const std::vector<int> &parents)
{
    // complete tiles of the old forest: its usual set plus the parents of
    // refined leaves, level by level
    std::vector<int> tslot = OD.T.tslot, fill;
    std::vector<int> off(kMaxLevel + 2, 0);
    int ntile = OD.T.ntile;
    std::vector<char> want(old.n(), 0);
    for (int r : parents) if (tslot[r] < 0) { want[r] = 1; tslot[r] = ntile++; }
    for (int l = 0; l <= kMaxLevel; ++l) {
        off[l] = (int)fill.size();
        for (int i = 0; i < old.n(); ++i)
            if (old.L[i].l == l && (want[i] || OD.T.tslot[i] >= 0)) fill.push_back(i);
    }
    off[kMaxLevel + 1] = (int)fill.size();
    const size_t p3 = (size_t)P3<M>();
    FC_TRY(gold.alloc((size_t)std::max(ntile, 1) * p3 * sizeof(T), c->stream));
    fc::DBuf<int> dts, dfill;
    FC_TRY(upload(dts, tslot, c->stream));
    FC_TRY(upload(dfill, fill, c->stream));
    Env3<T> e{};
    e.n = OD.n;
    e.level = OD.lv.p; e.x = OD.x.p; e.y = OD.y.p; e.z = OD.z.p; e.nb = OD.nb.p; e.tslot = dts.p; e.fslot = OD.fslot.p;
    e.q = reinterpret_cast<const T *>(qold.p);
    e.qold = e.q;
    for (int l = 0; l <= kMaxLevel; ++l) e.alpha[l] = T(1);
    e.gr = reinterpret_cast<T *>(gold.p);
    e.err = c->err.p;
    const size_t smem = p3 * sizeof(T);
    for (int l = 0; l <= kMaxLevel; ++l)
        if (off[l + 1] > off[l])
            k3_fill_tiles<T, M><<<off[l + 1] - off[l], 256, smem, c->stream>>>(e, dfill.p + off[l], off[l + 1] - off[l]);
    FC_CUDA(cudaGetLastError());
    // relation of each new leaf to the old forest
    const Forest3 &F = c->F;
    const int n = F.n();
    std::vector<int> src(n), rel(n);
    for (int p = 0; p < n; ++p) {
        const Leaf3 &f = F.L[p];
        const int r = old.locate(f.l, f.x, f.y, f.z);
        if (r < 0) { set_error("regrid transfer without a source"); return FC_ERR_INVALID_ARG; }
        src[p] = r;
        if (old.L[r].l == f.l) rel[p] = 0;
        else if (old.L[r].l == f.l - 1) rel[p] = 1;
        else if (old.L[r].l == f.l + 1) rel[p] = 2;
        else { set_error("a new leaf more than one level from its old leaves"); return FC_ERR_INVALID_ARG; }
    }
    fc::DBuf<int> dsrc, drel;
    FC_TRY(upload(dsrc, src, c->stream));
    FC_TRY(upload(drel, rel, c->stream));
    const long long th = (long long)n * M * M * M;
    k3_transfer<T, M><<<(int)((th + 255) / 256), 256, 0, c->stream>>>(
        n, c->D.lv.p, c->D.x.p, c->D.y.p, c->D.z.p, dsrc.p, drel.p, dts.p, OD.x.p, OD.y.p, OD.z.p,
        reinterpret_cast<const T *>(qold.p), reinterpret_cast<const T *>(gold.p), reinterpret_cast<T *>(c->q[c->cur].p));
    FC_CUDA(cudaGetLastError());
    return check_err(c);
}

// the forest after a regrid by flags: refinement wins, a family coarsens
// when all eight are flagged -1, then 2:1 balance (host only)
static int regrid_forest(const Forest3 &old, const int8_t *flags, int min_level, int max_level, Forest3 &F)
{
    const int n = old.n();
    std::vector<Leaf3> out;
    out.reserve((size_t)n * 2);
    for (int i = 0; i < n; ++i) {
        if (old.is_family(i) && old.L[i].l > min_level) {
            bool all = true;
            for (int k = 0; k < 8; ++k) all &= flags[i + k] == -1;
            if (all) {
                Leaf3 f{0, old.L[i].l - 1, old.L[i].x >> 1, old.L[i].y >> 1, old.L[i].z >> 1};
                f.key = key3(f.l, f.x, f.y, f.z);
                out.push_back(f);
                i += 7;
                continue;
            }
        }
        if (flags[i] == 1 && old.L[i].l < max_level) {
            for (int k = 0; k < 8; ++k) {
                Leaf3 f{0, old.L[i].l + 1, 2 * old.L[i].x + (k & 1), 2 * old.L[i].y + ((k >> 1) & 1), 2 * old.L[i].z + (k >> 2)};
                f.key = key3(f.l, f.x, f.y, f.z);
                out.push_back(f);
            }
        } else {
            out.push_back(old.L[i]);
        }
    }
    F.L.swap(out);
    F.index();
    return F.balance(max_level);
}

static int regrid(fc3_ctx *c, const int8_t *flags)
{
    const Forest3 old = c->F;
    std::vector<int> parents;
    FC_TRY(regrid_forest(old, flags, c->p.min_level, c->p.max_level, c->F));
    for (const Leaf3 &f : c->F.L) {
        const int r = old.locate(f.l, f.x, f.y, f.z);
        if (r >= 0 && old.L[r].l == f.l - 1) parents.push_back(r);
    }
    std::sort(parents.begin(), parents.end());
    parents.erase(std::unique(parents.begin(), parents.end()), parents.end());
    // keep the old device forest and state while the new one is installed
    DevForest OD;
    OD.lv.swap(c->D.lv); OD.x.swap(c->D.x); OD.y.swap(c->D.y); OD.z.swap(c->D.z);
    OD.nb.swap(c->D.nb); OD.tslot.swap(c->D.tslot); OD.fslot.swap(c->D.fslot);
    OD.fill.swap(c->D.fill); OD.reflux.swap(c->D.reflux); OD.lvl.swap(c->D.lvl); OD.rfl.swap(c->D.rfl);
    OD.n = c->D.n;
    OD.T = c->D.T;
    fc::DBuf<char> qold, gold;
    qold.swap(c->q[c->cur]);
    FC_TRY(install_forest(c));
    const int m = c->p.m;
    if (fp32(c)) return m == 4 ? transfer<float, 4>(c, old, OD, qold, gold, parents) : transfer<float, 8>(c, old, OD, qold, gold, parents);
    return m == 4 ? transfer<double, 4>(c, old, OD, qold, gold, parents) : transfer<double, 8>(c, old, OD, qold, gold, parents);
}

// the kernels' error flag (read after the stream drains, then cleared)
static int check_err(fc3_ctx *c)
{
    int h = 0;
    FC_CUDA(cudaMemcpyAsync(&h, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    if (h) {
        FC_CUDA(cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream));
        set_error("inconsistent neighbour data (a table entry pointed nowhere)");
        return FC_ERR_INVALID_ARG;
    }
    return FC_OK;
}

static int set_initial(fc3_ctx *c, int kind, const double *prm, int np)
{
    static const int need[3] = {8, 5, 6};
    if (kind < 0 || kind > 2 || !prm || np < need[kind]) { set_error("bad initial condition"); return FC_ERR_INVALID_ARG; }
    fc::DBuf<double> a;
    FC_TRY(a.alloc(8, c->stream));
    FC_CUDA(cudaMemcpyAsync(a.p, prm, need[kind] * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const int n = c->D.n, m = c->p.m;
    const long long th = (long long)n * m * m * m;
    const int blocks = (int)((th + 255) / 256);
    void *q = c->q[c->cur].p;
    if (fp32(c)) {
        if (m == 4) k3_init<float, 4><<<blocks, 256, 0, c->stream>>>(n, c->D.lv.p, c->D.x.p, c->D.y.p, c->D.z.p, kind, a.p, (float *)q);
        else k3_init<float, 8><<<blocks, 256, 0, c->stream>>>(n, c->D.lv.p, c->D.x.p, c->D.y.p, c->D.z.p, kind, a.p, (float *)q);
    } else {
        if (m == 4) k3_init<double, 4><<<blocks, 256, 0, c->stream>>>(n, c->D.lv.p, c->D.x.p, c->D.y.p, c->D.z.p, kind, a.p, (double *)q);
        else k3_init<double, 8><<<blocks, 256, 0, c->stream>>>(n, c->D.lv.p, c->D.x.p, c->D.y.p, c->D.z.p, kind, a.p, (double *)q);
    }
    FC_CUDA(cudaGetLastError());
    FC_CUDA(cudaStreamSynchronize(c->stream));
    c->t = 0.0;
    return FC_OK;
}

static int zero_fields(fc3_ctx *c)
{
    FC_CUDA(cudaMemsetAsync(c->q[c->cur].p, 0, (size_t)c->D.n * c->p.m * c->p.m * c->p.m * c->tsize, c->stream));
    return FC_OK;
}

}  // namespace fc3

using namespace fc3;

extern "C" {

int fc3_create(const fc3_params *p, fc3_ctx **out)
{
    if (!p || !out) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    *out = nullptr;
    if ((p->m != 4 && p->m != 8) || p->min_level < 0 || p->max_level < p->min_level || p->max_level > kMaxLevel ||
        (p->precision != FC_FP32 && p->precision != FC_FP64) || p->limiter < 0 || p->limiter > 1 ||
        p->transverse < 0 || p->transverse > 2 || p->refluxing < 0 || p->refluxing > 1 || p->subcycle < 0 ||
        p->subcycle > 1 || !(p->cfl > 0.0) ||
        p->cfl > 1.0 || !std::isfinite(p->u) || !std::isfinite(p->v) || !std::isfinite(p->w)) {
        set_error("invalid parameters");
        return FC_ERR_INVALID_ARG;
    }
    fc3_ctx *c = new fc3_ctx;
    c->p = *p;
    c->tsize = p->precision == FC_FP32 ? 4 : 8;
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
    int rc = c->err.alloc(1, c->stream);
    if (!rc && cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream) != cudaSuccess) rc = FC_ERR_CUDA;
    if (!rc) rc = fc3_forest_uniform(c, p->min_level);
    if (rc) { fc3_destroy(c); return rc; }
    *out = c;
    return FC_OK;
}

void fc3_destroy(fc3_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    cudaStream_t s = c->stream;
    const bool own = c->own_stream;
    delete c;                               // buffers released on the stream
    if (own) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
}

int fc3_forest_uniform(fc3_ctx *c, int level)
{
    if (!c || level < 0 || level > c->p.max_level) { set_error("level out of range"); return FC_ERR_INVALID_ARG; }
    const int w = 1 << level;
    c->F.L.clear();
    for (int z = 0; z < w; ++z)
        for (int y = 0; y < w; ++y)
            for (int x = 0; x < w; ++x) c->F.L.push_back(Leaf3{key3(level, x, y, z), level, x, y, z});
    c->F.sort();
    FC_TRY(install_forest(c));
    c->t = 0.0;
    return zero_fields(c);
}

int fc3_forest_set_leaves(fc3_ctx *c, int64_t n, const int8_t *level, const int32_t *x, const int32_t *y,
                          const int32_t *z)
{
    if (!c || n <= 0 || !level || !x || !y || !z) { set_error("invalid leaves"); return FC_ERR_INVALID_ARG; }
    Forest3 F;
    F.L.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        const int l = level[i];
        if (l < 0 || l > c->p.max_level || x[i] < 0 || y[i] < 0 || z[i] < 0 || x[i] >= (1 << l) || y[i] >= (1 << l) ||
            z[i] >= (1 << l)) {
            set_error("leaf %lld out of range", (long long)i);
            return FC_ERR_INVALID_ARG;
        }
        F.L[i] = Leaf3{key3(l, x[i], y[i], z[i]), l, x[i], y[i], z[i]};
        if (i > 0 && F.L[i].key <= F.L[i - 1].key) { set_error("leaves not in Morton order"); return FC_ERR_INVALID_ARG; }
    }
    F.index();
    if (!F.covers()) { set_error("leaves do not tile the cube"); return FC_ERR_INVALID_ARG; }
    if (!F.balanced()) { set_error("forest is not 2:1 balanced"); return FC_ERR_UNBALANCED; }
    c->F = std::move(F);
    FC_TRY(install_forest(c));
    return zero_fields(c);
}

int fc3_forest_num_leaves(const fc3_ctx *c, int64_t *n)
{
    if (!c || !n) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    *n = c->F.n();
    return FC_OK;
}

int fc3_forest_get_leaves(const fc3_ctx *c, int8_t *level, int32_t *x, int32_t *y, int32_t *z, int64_t cap)
{
    if (!c || !level || !x || !y || !z) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    if (cap < c->F.n()) { set_error("capacity %lld below %d leaves", (long long)cap, c->F.n()); return FC_ERR_CAPACITY; }
    for (int i = 0; i < c->F.n(); ++i) {
        level[i] = (int8_t)c->F.L[i].l; x[i] = c->F.L[i].x; y[i] = c->F.L[i].y; z[i] = c->F.L[i].z;
    }
    return FC_OK;
}

int fc3_write_fields(fc3_ctx *c, const void *src, int64_t count)
{
    if (!c || !src) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    const int64_t need = (int64_t)c->D.n * c->p.m * c->p.m * c->p.m;
    if (count < need) { set_error("buffer holds %lld values, %lld needed", (long long)count, (long long)need); return FC_ERR_CAPACITY; }
    FC_CUDA(cudaMemcpyAsync(c->q[c->cur].p, src, need * c->tsize, cudaMemcpyHostToDevice, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

int fc3_read_fields(fc3_ctx *c, void *dst, int64_t count)
{
    if (!c || !dst) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    const int64_t need = (int64_t)c->D.n * c->p.m * c->p.m * c->p.m;
    if (count < need) { set_error("buffer holds %lld values, %lld needed", (long long)count, (long long)need); return FC_ERR_CAPACITY; }
    FC_CUDA(cudaMemcpyAsync(dst, c->q[c->cur].p, need * c->tsize, cudaMemcpyDeviceToHost, c->stream));
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

int fc3_set_initial(fc3_ctx *c, int kind, const double *prm, int np)
{
    if (!c) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    return set_initial(c, kind, prm, np);
}

int fc3_init_refine(fc3_ctx *c, int kind, const double *prm, int np)
{
    fc::Range nvtx_range("fc3_init_refine");
    if (!c) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    FC_TRY(fc3_forest_uniform(c, c->p.min_level));
    for (int r = 0; r < c->p.max_level - c->p.min_level; ++r) {
        FC_TRY(set_initial(c, kind, prm, np));
        std::vector<int8_t> flags;
        FC_TRY(tag(c, flags));
        std::vector<char> mark(c->F.n(), 0);
        bool any = false;
        for (int i = 0; i < c->F.n(); ++i) if (flags[i] == 1) { mark[i] = 1; any = true; }
        if (any) c->F.refine(mark);
        FC_TRY(c->F.balance(c->p.max_level));
        FC_TRY(install_forest(c));
    }
    return set_initial(c, kind, prm, np);
}

int fc3_tag(fc3_ctx *c, int8_t *flags)
{
    fc::Range nvtx_range("fc3_tag");
    if (!c || !flags) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    std::vector<int8_t> f;
    FC_TRY(tag(c, f));
    std::memcpy(flags, f.data(), f.size());
    return FC_OK;
}

int fc3_regrid(fc3_ctx *c, const int8_t *flags)
{
    fc::Range nvtx_range("fc3_regrid");
    if (!c || !flags) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    for (int i = 0; i < c->F.n(); ++i)
        if (flags[i] < -1 || flags[i] > 1) { set_error("flag %d of leaf %d not in -1..1", flags[i], i); return FC_ERR_INVALID_ARG; }
    return regrid(c, flags);
}

int fc3_advance(fc3_ctx *c, int nsteps, double dt, double *t_out, double *dt_out)
{
    fc::Range nvtx_range("fc3_advance");
    if (!c || nsteps < 0) { set_error("invalid arguments"); return FC_ERR_INVALID_ARG; }
    if (dt <= 0.0) dt = next_dt(c);
    if (!(dt > 0.0) || !std::isfinite(dt)) { set_error("no time step (zero velocity)"); return FC_ERR_INVALID_ARG; }
    const double dxf = 1.0 / ((double)c->p.m * (double)(1 << cfl_level(c)));
    if (dt * smax(c) / dxf > 1.0) { set_error("Courant number %g above 1", dt * smax(c) / dxf); return FC_ERR_CFL_VIOLATION; }
    if (nsteps > 0) {
        FC_TRY(ensure_graphs(c, dt));
        for (int s = 0; s < nsteps; ++s) {
            FC_CUDA(cudaGraphLaunch(c->gexec[c->cur], c->stream));
            if (!c->p.subcycle) c->cur = 1 - c->cur;
            c->t += dt;
        }
        double per = 0.0;
        const int lo = coarsest(c);
        for (const Leaf3 &f : c->F.L) per += c->p.subcycle ? (double)(1LL << (f.l - lo)) : 1.0;
        c->cell_updates += (double)nsteps * per * c->p.m * c->p.m * c->p.m;
        FC_TRY(check_err(c));
    }
    if (t_out) *t_out = c->t;
    if (dt_out) *dt_out = dt;
    return FC_OK;
}

int fc3_conservation_sum(fc3_ctx *c, double *sum)
{
    if (!c || !sum) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    std::vector<double> s;
    FC_TRY(fp32(c) ? patch_stats<float>(c, &s, nullptr) : patch_stats<double>(c, &s, nullptr));
    double acc = 0.0, comp = 0.0;          // Neumaier's compensated sum over the patch partials
    for (double v : s) {
        const double t = acc + v;
        comp += std::fabs(acc) >= std::fabs(v) ? (acc - t) + v : (v - t) + acc;
        acc = t;
    }
    *sum = acc + comp;
    return FC_OK;
}

int fc3_stats(fc3_ctx *c, double *time, double *next, double *cell_updates)
{
    if (!c) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    if (time) *time = c->t;
    if (next) *next = next_dt(c);
    if (cell_updates) *cell_updates = c->cell_updates;
    return FC_OK;
}

int fc3_sync(fc3_ctx *c)
{
    if (!c) { set_error("null argument"); return FC_ERR_INVALID_ARG; }
    FC_CUDA(cudaStreamSynchronize(c->stream));
    return FC_OK;
}

}  // extern "C"
