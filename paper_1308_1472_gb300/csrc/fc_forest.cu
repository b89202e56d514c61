// fc_forest.cu -- forest of quadtrees kept in HBM; every topology change is a
// data-parallel count / scan / scatter over the leaves.
//
// Sec. 2 of the paper: a forest of quadtrees whose leaves carry the patches,
// refined and coarsened from per-leaf flags only, with 2:1 balance between
// neighbours.  Sec. 4: leaves stay in space-filling-curve order and neighbours
// are found by lookup relative to the current leaf.
//
// Splitting a leaf into its four children (in Morton order) and merging four
// siblings into their parent both preserve the Morton order of the leaf
// array, so no sort is ever needed after the first construction: new
// positions come from an exclusive scan of per-leaf output counts.
// Point location is a binary search over the sorted 64-bit keys.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <numeric>

#include "fc_forest.cuh"
#include "fc_sphere.cuh"

namespace fc {

// ---------------------------------------------------------------------------
// scan
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 2;   // per thread

__device__ int block_exclusive_scan(int v, int *sh, int *total)
{
    // Hillis-Steele over one block of kScanBlock threads (values per thread)
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        int a = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += a;
        __syncthreads();
    }
    int incl = sh[t];
    if (total) *total = sh[kScanBlock - 1];
    __syncthreads();
    return incl - v;
}

__global__ void k_scan_blocks(const int *in, int *out, int n, int *bsum)
{
    __shared__ int sh[kScanBlock];
    __shared__ int tot;
    int base = (blockIdx.x * kScanBlock + threadIdx.x) * kScanItems;
    int v[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int ex = block_exclusive_scan(s, sh, &tot);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int *bsum, int nb, int *total)
{
    __shared__ int sh[kScanBlock];
    __shared__ int tot;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanBlock) {
        int i = b0 + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) bsum[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int *out, int n, const int *bsum)
{
    int base = (blockIdx.x * kScanBlock + threadIdx.x) * kScanItems;
    int add = bsum[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) out[base + k] += add;
}

int exclusive_scan(const int *d_in, int *d_out, int n, int *h_total, DBuf<int> &blocksum, cudaStream_t s)
{
    int per = kScanBlock * kScanItems;
    int nb = (n + per - 1) / per;
    if (nb < 1) nb = 1;
    FC_TRY(blocksum.alloc(nb + 1, s));
    k_scan_blocks<<<nb, kScanBlock, 0, s>>>(d_in, d_out, n, blocksum.p);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(blocksum.p, nb, blocksum.p + nb);
    k_scan_add<<<nb, kScanBlock, 0, s>>>(d_out, n, blocksum.p);
    FC_CUDA(cudaGetLastError());
    if (h_total) {
        FC_CUDA(cudaMemcpyAsync(h_total, blocksum.p + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        FC_CUDA(cudaStreamSynchronize(s));
    }
    return FC_OK;
}

// ---------------------------------------------------------------------------
// point location
__device__ inline int map_point(int conn, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    const long long N = 1LL << kMaxBits;
    if (X >= 0 && X < N && Y >= 0 && Y < N) { *Xo = X; *Yo = Y; return t; }
    if (conn == FC_CONN_PERIODIC) { *Xo = X & (N - 1); *Yo = Y & (N - 1); return t; }
    if (conn == FC_CONN_SPHERE || conn == FC_CONN_PILLOW) return sphere_map_point(conn, t, X, Y, Xo, Yo);
    return -1;   // walls
}

// Table connectivity: crossing side s of tree t (0 -x, 1 +x, 2 -y, 3 +y)
// into the tree of its table entry {tree, side, reversed}; the depth of the
// point beyond side s becomes its depth inside the neighbour's side, the
// coordinate along the side keeps or reverses its direction.
__device__ inline int tab_cross(const int *tab, int t, int s, long long X, long long Y, long long *Xo, long long *Yo)
{
    const long long N = 1LL << kMaxBits;
    const int *e = tab + (t * 4 + s) * 3;
    const int t2 = e[0], s2 = e[1];
    if (t2 < 0) return -1;
    const long long depth = s == 0 ? -1 - X : (s == 1 ? X - N : (s == 2 ? -1 - Y : Y - N));
    const long long a0 = s < 2 ? Y : X, along = e[2] ? N - 1 - a0 : a0;
    const long long inward = (s2 & 1) ? N - 1 - depth : depth;
    if (s2 < 2) { *Xo = inward; *Yo = along; }
    else { *Xo = along; *Yo = inward; }
    return t2;
}

__device__ inline int side_out(long long v, int low)
{
    const long long N = 1LL << kMaxBits;
    return v < 0 ? low : (v >= N ? low + 1 : -1);
}

// across side s, then across the one side the point is still beyond
__device__ inline int tab_two(const int *tab, int t, int s, long long X, long long Y, long long *Xo, long long *Yo)
{
    long long X1, Y1;
    const int t1 = tab_cross(tab, t, s, X, Y, &X1, &Y1);
    if (t1 < 0) return -1;
    const int ax = side_out(X1, 0), ay = side_out(Y1, 2);
    if ((ax >= 0) == (ay >= 0)) return -1;
    const int t2 = tab_cross(tab, t1, ax >= 0 ? ax : ay, X1, Y1, Xo, Yo);
    if (t2 < 0 || side_out(*Xo, 0) >= 0 || side_out(*Yo, 2) >= 0) return -1;
    return t2;
}

// a finest-level point of tree t (possibly beyond its sides) in the tree
// that holds it; beyond a corner both orders of crossing must agree
__device__ inline int tab_map_point(const int *tab, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    const int bx = side_out(X, 0), by = side_out(Y, 2);
    if (bx < 0 && by < 0) { *Xo = X; *Yo = Y; return t; }
    if (bx < 0 || by < 0) {
        const int t1 = tab_cross(tab, t, bx >= 0 ? bx : by, X, Y, Xo, Yo);
        return (t1 < 0 || side_out(*Xo, 0) >= 0 || side_out(*Yo, 2) >= 0) ? -1 : t1;
    }
    long long Xa, Ya, Xb, Yb;
    const int ta = tab_two(tab, t, bx, X, Y, &Xa, &Ya), tb = tab_two(tab, t, by, X, Y, &Xb, &Yb);
    if (ta < 0 || ta != tb || Xa != Xb || Ya != Yb) return -1;
    *Xo = Xa; *Yo = Ya;
    return ta;
}

__device__ inline int forest_map_point(const ForestDev &f, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    if (f.conn == FC_CONN_TABLE)       // no table yet: one tree bounded on every side
        return f.ctab ? tab_map_point(f.ctab, t, X, Y, Xo, Yo) : map_point(FC_CONN_SQUARE, t, X, Y, Xo, Yo);
    return map_point(f.conn, t, X, Y, Xo, Yo);
}

// orientation code of the crossing at point (X, Y) beyond tree t's sides
// (table connectivity): the images of unit steps along +x and +y
__device__ inline int tab_orientation(const ForestDev &f, int t, long long X, long long Y)
{
    const long long N = 1LL << kMaxBits;
    if (!f.ctab || (X >= 0 && X < N && Y >= 0 && Y < N)) return 0;
    long long X0, Y0, X1, Y1, X2, Y2;
    if (tab_map_point(f.ctab, t, X, Y, &X0, &Y0) < 0) return 0;
    const long long sx = X < 0 ? -1 : (X >= N ? 1 : (X + 1 >= N ? -1 : 1));
    const long long sy = Y < 0 ? -1 : (Y >= N ? 1 : (Y + 1 >= N ? -1 : 1));
    tab_map_point(f.ctab, t, X + sx, Y, &X1, &Y1);
    tab_map_point(f.ctab, t, X, Y + sy, &X2, &Y2);
    const long long ix = (X1 - X0) * sx, iy = (Y1 - Y0) * sx;
    const long long jx = (X2 - X0) * sy, jy = (Y2 - Y0) * sy;
    const int swap = ix == 0;
    const int r0 = swap ? (jx < 0) : (ix < 0);
    const int r1 = swap ? (iy < 0) : (jy < 0);
    return 1 + 4 * swap + 2 * r0 + r1;
}

__device__ inline int locate(const ForestDev &f, int t, long long X, long long Y)
{
    uint64_t k = ((uint64_t)t << kTreeShift) | spread_bits((uint32_t)X) | (spread_bits((uint32_t)Y) << 1);
    int lo = 0, hi = f.n;           // first key > k
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (f.key[mid] <= k) lo = mid + 1; else hi = mid;
    }
    int c = lo - 1;
    if (c < 0) return -1;
    int s = kMaxBits - f.level[c];
    if (f.tree[c] != t || (X >> s) != f.x[c] || (Y >> s) != f.y[c]) return -1;
    return c;
}

// probe point q (0 or 1) just outside leaf i in direction d
__device__ inline void probe(const ForestDev &f, int i, int d, int q, long long *X, long long *Y)
{
    int s = kMaxBits - f.level[i];
    long long S = 1LL << s, X0 = (long long)f.x[i] << s, Y0 = (long long)f.y[i] << s;
    long long a = q ? 3 * (S >> 2) : (S >> 2);
    const int ox[8] = {-1, 1, 0, 0, -1, 1, -1, 1};
    const int oy[8] = {0, 0, -1, 1, -1, -1, 1, 1};
    *X = ox[d] < 0 ? X0 - 1 : (ox[d] > 0 ? X0 + S : X0 + a);
    *Y = oy[d] < 0 ? Y0 - 1 : (oy[d] > 0 ? Y0 + S : Y0 + a);
}

__device__ inline int locate_probe(const ForestDev &f, int i, int d, int q)
{
    long long X, Y, Xm, Ym;
    probe(f, i, d, q, &X, &Y);
    int t2 = forest_map_point(f, f.tree[i], X, Y, &Xm, &Ym);
    return t2 < 0 ? -1 : locate(f, t2, Xm, Ym);
}

// ---------------------------------------------------------------------------
__global__ void k_uniform(int *tree, int *level, int *x, int *y, int lev, int per_tree, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int t = i / per_tree, r = i - t * per_tree;
    tree[i] = t;
    level[i] = lev;
    x[i] = (int)compact_bits((uint64_t)r);
    y[i] = (int)compact_bits((uint64_t)r >> 1);
}

__global__ void k_keys(ForestDev f, uint64_t *key)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < f.n) key[i] = leaf_key(f.tree[i], f.level[i], f.x[i], f.y[i]);
}

// table entry for (leaf, direction); *bad set when levels differ by > 1
__global__ void k_neighbors(ForestDev f, int *nbr, int *bad)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= f.n * 8) return;
    int i = g >> 3, d = g & 7;
    int *e = nbr + (size_t)g * 4;
    int n0 = locate_probe(f, i, d, 0);
    int kind = FC_NB_NONE, id0 = -1, id1 = -1, orient = 0;
    if (n0 >= 0) {
        if (is_sphere_conn(f.conn) || f.conn == FC_CONN_TABLE) {
            long long X, Y;
            probe(f, i, d, 0, &X, &Y);
            orient = f.conn == FC_CONN_TABLE ? tab_orientation(f, f.tree[i], X, Y)
                                             : sphere_orientation(f.conn, f.tree[i], X, Y);
        }
        int dl = f.level[n0] - f.level[i];
        id0 = n0;
        if (dl == 0) kind = FC_NB_SAME;
        else if (dl == -1) kind = FC_NB_COARSER;
        else if (dl == 1) {
            kind = FC_NB_FINER;
            if (d < 4) {
                id1 = locate_probe(f, i, d, 1);
                if (id1 < 0 || f.level[id1] != f.level[i] + 1) *bad = 1;
            }
        } else *bad = 1;
    }
    e[0] = kind; e[1] = id0; e[2] = id1; e[3] = orient;
}

// mark leaves that are more than one level coarser than a probing neighbour
__global__ void k_balance_mark(ForestDev f, int *mark, int *any)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= f.n * 8) return;
    int i = g >> 3, d = g & 7;
    int n0 = locate_probe(f, i, d, 0);
    if (n0 >= 0 && f.level[n0] < f.level[i] - 1) {
        mark[n0] = 1;
        *any = 1;
    }
}

__global__ void k_counts_from_marks(const int *mark, int *cnt, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = mark[i] ? 4 : 1;
}

// write each old leaf (or its four children) at its scanned position and
// carry the origin record through the split
__global__ void k_split(ForestDev f, const int *mark, const int *off, int *t2, int *l2, int *x2, int *y2,
                        const int *org_in, int *org_out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    int o = off[i];
    if (!mark[i]) {
        t2[o] = f.tree[i]; l2[o] = f.level[i]; x2[o] = f.x[i]; y2[o] = f.y[i];
        if (org_out) for (int k = 0; k < 3; ++k) org_out[3 * o + k] = org_in[3 * i + k];
        return;
    }
    for (int c = 0; c < 4; ++c) {
        t2[o + c] = f.tree[i]; l2[o + c] = f.level[i] + 1;
        x2[o + c] = 2 * f.x[i] + (c & 1); y2[o + c] = 2 * f.y[i] + (c >> 1);
        if (org_out) {
            int kind = org_in[3 * i], src = org_in[3 * i + 1], dl = org_in[3 * i + 2];
            if (kind == 2) {               // a merged parent split again: the old children
                org_out[3 * (o + c)] = 0; org_out[3 * (o + c) + 1] = src + c; org_out[3 * (o + c) + 2] = 0;
            } else {                       // one level deeper below the same old leaf
                org_out[3 * (o + c)] = 1; org_out[3 * (o + c) + 1] = src; org_out[3 * (o + c) + 2] = dl + 1;
            }
        }
    }
}

// per-leaf output count for the flag rule; families are detected at their
// first child and the other three members emit nothing
__global__ void k_adapt_count(ForestDev f, const int8_t *flags, int min_level, int max_level, int *cnt, int *kind)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    int lv = f.level[i];
    // member c of a coarsening family starting at i - c ?
    int xi = f.x[i], yi = f.y[i];
    int c = (xi & 1) + 2 * (yi & 1);
    int first = i - c;
    bool fam = false;
    if (lv > min_level && first >= 0 && first + 3 < f.n) {
        fam = true;
        int px = xi >> 1, py = yi >> 1;
        for (int k = 0; k < 4; ++k) {
            int j = first + k;
            if (f.tree[j] != f.tree[i] || f.level[j] != lv || f.x[j] != 2 * px + (k & 1) ||
                f.y[j] != 2 * py + (k >> 1) || flags[j] != -1)
                fam = false;
        }
    }
    if (fam) { cnt[i] = c == 0 ? 1 : 0; kind[i] = 2; return; }
    if (flags[i] > 0 && lv < max_level) { cnt[i] = 4; kind[i] = 1; return; }
    cnt[i] = 1; kind[i] = 0;
}

__global__ void k_adapt_scatter(ForestDev f, const int *kind, const int *cnt, const int *off, int *t2, int *l2,
                                int *x2, int *y2, int *org)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n || cnt[i] == 0) return;
    int o = off[i];
    if (kind[i] == 2) {
        t2[o] = f.tree[i]; l2[o] = f.level[i] - 1; x2[o] = f.x[i] >> 1; y2[o] = f.y[i] >> 1;
        org[3 * o] = 2; org[3 * o + 1] = i; org[3 * o + 2] = -1;
    } else if (kind[i] == 1) {
        for (int c = 0; c < 4; ++c) {
            t2[o + c] = f.tree[i]; l2[o + c] = f.level[i] + 1;
            x2[o + c] = 2 * f.x[i] + (c & 1); y2[o + c] = 2 * f.y[i] + (c >> 1);
            org[3 * (o + c)] = 1; org[3 * (o + c) + 1] = i; org[3 * (o + c) + 2] = 1;
        }
    } else {
        t2[o] = f.tree[i]; l2[o] = f.level[i]; x2[o] = f.x[i]; y2[o] = f.y[i];
        org[3 * o] = 0; org[3 * o + 1] = i; org[3 * o + 2] = 0;
    }
}

__global__ void k_origin_identity(int *org, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { org[3 * i] = 0; org[3 * i + 1] = i; org[3 * i + 2] = 0; }
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
int Forest::uniform(int lev)
{
    if (lev < 0 || lev > 14) { set_error("uniform level %d out of range", lev); return FC_ERR_INVALID_ARG; }
    int per = 1 << (2 * lev);
    n = ntrees() * per;
    FC_TRY(tree.alloc(n, stream)); FC_TRY(level.alloc(n, stream));
    FC_TRY(x.alloc(n, stream)); FC_TRY(y.alloc(n, stream));
    k_uniform<<<nblk(n, 256), 256, 0, stream>>>(tree.p, level.p, x.p, y.p, lev, per, n);
    FC_CUDA(cudaGetLastError());
    return rebuild_tables();
}

int Forest::set_leaves(int64_t nn, const int32_t *t, const int32_t *l, const int32_t *xx, const int32_t *yy)
{
    // host-side validation and initial ordering of an imported forest
    if (nn <= 0 || nn > (1 << 26)) { set_error("bad leaf count"); return FC_ERR_INVALID_ARG; }
    std::vector<uint64_t> k(nn);
    std::vector<int> idx(nn);
    unsigned long long area = 0;
    for (int64_t i = 0; i < nn; ++i) {
        if (t[i] < 0 || t[i] >= ntrees() || l[i] < 0 || l[i] > 14 || xx[i] < 0 || yy[i] < 0 ||
            xx[i] >= (1 << l[i]) || yy[i] >= (1 << l[i])) {
            set_error("leaf %lld out of range", (long long)i);
            return FC_ERR_INVALID_ARG;
        }
        k[i] = leaf_key(t[i], l[i], xx[i], yy[i]);
        idx[i] = (int)i;
        area += 1ULL << (2 * (14 - l[i]));
    }
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return k[a] < k[b]; });
    for (int64_t i = 0; i + 1 < nn; ++i) {
        int a = idx[i], b = idx[i + 1];
        uint64_t span = 1ULL << (2 * (kMaxBits - l[a]));
        if (t[a] == t[b] && k[b] < k[a] + span) { set_error("leaves overlap"); return FC_ERR_INVALID_ARG; }
    }
    if (area != (unsigned long long)ntrees() << 28) { set_error("leaves do not cover the domain"); return FC_ERR_INVALID_ARG; }
    std::vector<int> ht(nn), hl(nn), hx(nn), hy(nn);
    for (int64_t i = 0; i < nn; ++i) { ht[i] = t[idx[i]]; hl[i] = l[idx[i]]; hx[i] = xx[idx[i]]; hy[i] = yy[idx[i]]; }
    n = (int)nn;
    FC_TRY(tree.alloc(n, stream)); FC_TRY(level.alloc(n, stream));
    FC_TRY(x.alloc(n, stream)); FC_TRY(y.alloc(n, stream));
    FC_CUDA(cudaMemcpyAsync(tree.p, ht.data(), n * sizeof(int), cudaMemcpyHostToDevice, stream));
    FC_CUDA(cudaMemcpyAsync(level.p, hl.data(), n * sizeof(int), cudaMemcpyHostToDevice, stream));
    FC_CUDA(cudaMemcpyAsync(x.p, hx.data(), n * sizeof(int), cudaMemcpyHostToDevice, stream));
    FC_CUDA(cudaMemcpyAsync(y.p, hy.data(), n * sizeof(int), cudaMemcpyHostToDevice, stream));
    FC_CUDA(cudaStreamSynchronize(stream));   // host vectors go out of scope
    return FC_OK;
}

// keys + neighbour table; returns FC_ERR_UNBALANCED when a neighbour differs
// by more than one level (the table is still written)
int Forest::rebuild_tables()
{
    FC_TRY(key.alloc(n, stream));
    FC_TRY(nbr.alloc((size_t)n * 32, stream));
    FC_TRY(tmp_i.alloc(2, stream));
    k_keys<<<nblk(n, 256), 256, 0, stream>>>(dev(), key.p);
    FC_CUDA(cudaMemsetAsync(tmp_i.p, 0, sizeof(int), stream));
    k_neighbors<<<nblk((long long)n * 8, 256), 256, 0, stream>>>(dev(), nbr.p, tmp_i.p);
    FC_CUDA(cudaGetLastError());
    int bad = 0;
    FC_CUDA(cudaMemcpyAsync(&bad, tmp_i.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
    FC_CUDA(cudaStreamSynchronize(stream));
    if (bad) { set_error("forest is not 2:1 balanced"); return FC_ERR_UNBALANCED; }
    return FC_OK;
}

int Forest::balance(DBuf<int> *origin)
{
    DBuf<int> t2, l2, x2, y2, org2;
    for (int iter = 0; iter < 64; ++iter) {
        FC_TRY(key.alloc(n, stream));
        k_keys<<<nblk(n, 256), 256, 0, stream>>>(dev(), key.p);
        FC_TRY(cnt.alloc(n, stream)); FC_TRY(off.alloc(n, stream)); FC_TRY(tmp_i.alloc(2, stream));
        FC_CUDA(cudaMemsetAsync(cnt.p, 0, n * sizeof(int), stream));
        FC_CUDA(cudaMemsetAsync(tmp_i.p, 0, sizeof(int), stream));
        k_balance_mark<<<nblk((long long)n * 8, 256), 256, 0, stream>>>(dev(), cnt.p, tmp_i.p);
        FC_CUDA(cudaGetLastError());
        int any = 0;
        FC_CUDA(cudaMemcpyAsync(&any, tmp_i.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
        FC_CUDA(cudaStreamSynchronize(stream));
        if (!any) return rebuild_tables();
        // cnt holds marks; turn into output counts in off, scan into off
        DBuf<int> counts;
        FC_TRY(counts.alloc(n, stream));
        k_counts_from_marks<<<nblk(n, 256), 256, 0, stream>>>(cnt.p, counts.p, n);
        int total = 0;
        FC_TRY(exclusive_scan(counts.p, off.p, n, &total, blocksum, stream));
        FC_TRY(t2.alloc(total, stream)); FC_TRY(l2.alloc(total, stream));
        FC_TRY(x2.alloc(total, stream)); FC_TRY(y2.alloc(total, stream));
        if (origin) FC_TRY(org2.alloc((size_t)total * 3, stream));
        k_split<<<nblk(n, 256), 256, 0, stream>>>(dev(), cnt.p, off.p, t2.p, l2.p, x2.p, y2.p,
                                                  origin ? origin->p : nullptr, origin ? org2.p : nullptr);
        FC_CUDA(cudaGetLastError());
        tree.swap(t2); level.swap(l2); x.swap(x2); y.swap(y2);
        if (origin) origin->swap(org2);
        n = total;
    }
    set_error("balance did not converge");
    return FC_ERR_UNBALANCED;
}

int Forest::adapt(const int8_t *d_flags, int min_level, int max_level, DBuf<int> *origin)
{
    DBuf<int> kind, t2, l2, x2, y2;
    FC_TRY(cnt.alloc(n, stream)); FC_TRY(off.alloc(n, stream)); FC_TRY(kind.alloc(n, stream));
    k_adapt_count<<<nblk(n, 256), 256, 0, stream>>>(dev(), d_flags, min_level, max_level, cnt.p, kind.p);
    FC_CUDA(cudaGetLastError());
    int total = 0;
    FC_TRY(exclusive_scan(cnt.p, off.p, n, &total, blocksum, stream));
    FC_TRY(t2.alloc(total, stream)); FC_TRY(l2.alloc(total, stream));
    FC_TRY(x2.alloc(total, stream)); FC_TRY(y2.alloc(total, stream));
    FC_TRY(origin->alloc((size_t)total * 3, stream));
    k_adapt_scatter<<<nblk(n, 256), 256, 0, stream>>>(dev(), kind.p, cnt.p, off.p, t2.p, l2.p, x2.p, y2.p,
                                                      origin->p);
    FC_CUDA(cudaGetLastError());
    tree.swap(t2); level.swap(l2); x.swap(x2); y.swap(y2);
    n = total;
    return balance(origin);
}

int Forest::download(std::vector<int> &t, std::vector<int> &l, std::vector<int> &xx, std::vector<int> &yy) const
{
    t.resize(n); l.resize(n); xx.resize(n); yy.resize(n);
    FC_CUDA(cudaMemcpyAsync(t.data(), tree.p, n * sizeof(int), cudaMemcpyDeviceToHost, stream));
    FC_CUDA(cudaMemcpyAsync(l.data(), level.p, n * sizeof(int), cudaMemcpyDeviceToHost, stream));
    FC_CUDA(cudaMemcpyAsync(xx.data(), x.p, n * sizeof(int), cudaMemcpyDeviceToHost, stream));
    FC_CUDA(cudaMemcpyAsync(yy.data(), y.p, n * sizeof(int), cudaMemcpyDeviceToHost, stream));
    FC_CUDA(cudaStreamSynchronize(stream));
    return FC_OK;
}

}  // namespace fc
