// fc_forest.cuh -- device-resident forest of quadtrees (integer work).
#pragma once
#include <vector>

#include "fc_internal.cuh"

namespace fc {

// RAII device buffer allocated on a stream
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t count = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release()
    {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        count = 0;
    }
    int alloc(size_t n, cudaStream_t st)
    {
        if (n <= count && p) return FC_OK;
        release();
        s = st;
        FC_CUDA(cudaMallocAsync(&p, (n ? n : 1) * sizeof(T), st));
        count = n;
        return FC_OK;
    }
    void swap(DBuf &o)
    {
        std::swap(p, o.p);
        std::swap(count, o.count);
        std::swap(s, o.s);
    }
};

struct Forest {
    cudaStream_t stream = nullptr;
    int conn = FC_CONN_SQUARE;
    int ntab = 1;            // trees of a table connectivity
    DBuf<int> ctab;          // its table [ntab][4][3] (device)
    int n = 0;
    DBuf<int> tree, level, x, y;
    DBuf<uint64_t> key;
    DBuf<int> nbr;           // [n][8][4]
    // scratch
    DBuf<int> cnt, off, tmp_i;
    DBuf<int> blocksum;

    int ntrees() const
    {
        return conn == FC_CONN_TABLE ? ntab : (conn == FC_CONN_SPHERE ? 6 : (conn == FC_CONN_PILLOW ? 2 : 1));
    }
    ForestDev dev() const
    {
        ForestDev d;
        d.n = n; d.conn = conn;
        d.ctab = ctab.p; d.ntrees = ntrees();
        d.tree = tree.p; d.level = level.p; d.x = x.p; d.y = y.p;
        d.key = key.p; d.nbr = nbr.p;
        return d;
    }

    int uniform(int lev);
    int set_leaves(int64_t n, const int32_t *t, const int32_t *l, const int32_t *x, const int32_t *y);
    int rebuild_tables();       // keys + neighbour table; FC_ERR_UNBALANCED if not 2:1
    int balance(DBuf<int> *origin);   // origin[n][3] tracked when non-null
    // apply per-leaf flags (device int8) -> new topology; origin[n][3]
    // {kind 0 same / 1 descendant / 2 parent, old index, level difference}
    int adapt(const int8_t *d_flags, int min_level, int max_level, DBuf<int> *origin);
    int download(std::vector<int> &t, std::vector<int> &l, std::vector<int> &xx, std::vector<int> &yy) const;
};

// exclusive scan of n int32 values (device), total into *h_total (host)
int exclusive_scan(const int *d_in, int *d_out, int n, int *h_total, DBuf<int> &blocksum, cudaStream_t s);

}  // namespace fc
