/*
 * fco_forest.c -- forest of quadtrees for the oracle (TEST INFRASTRUCTURE).
 *
 * Sec. 2 of the paper: the mesh is a forest of quadtrees whose leaves each
 * carry one patch; only per-leaf refine/coarsen flags flow into the mesher;
 * neighbouring leaves may differ by at most one level (2:1 balance).
 * Sec. 4: leaves are kept in space-filling-curve order and neighbours are
 * found by lookup relative to the current leaf, across tree boundaries with a
 * coordinate transformation where the trees are oriented differently.
 *
 * Representation chosen here (plain and slow on purpose):
 *   leaf = (tree, level, x, y), x,y = integer position at the leaf's level;
 *   order = (tree, Morton key of the lower-left corner at FCO_MAXLEVEL bits,
 *            x in the lower interleaved bit), kept by re-sorting with qsort
 *            after every topology change;
 *   point location = binary search for the last leaf whose key is <= the
 *            point's key, then an explicit containment check.
 */
#include "fco_internal.h"
#include <stdlib.h>
#include <string.h>

uint64_t fco_morton(uint32_t X, uint32_t Y)
{
    uint64_t k = 0;
    for (int b = 0; b < FCO_MAXLEVEL; ++b) {
        k |= (uint64_t)((X >> b) & 1u) << (2 * b);
        k |= (uint64_t)((Y >> b) & 1u) << (2 * b + 1);
    }
    return k;
}

uint64_t fco_leaf_key(const fco_leaf *l)
{
    int s = FCO_MAXLEVEL - l->level;
    return fco_morton((uint32_t)l->x << s, (uint32_t)l->y << s);
}

static int cmp_leaf(const void *a, const void *b)
{
    const fco_leaf *p = (const fco_leaf *)a, *q = (const fco_leaf *)b;
    if (p->tree != q->tree) return p->tree < q->tree ? -1 : 1;
    uint64_t kp = fco_leaf_key(p), kq = fco_leaf_key(q);
    if (kp != kq) return kp < kq ? -1 : 1;
    return p->level < q->level ? -1 : (p->level > q->level);
}

void fco_sort_leaves(fco_leaf *l, int n) { qsort(l, (size_t)n, sizeof(fco_leaf), cmp_leaf); }

int fco_num_trees(int conn) { return conn == FCO_CONN_SPHERE ? 6 : (conn == FCO_CONN_PILLOW ? 2 : 1); }

/* ---------------------------------------------------------------------- */
/* Cubed sphere: tree t covers the cube face with outward normal n[t] and  */
/* in-face axes a[t] (the tree's x) and b[t] (the tree's y), a x b = n.   */
const int fco_cube_n[6][3] = {{1,0,0},{0,1,0},{-1,0,0},{0,-1,0},{0,0,1},{0,0,-1}};
const int fco_cube_a[6][3] = {{0,1,0},{-1,0,0},{0,-1,0},{1,0,0},{0,1,0},{0,1,0}};
const int fco_cube_b[6][3] = {{0,0,1},{0,0,1},{0,0,1},{0,0,1},{-1,0,0},{1,0,0}};

static long long dot3(const long long *p, const int *v)
{
    return p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
}

static int tree_with_normal(const long long *v)
{
    for (int t = 0; t < 6; ++t)
        if (fco_cube_n[t][0] == v[0] && fco_cube_n[t][1] == v[1] && fco_cube_n[t][2] == v[2])
            return t;
    return -1;
}

/*
 * Map a point given in doubled centred coordinates (U, V) of tree t -- the
 * cube point is N*n + U*a + V*b with N = 2^FCO_MAXLEVEL -- onto the tree that
 * contains it, folding across a cube edge when exactly one of |U|, |V| is
 * beyond N.  Returns the new tree, or -1 across a cube corner.
 */
static int cube_fold(int t, long long U, long long V, long long *Uo, long long *Vo)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    int outU = (U >= N || U <= -N), outV = (V >= N || V <= -N);
    if (!outU && !outV) { *Uo = U; *Vo = V; return t; }
    if (outU && outV) return -1;
    long long P[3], nn[3];
    long long E, sgn;
    const int *axis;
    if (outU) { sgn = U > 0 ? 1 : -1; E = sgn * U - N; axis = fco_cube_a[t]; }
    else      { sgn = V > 0 ? 1 : -1; E = sgn * V - N; axis = fco_cube_b[t]; }
    for (int k = 0; k < 3; ++k) {
        /* fold the part beyond the edge down along -n */
        long long on = outU ? 0 : U * fco_cube_a[t][k];
        long long ov = outV ? 0 : V * fco_cube_b[t][k];
        P[k] = (N - E) * fco_cube_n[t][k] + sgn * N * axis[k] + on + ov;
        nn[k] = sgn * axis[k];
    }
    int t2 = tree_with_normal(nn);
    *Uo = dot3(P, fco_cube_a[t2]);
    *Vo = dot3(P, fco_cube_b[t2]);
    return t2;
}

/*
 * Locate the tree holding a finest-resolution point (t, X, Y) whose
 * coordinates may lie just outside [0, N).  Returns the tree index and the
 * mapped coordinates, or -1 if the point is outside the domain.
 */
int fco_map_point(int conn, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    if (X >= 0 && X < N && Y >= 0 && Y < N) { *Xo = X; *Yo = Y; return t; }
    if (conn == FCO_CONN_SQUARE) return -1;
    if (conn == FCO_CONN_PERIODIC) {
        *Xo = ((X % N) + N) % N;
        *Yo = ((Y % N) + N) % N;
        return t;
    }
    if (conn == FCO_CONN_PILLOW) {
        /* x beyond a border: the other tree, x continued (the two trees form
         * one strip periodic in x); y beyond a border: the other tree with a
         * half turn; both: the same tree, reflected through the corner */
        if (X >= N) { X -= N; t = 1 - t; }
        else if (X < 0) { X += N; t = 1 - t; }
        if (Y >= N) { Y = 2 * N - 1 - Y; X = N - 1 - X; t = 1 - t; }
        else if (Y < 0) { Y = -1 - Y; X = N - 1 - X; t = 1 - t; }
        *Xo = X; *Yo = Y;
        return t;
    }
    long long U = 2 * X + 1 - N, V = 2 * Y + 1 - N, Uo, Vo;
    int t2 = cube_fold(t, U, V, &Uo, &Vo);
    if (t2 < 0) return -1;
    *Xo = (Uo + N - 1) / 2;
    *Yo = (Vo + N - 1) / 2;
    return t2;
}

/*
 * Table-driven connectivity (Sec. 2: every tree is a reference square, and the
 * trees' connectivity may come from outside, e.g. a mesh generator).
 * tab[(t * 4 + s) * 3 + {0, 1, 2}] for tree t and side s (0 -x, 1 +x, 2 -y,
 * 3 +y) = {neighbour tree (-1: domain boundary), the neighbour's side facing
 * t, 1 if the coordinate along the shared side runs the other way}.  A point
 * beyond one side is carried across it (depth beyond the side = depth inside
 * the neighbour).  A point beyond two sides is carried across both in either
 * order; if both orders end at the same point of the same tree (four cells meet
 * at the corner, or two as on the two-tree sphere) that is the image, otherwise
 * (three trees meet, as at a cube corner) the corner has no image (-1).
 */
static int table_cross(const int32_t *tab, int t, int s, long long X, long long Y, long long *Xo, long long *Yo)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    const int32_t *e = tab + ((size_t)t * 4 + s) * 3;
    if (e[0] < 0) return -1;
    long long along = s < 2 ? Y : X;
    long long depth = s == 0 ? -1 - X : s == 1 ? X - N : s == 2 ? -1 - Y : Y - N;
    long long a2 = e[2] ? N - 1 - along : along;
    switch (e[1]) {
    case 0: *Xo = depth; *Yo = a2; break;
    case 1: *Xo = N - 1 - depth; *Yo = a2; break;
    case 2: *Xo = a2; *Yo = depth; break;
    default: *Xo = a2; *Yo = N - 1 - depth; break;
    }
    return e[0];
}

static int side_beyond(long long v, int lo_side)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    return v < 0 ? lo_side : v >= N ? lo_side + 1 : -1;
}

/* across side s, then across whichever side the point is still beyond */
static int table_two(const int32_t *tab, int t, int s, long long X, long long Y, long long *Xo, long long *Yo)
{
    long long X1, Y1;
    int t1 = table_cross(tab, t, s, X, Y, &X1, &Y1);
    if (t1 < 0) return -1;
    int sx = side_beyond(X1, 0), sy = side_beyond(Y1, 2);
    if ((sx >= 0) == (sy >= 0)) return -1;          /* must be beyond exactly one side now */
    int t2 = table_cross(tab, t1, sx >= 0 ? sx : sy, X1, Y1, Xo, Yo);
    if (t2 < 0 || side_beyond(*Xo, 0) >= 0 || side_beyond(*Yo, 2) >= 0) return -1;
    return t2;
}

int fco_table_map_point(const int32_t *tab, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    int sx = side_beyond(X, 0), sy = side_beyond(Y, 2);
    if (sx < 0 && sy < 0) { *Xo = X; *Yo = Y; return t; }
    if (sx < 0 || sy < 0) {
        int t1 = table_cross(tab, t, sx >= 0 ? sx : sy, X, Y, Xo, Yo);
        if (t1 < 0 || side_beyond(*Xo, 0) >= 0 || side_beyond(*Yo, 2) >= 0) return -1;
        return t1;
    }
    long long Xa, Ya, Xb, Yb;
    int ta = table_two(tab, t, sx, X, Y, &Xa, &Ya);
    int tb = table_two(tab, t, sy, X, Y, &Xb, &Yb);
    if (ta < 0 || tb < 0 || ta != tb || Xa != Xb || Ya != Yb) return -1;
    *Xo = Xa; *Yo = Ya;
    return ta;
}

int fco_sim_num_trees(const fco_sim *s)
{
    return s->p.conn == FCO_CONN_TABLE ? s->ntab : fco_num_trees(s->p.conn);
}

int fco_sim_map_point(const fco_sim *s, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    if (s->p.conn != FCO_CONN_TABLE) return fco_map_point(s->p.conn, t, X, Y, Xo, Yo);
    if (!s->table) return -1;
    return fco_table_map_point(s->table, t, X, Y, Xo, Yo);
}

/*
 * Orientation of the index map from tree t into tree t2 across the face
 * crossed by the point (X, Y).  Encoded from the 2x2 matrix M taking offsets
 * (dX, dY) in t to offsets in t2: 0 = same tree without transform, else
 * 1 + 4*swap + 2*(row 0 negative) + (row 1 negative).
 */
int fco_orientation(int conn, int t, long long X, long long Y)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    if (conn != FCO_CONN_SPHERE && conn != FCO_CONN_PILLOW) return 0;
    if (X >= 0 && X < N && Y >= 0 && Y < N) return 0;
    long long X0, Y0, X1, Y1, X2, Y2;
    int ta = fco_map_point(conn, t, X, Y, &X0, &Y0);
    if (ta < 0) return 0;
    /* step one unit along x and y, staying on the same side of the edge */
    long long sx = (X < 0 || X >= N) ? (X < 0 ? -1 : 1) : 1;
    long long sy = (Y < 0 || Y >= N) ? (Y < 0 ? -1 : 1) : 1;
    if (X >= 0 && X < N && X + sx >= N) sx = -1;
    if (Y >= 0 && Y < N && Y + sy >= N) sy = -1;
    fco_map_point(conn, t, X + sx, Y, &X1, &Y1);
    fco_map_point(conn, t, X, Y + sy, &X2, &Y2);
    long long m00 = (X1 - X0) * sx, m10 = (Y1 - Y0) * sx; /* image of +x */
    long long m01 = (X2 - X0) * sy, m11 = (Y2 - Y0) * sy; /* image of +y */
    int swap = (m00 == 0);
    int r0 = swap ? (m01 < 0) : (m00 < 0);
    int r1 = swap ? (m10 < 0) : (m11 < 0);
    return 1 + 4 * swap + 2 * r0 + r1;
}

/* as fco_orientation, for the simulation's connectivity; with a table every
 * crossing of a tree side is encoded (the identity as 1), a point inside the
 * tree as 0 */
int fco_sim_orientation(const fco_sim *s, int t, long long X, long long Y)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    if (s->p.conn != FCO_CONN_TABLE) return fco_orientation(s->p.conn, t, X, Y);
    if (X >= 0 && X < N && Y >= 0 && Y < N) return 0;
    long long X0, Y0, X1, Y1, X2, Y2;
    if (fco_sim_map_point(s, t, X, Y, &X0, &Y0) < 0) return 0;
    long long sx = (X < 0 || X >= N) ? (X < 0 ? -1 : 1) : 1;
    long long sy = (Y < 0 || Y >= N) ? (Y < 0 ? -1 : 1) : 1;
    if (X >= 0 && X < N && X + sx >= N) sx = -1;
    if (Y >= 0 && Y < N && Y + sy >= N) sy = -1;
    fco_sim_map_point(s, t, X + sx, Y, &X1, &Y1);
    fco_sim_map_point(s, t, X, Y + sy, &X2, &Y2);
    long long m00 = (X1 - X0) * sx, m10 = (Y1 - Y0) * sx;
    long long m01 = (X2 - X0) * sy, m11 = (Y2 - Y0) * sy;
    int swap = (m00 == 0);
    int r0 = swap ? (m01 < 0) : (m00 < 0);
    int r1 = swap ? (m10 < 0) : (m11 < 0);
    return 1 + 4 * swap + 2 * r0 + r1;
}

/* last leaf in tree t whose key <= key(X,Y), checked for containment */
int fco_find_leaf(const fco_sim *s, int t, long long X, long long Y)
{
    int lo = s->tree_first[t], hi = s->tree_first[t + 1] - 1, best = -1;
    uint64_t k = fco_morton((uint32_t)X, (uint32_t)Y);
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (fco_leaf_key(&s->leaves[mid]) <= k) { best = mid; lo = mid + 1; }
        else hi = mid - 1;
    }
    if (best < 0) return -1;
    const fco_leaf *l = &s->leaves[best];
    int sh = FCO_MAXLEVEL - l->level;
    if ((X >> sh) != l->x || (Y >> sh) != l->y) return -1;
    return best;
}

void fco_index_trees(fco_sim *s)
{
    int nt = fco_sim_num_trees(s);
    for (int t = 0; t <= nt; ++t) s->tree_first[t] = s->n;
    for (int i = s->n - 1; i >= 0; --i) s->tree_first[s->leaves[i].tree] = i;
    for (int t = nt - 1; t >= 0; --t)
        if (s->tree_first[t] > s->tree_first[t + 1]) s->tree_first[t] = s->tree_first[t + 1];
}

/* probe points (finest resolution) outside leaf l in direction d, q-th probe */
static void probe_point(const fco_leaf *l, int d, int q, long long *X, long long *Y)
{
    int sh = FCO_MAXLEVEL - l->level;
    long long S = 1LL << sh, X0 = (long long)l->x << sh, Y0 = (long long)l->y << sh;
    long long along = q == 0 ? S / 4 : 3 * S / 4;
    switch (d) {
    case 0: *X = X0 - 1; *Y = Y0 + along; break;
    case 1: *X = X0 + S; *Y = Y0 + along; break;
    case 2: *X = X0 + along; *Y = Y0 - 1; break;
    case 3: *X = X0 + along; *Y = Y0 + S; break;
    case 4: *X = X0 - 1; *Y = Y0 - 1; break;
    case 5: *X = X0 + S; *Y = Y0 - 1; break;
    case 6: *X = X0 - 1; *Y = Y0 + S; break;
    default: *X = X0 + S; *Y = Y0 + S; break;
    }
}

/* leaf containing a probe point, or -1 outside the domain */
static int locate(const fco_sim *s, int t, long long X, long long Y)
{
    long long Xm, Ym;
    int t2 = fco_sim_map_point(s, t, X, Y, &Xm, &Ym);
    if (t2 < 0) return -1;
    return fco_find_leaf(s, t2, Xm, Ym);
}

int fco_build_neighbors(fco_sim *s, int32_t *tab)
{
    for (int i = 0; i < s->n; ++i) {
        const fco_leaf *l = &s->leaves[i];
        for (int d = 0; d < 8; ++d) {
            int32_t *e = tab + ((size_t)i * 8 + d) * 4;
            long long X, Y;
            probe_point(l, d, 0, &X, &Y);
            int n0 = locate(s, l->tree, X, Y);
            e[0] = FCO_NB_NONE; e[1] = -1; e[2] = -1; e[3] = 0;
            if (n0 < 0) continue;
            e[3] = fco_sim_orientation(s, l->tree, X, Y);
            int dl = s->leaves[n0].level - l->level;
            if (dl == 0) { e[0] = FCO_NB_SAME; e[1] = n0; }
            else if (dl == -1) { e[0] = FCO_NB_COARSER; e[1] = n0; }
            else if (dl == 1) {
                e[0] = FCO_NB_FINER; e[1] = n0;
                if (d < 4) {
                    long long X1, Y1;
                    probe_point(l, d, 1, &X1, &Y1);
                    int n1 = locate(s, l->tree, X1, Y1);
                    if (n1 < 0 || s->leaves[n1].level != l->level + 1) return FCO_ERR_UNBALANCED;
                    e[2] = n1;
                }
            } else return FCO_ERR_UNBALANCED;
        }
    }
    return FCO_OK;
}

int fco_get_neighbors(const fco_sim *s, int32_t *table)
{
    return fco_build_neighbors((fco_sim *)s, table);
}

/* 1 if every face and corner neighbour differs by at most one level */
int fco_is_balanced(const fco_sim *s)
{
    for (int i = 0; i < s->n; ++i) {
        const fco_leaf *l = &s->leaves[i];
        for (int d = 0; d < 8; ++d)
            for (int q = 0; q < (d < 4 ? 2 : 1); ++q) {
                long long X, Y;
                probe_point(l, d, q, &X, &Y);
                int n0 = locate(s, l->tree, X, Y);
                if (n0 < 0) continue;
                int dl = s->leaves[n0].level - l->level;
                if (dl < -1 || dl > 1) return 0;
            }
    }
    return 1;
}

/* replace every marked leaf by its four children; returns the new count */
static int split_marked(fco_leaf **leaves, int n, const char *mark)
{
    int nn = 0;
    for (int i = 0; i < n; ++i) nn += mark[i] ? 4 : 1;
    fco_leaf *out = (fco_leaf *)malloc(sizeof(fco_leaf) * (size_t)nn);
    int k = 0;
    for (int i = 0; i < n; ++i) {
        fco_leaf l = (*leaves)[i];
        if (!mark[i]) { out[k++] = l; continue; }
        for (int c = 0; c < 4; ++c) {
            fco_leaf ch = {l.tree, l.level + 1, 2 * l.x + (c & 1), 2 * l.y + (c >> 1)};
            out[k++] = ch;
        }
    }
    fco_sort_leaves(out, nn);
    free(*leaves);
    *leaves = out;
    return nn;
}

/*
 * Ripple balance (face and corner): any leaf that a neighbour probe finds
 * more than one level coarser than the probing leaf is split; repeat until
 * nothing is marked.  The result is the coarsest balanced refinement.
 */
int fco_balance_topology(fco_sim *s)
{
    for (;;) {
        char *mark = (char *)calloc((size_t)s->n, 1);
        int any = 0;
        for (int i = 0; i < s->n; ++i) {
            const fco_leaf *l = &s->leaves[i];
            for (int d = 0; d < 8; ++d) {
                long long X, Y;
                probe_point(l, d, 0, &X, &Y);
                int n0 = locate(s, l->tree, X, Y);
                if (n0 >= 0 && s->leaves[n0].level < l->level - 1) { mark[n0] = 1; any = 1; }
            }
        }
        if (any) { s->n = split_marked(&s->leaves, s->n, mark); fco_index_trees(s); }
        free(mark);
        if (!any) return FCO_OK;
    }
}

int fco_num_leaves(const fco_sim *s) { return s->n; }

int fco_get_leaves(const fco_sim *s, int32_t *tree, int32_t *level, int32_t *x, int32_t *y)
{
    for (int i = 0; i < s->n; ++i) {
        if (tree) tree[i] = s->leaves[i].tree;
        if (level) level[i] = s->leaves[i].level;
        if (x) x[i] = s->leaves[i].x;
        if (y) y[i] = s->leaves[i].y;
    }
    return FCO_OK;
}

void fco_set_topology(fco_sim *s, fco_leaf *leaves, int n)
{
    free(s->leaves);
    s->leaves = leaves;
    s->n = n;
    fco_index_trees(s);
}

int fco_forest_uniform_topology(fco_sim *s, int level)
{
    if (level < 0 || level > 15) return FCO_ERR_ARG;
    int nt = fco_sim_num_trees(s), side = 1 << level;
    int n = nt * side * side;
    fco_leaf *l = (fco_leaf *)malloc(sizeof(fco_leaf) * (size_t)n);
    int k = 0;
    for (int t = 0; t < nt; ++t)
        for (int y = 0; y < side; ++y)
            for (int x = 0; x < side; ++x) { fco_leaf a = {t, level, x, y}; l[k++] = a; }
    fco_sort_leaves(l, n);
    fco_set_topology(s, l, n);
    return FCO_OK;
}

int fco_forest_set_leaves_topology(fco_sim *s, int n, const int32_t *tree, const int32_t *level,
                                   const int32_t *x, const int32_t *y)
{
    int nt = fco_sim_num_trees(s);
    fco_leaf *l = (fco_leaf *)malloc(sizeof(fco_leaf) * (size_t)(n > 0 ? n : 1));
    unsigned long long area = 0, full = (unsigned long long)nt << 40;
    for (int i = 0; i < n; ++i) {
        if (tree[i] < 0 || tree[i] >= nt || level[i] < 0 || level[i] > 20 ||
            x[i] < 0 || y[i] < 0 || x[i] >= (1 << level[i]) || y[i] >= (1 << level[i])) {
            free(l); return FCO_ERR_ARG;
        }
        fco_leaf a = {tree[i], level[i], x[i], y[i]};
        l[i] = a;
        area += 1ULL << (2 * (20 - level[i]));
    }
    fco_sort_leaves(l, n);
    /* leaves must tile the domain: no overlaps and full area */
    for (int i = 0; i + 1 < n; ++i) {
        const fco_leaf *a = &l[i], *b = &l[i + 1];
        if (a->tree != b->tree) continue;
        int sh = FCO_MAXLEVEL - a->level;
        uint64_t ka = fco_leaf_key(a), kb = fco_leaf_key(b);
        if (kb < ka + (1ULL << (2 * sh))) { free(l); return FCO_ERR_ARG; }
    }
    if (area != full) { free(l); return FCO_ERR_ARG; }
    fco_set_topology(s, l, n);
    return FCO_OK;
}

/*
 * New topology from flags (regrid rule used throughout):
 *   refine wins over coarsen; a family of four sibling leaves coarsens iff all
 *   four are flagged -1 and the family's level is above min_level; leaves
 *   flagged +1 below max_level split; then the forest is balanced by
 *   refinement only.  The result does not depend on the order of the leaves.
 * origin[k] for every new leaf k: {kind, old index, level difference}, kind
 * 0 = same leaf, 1 = descendant of old leaf, 2 = parent of old leaves
 * old..old+3.
 */
int fco_adapt(fco_sim *s, const int8_t *flags, int32_t **origin_out)
{
    int n = s->n;
    fco_leaf *tmp = (fco_leaf *)malloc(sizeof(fco_leaf) * (size_t)(4 * n + 4));
    int k = 0;
    for (int i = 0; i < n;) {
        const fco_leaf *l = &s->leaves[i];
        int fam = 0;
        if (l->level > s->p.min_level && (l->x & 1) == 0 && (l->y & 1) == 0 && i + 3 < n) {
            fam = 1;
            for (int c = 0; c < 4; ++c) {
                const fco_leaf *m = &s->leaves[i + c];
                if (m->tree != l->tree || m->level != l->level ||
                    m->x != l->x + (c & 1) || m->y != l->y + (c >> 1) || flags[i + c] != -1) fam = 0;
            }
        }
        if (fam) {
            fco_leaf p = {l->tree, l->level - 1, l->x >> 1, l->y >> 1};
            tmp[k++] = p;
            i += 4;
            continue;
        }
        if (flags[i] > 0 && l->level < s->p.max_level) {
            for (int c = 0; c < 4; ++c) {
                fco_leaf ch = {l->tree, l->level + 1, 2 * l->x + (c & 1), 2 * l->y + (c >> 1)};
                tmp[k++] = ch;
            }
        } else tmp[k++] = *l;
        ++i;
    }
    fco_leaf *old = s->leaves;
    int nold = s->n;
    s->leaves = (fco_leaf *)malloc(sizeof(fco_leaf) * (size_t)k);
    memcpy(s->leaves, tmp, sizeof(fco_leaf) * (size_t)k);
    free(tmp);
    s->n = k;
    fco_sort_leaves(s->leaves, s->n);
    fco_index_trees(s);
    fco_balance_topology(s);

    if (origin_out) {
        int32_t *org = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)s->n);
        /* locate each new leaf relative to the old forest by its lower-left
         * corner: the old leaf containing that corner is either the same
         * leaf, an ancestor (new leaf is a descendant) or a child (new leaf is
         * the parent of a coarsened family). */
        fco_sim olds = *s;
        olds.leaves = old; olds.n = nold;
        fco_index_trees(&olds);
        for (int j = 0; j < s->n; ++j) {
            const fco_leaf *l = &s->leaves[j];
            int sh = FCO_MAXLEVEL - l->level;
            int o = fco_find_leaf(&olds, l->tree, (long long)l->x << sh, (long long)l->y << sh);
            int dl = l->level - old[o].level;
            org[3 * j] = dl == 0 ? 0 : (dl > 0 ? 1 : 2);
            org[3 * j + 1] = o;
            org[3 * j + 2] = dl;
        }
        *origin_out = org;
    }
    free(old);
    return FCO_OK;
}
