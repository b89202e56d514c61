/*
 * fco3.c -- FP64 oracle of the three-dimensional patch method (octree of
 * m^3 patches, scalar advection with a constant velocity, periodic unit
 * cube).  TEST INFRASTRUCTURE ONLY; see fco3.h for the scope and for the
 * readings taken where the paper (arXiv:1308.1472) gives no 3D detail.
 *
 * Written for clarity, not speed: leaves are located by binary search on
 * their Morton keys for every ghost cell, every face cell and every transfer.
 */
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "fco3.h"

static char g_err[256];
static void seterr(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
const char *fco3_last_error(void) { return g_err; }

struct fco3 {
    fco3_params p;
    int n;
    int8_t *lv;
    int32_t *x, *y, *z;
    uint64_t *key;
    double *q;          /* n * m^3 */
    double t;
};

/* ------------------------------------------------------------------ keys */
static uint64_t spread3(uint32_t a)
{
    uint64_t r = 0;
    for (int b = 0; b < FCO3_L; ++b) r |= (uint64_t)((a >> b) & 1u) << (3 * b);
    return r;
}
/* Morton key of the lower corner of leaf (l, x, y, z): x takes the lowest bit */
static uint64_t mkey(int l, int32_t x, int32_t y, int32_t z)
{
    int sh = FCO3_L - l;
    return spread3((uint32_t)x << sh) | (spread3((uint32_t)y << sh) << 1) | (spread3((uint32_t)z << sh) << 2);
}
static uint64_t span(int l) { return (uint64_t)1 << (3 * (FCO3_L - l)); }

static int wrap(long long a, long long n) { long long r = a % n; return (int)(r < 0 ? r + n : r); }

/* leaf containing the level-g block (a, b, c) or the first leaf inside it */
static int locate(const fco3 *s, int g, int32_t a, int32_t b, int32_t c)
{
    uint64_t pk = mkey(g, a, b, c);
    int lo = 0, hi = s->n - 1, best = -1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (s->key[mid] <= pk) { best = mid; lo = mid + 1; }
        else hi = mid - 1;
    }
    if (best < 0) return -1;
    int l = s->lv[best];
    if (l <= g) {
        if ((a >> (g - l)) != s->x[best] || (b >> (g - l)) != s->y[best] || (c >> (g - l)) != s->z[best]) return -1;
    } else {
        if ((s->x[best] >> (l - g)) != a || (s->y[best] >> (l - g)) != b || (s->z[best] >> (l - g)) != c) return -1;
    }
    return best;
}

/* ------------------------------------------------------------- storage */
static int mm3(const fco3 *s) { return s->p.m * s->p.m * s->p.m; }
static int P3(const fco3 *s) { int P = s->p.m + 4; return P * P * P; }
/* tile index of cell (i, j, k), each in -2 .. m+1 */
static int tix(const fco3 *s, int i, int j, int k)
{
    int P = s->p.m + 4;
    return (i + 2) + P * ((j + 2) + P * (k + 2));
}
static int cix(const fco3 *s, int i, int j, int k) { int m = s->p.m; return i + m * (j + m * k); }

static void free_forest(fco3 *s)
{
    free(s->lv); free(s->x); free(s->y); free(s->z); free(s->key); free(s->q);
    s->lv = NULL; s->x = s->y = s->z = NULL; s->key = NULL; s->q = NULL; s->n = 0;
}

typedef struct { uint64_t key; int8_t l; int32_t x, y, z; } Leaf;
static int cmp_leaf(const void *a, const void *b)
{
    uint64_t ka = ((const Leaf *)a)->key, kb = ((const Leaf *)b)->key;
    return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

/* replace the forest by the given leaves (sorted here); fields dropped */
static int install(fco3 *s, Leaf *L, int n)
{
    for (int i = 0; i < n; ++i) L[i].key = mkey(L[i].l, L[i].x, L[i].y, L[i].z);
    qsort(L, n, sizeof(Leaf), cmp_leaf);
    free_forest(s);
    s->n = n;
    s->lv = malloc(n); s->x = malloc(4 * (size_t)n); s->y = malloc(4 * (size_t)n); s->z = malloc(4 * (size_t)n);
    s->key = malloc(8 * (size_t)n);
    s->q = calloc((size_t)n * mm3(s), sizeof(double));
    for (int i = 0; i < n; ++i) {
        s->lv[i] = L[i].l; s->x[i] = L[i].x; s->y[i] = L[i].y; s->z[i] = L[i].z; s->key[i] = L[i].key;
    }
    return FCO3_OK;
}

/* the leaves tile the cube in Morton order without gap or overlap */
static int check_cover(const fco3 *s)
{
    uint64_t at = 0;
    for (int i = 0; i < s->n; ++i) {
        if (s->key[i] != at) return 0;
        at += span(s->lv[i]);
    }
    return at == span(0);
}

/* ---------------------------------------------------------- life cycle */
fco3 *fco3_create(const fco3_params *p)
{
    if (!p || p->m < 4 || (p->m & 1) || p->min_level < 0 || p->max_level < p->min_level || p->max_level > 12 ||
        p->limiter < 0 || p->limiter > 1 || p->transverse < 0 || p->transverse > 2 || !(p->cfl > 0.0) ||
        p->subcycle < 0 || p->subcycle > 1) {
        seterr("invalid parameters");
        return NULL;
    }
    fco3 *s = calloc(1, sizeof *s);
    s->p = *p;
    if (fco3_forest_uniform(s, p->min_level) != FCO3_OK) { fco3_destroy(s); return NULL; }
    return s;
}

void fco3_destroy(fco3 *s)
{
    if (!s) return;
    free_forest(s);
    free(s);
}

int fco3_num_leaves(const fco3 *s) { return s->n; }
double fco3_time(const fco3 *s) { return s->t; }

int fco3_forest_uniform(fco3 *s, int level)
{
    if (level < 0 || level > s->p.max_level) { seterr("level out of range"); return FCO3_ERR_ARG; }
    int w = 1 << level, n = w * w * w;
    Leaf *L = malloc(sizeof(Leaf) * n);
    int k = 0;
    for (int z = 0; z < w; ++z)
        for (int y = 0; y < w; ++y)
            for (int x = 0; x < w; ++x) { L[k].l = (int8_t)level; L[k].x = x; L[k].y = y; L[k].z = z; ++k; }
    install(s, L, n);
    free(L);
    s->t = 0.0;
    return FCO3_OK;
}

int fco3_set_leaves(fco3 *s, int n, const int8_t *level, const int32_t *x, const int32_t *y, const int32_t *z)
{
    if (n <= 0) { seterr("no leaves"); return FCO3_ERR_ARG; }
    Leaf *L = malloc(sizeof(Leaf) * n);
    for (int i = 0; i < n; ++i) {
        int l = level[i];
        if (l < 0 || l > s->p.max_level || x[i] < 0 || y[i] < 0 || z[i] < 0 || x[i] >= (1 << l) || y[i] >= (1 << l) ||
            z[i] >= (1 << l)) {
            free(L);
            seterr("leaf %d out of range", i);
            return FCO3_ERR_ARG;
        }
        L[i].l = (int8_t)l; L[i].x = x[i]; L[i].y = y[i]; L[i].z = z[i];
        L[i].key = mkey(l, x[i], y[i], z[i]);
        if (i > 0 && L[i].key <= L[i - 1].key) { free(L); seterr("leaves not in Morton order"); return FCO3_ERR_ARG; }
    }
    fco3 tmp = *s;
    tmp.lv = NULL; tmp.x = tmp.y = tmp.z = NULL; tmp.key = NULL; tmp.q = NULL; tmp.n = 0;
    install(&tmp, L, n);
    free(L);
    if (!check_cover(&tmp)) { free_forest(&tmp); seterr("leaves do not tile the cube"); return FCO3_ERR_ARG; }
    if (!fco3_is_balanced(&tmp)) { free_forest(&tmp); seterr("forest not 2:1 balanced"); return FCO3_ERR_UNBALANCED; }
    free_forest(s);
    *s = tmp;
    return FCO3_OK;
}

int fco3_get_leaves(const fco3 *s, int8_t *level, int32_t *x, int32_t *y, int32_t *z)
{
    for (int i = 0; i < s->n; ++i) { level[i] = s->lv[i]; x[i] = s->x[i]; y[i] = s->y[i]; z[i] = s->z[i]; }
    return FCO3_OK;
}

/* ------------------------------------------------------------- balance */
/* coarsest leaf touching leaf i across direction (dx, dy, dz), or -1 when
   finer leaves cover that side */
static int touching(const fco3 *s, int i, int dx, int dy, int dz)
{
    int l = s->lv[i], w = 1 << l;
    int j = locate(s, l, wrap(s->x[i] + dx, w), wrap(s->y[i] + dy, w), wrap(s->z[i] + dz, w));
    if (j < 0 || s->lv[j] > l) return -1;
    return j;
}

int fco3_is_balanced(const fco3 *s)
{
    for (int i = 0; i < s->n; ++i)
        for (int d = 0; d < 27; ++d) {
            if (d == 13) continue;
            int j = touching(s, i, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1);
            if (j >= 0 && s->lv[j] < s->lv[i] - 1) return 0;
        }
    return 1;
}

/* refine the marked leaves (fields dropped) */
static void refine_marked(fco3 *s, const char *mark)
{
    int add = 0;
    for (int i = 0; i < s->n; ++i) add += mark[i] ? 7 : 0;
    Leaf *L = malloc(sizeof(Leaf) * (s->n + add));
    int k = 0;
    for (int i = 0; i < s->n; ++i) {
        if (!mark[i]) { L[k].l = s->lv[i]; L[k].x = s->x[i]; L[k].y = s->y[i]; L[k].z = s->z[i]; ++k; continue; }
        for (int c = 0; c < 8; ++c) {
            L[k].l = (int8_t)(s->lv[i] + 1);
            L[k].x = 2 * s->x[i] + (c & 1); L[k].y = 2 * s->y[i] + ((c >> 1) & 1); L[k].z = 2 * s->z[i] + (c >> 2);
            ++k;
        }
    }
    install(s, L, k);
    free(L);
}

/* ripple: refine every leaf more than one level coarser than a leaf it
   touches, until none is */
static int balance_forest(fco3 *s)
{
    for (;;) {
        char *mark = calloc(s->n, 1);
        int any = 0;
        for (int i = 0; i < s->n; ++i)
            for (int d = 0; d < 27; ++d) {
                if (d == 13) continue;
                int j = touching(s, i, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1);
                if (j >= 0 && s->lv[j] < s->lv[i] - 1 && !mark[j]) { mark[j] = 1; any = 1; }
            }
        if (!any) { free(mark); return FCO3_OK; }
        for (int i = 0; i < s->n; ++i)
            if (mark[i] && s->lv[i] >= s->p.max_level) { free(mark); seterr("balance needs a level above max_level"); return FCO3_ERR_ARG; }
        refine_marked(s, mark);
        free(mark);
    }
}

int fco3_balance(fco3 *s)
{
    return balance_forest(s);
}

/* -------------------------------------------------------------- fields */
int fco3_set_fields(fco3 *s, const double *q)
{
    memcpy(s->q, q, sizeof(double) * (size_t)s->n * mm3(s));
    return FCO3_OK;
}
int fco3_get_fields(const fco3 *s, double *q)
{
    memcpy(q, s->q, sizeof(double) * (size_t)s->n * mm3(s));
    return FCO3_OK;
}

static double init_value(int kind, const double *a, double x, double y, double z)
{
    if (kind == FCO3_INIT_BOX)
        return (x >= a[0] && x < a[1] && y >= a[2] && y < a[3] && z >= a[4] && z < a[5]) ? a[6] : a[7];
    if (kind == FCO3_INIT_SINE) return a[0] + a[1] * sin(2.0 * M_PI * (a[2] * x + a[3] * y + a[4] * z));
    double dx = x - a[2], dy = y - a[3], dz = z - a[4];
    return a[0] + a[1] * exp(-(dx * dx + dy * dy + dz * dz) / (a[5] * a[5]));
}

int fco3_init(fco3 *s, int kind, const double *prm, int np)
{
    static const int need[3] = {8, 5, 6};
    if (kind < 0 || kind > 2 || np < need[kind]) { seterr("bad initial condition"); return FCO3_ERR_ARG; }
    int m = s->p.m;
    for (int p = 0; p < s->n; ++p) {
        double dx = 1.0 / ((double)m * (double)(1 << s->lv[p]));
        for (int k = 0; k < m; ++k)
            for (int j = 0; j < m; ++j)
                for (int i = 0; i < m; ++i) {
                    double xc = ((double)s->x[p] * m + i + 0.5) * dx;      /* cell-centre point samples */
                    double yc = ((double)s->y[p] * m + j + 0.5) * dx;
                    double zc = ((double)s->z[p] * m + k + 0.5) * dx;
                    s->q[(size_t)p * mm3(s) + cix(s, i, j, k)] = init_value(kind, prm, xc, yc, zc);
                }
    }
    s->t = 0.0;
    return FCO3_OK;
}

/* ----------------------------------------------------------- ghost fill */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* limited linear value of the level-(l+1) cell (gi, gj, gk) inside coarse
   leaf c (level l) from c's complete tile */
static double interp_child(const fco3 *s, int c, const double *tile, long long gi, long long gj, long long gk)
{
    int m = s->p.m;
    int ci = (int)((gi >> 1) - (long long)s->x[c] * m), cj = (int)((gj >> 1) - (long long)s->y[c] * m),
        ck = (int)((gk >> 1) - (long long)s->z[c] * m);
    double qc = tile[tix(s, ci, cj, ck)];
    double sx = minmod(tile[tix(s, ci + 1, cj, ck)] - qc, qc - tile[tix(s, ci - 1, cj, ck)]);
    double sy = minmod(tile[tix(s, ci, cj + 1, ck)] - qc, qc - tile[tix(s, ci, cj - 1, ck)]);
    double sz = minmod(tile[tix(s, ci, cj, ck + 1)] - qc, qc - tile[tix(s, ci, cj, ck - 1)]);
    double ox = (gi & 1) ? 0.25 : -0.25, oy = (gj & 1) ? 0.25 : -0.25, oz = (gk & 1) ? 0.25 : -0.25;
    return ((qc + ox * sx) + oy * sy) + oz * sz;
}

/* the interior values of every level at the time of a fill: a level's
   newer state (cur) and older state (old) blended with weight alpha[l] */
typedef struct {
    const double *cur, *old;
    double alpha[FCO3_L + 1];
} view3;

static void view_now(const fco3 *s, const double *q, view3 *v)
{
    (void)s;
    v->cur = v->old = q;
    for (int l = 0; l <= FCO3_L; ++l) v->alpha[l] = 1.0;
}

static double vval(const fco3 *s, const view3 *v, int p, int c)
{
    size_t o = (size_t)p * mm3(s) + c;
    double a = v->alpha[s->lv[p]];
    if (a == 1.0) return v->cur[o];
    if (a == 0.0) return v->old[o];
    return (1.0 - a) * v->old[o] + a * v->cur[o];
}

/* mean of the eight level-(l+1) cells 2g + {0,1}^3, all inside fine leaf f */
static double average_children(const fco3 *s, const view3 *v, int f, long long gi, long long gj, long long gk)
{
    int m = s->p.m;
    int fi = (int)(2 * gi - (long long)s->x[f] * m), fj = (int)(2 * gj - (long long)s->y[f] * m),
        fk = (int)(2 * gk - (long long)s->z[f] * m);
#define Qv(i, j, k) vval(s, v, f, cix(s, i, j, k))
    double a = Qv(fi, fj, fk) + Qv(fi + 1, fj, fk);
    double b = Qv(fi, fj + 1, fk) + Qv(fi + 1, fj + 1, fk);
    double c = Qv(fi, fj, fk + 1) + Qv(fi + 1, fj, fk + 1);
    double d = Qv(fi, fj + 1, fk + 1) + Qv(fi + 1, fj + 1, fk + 1);
#undef Qv
    return 0.125 * ((a + b) + (c + d));
}

/* complete tiles of the leaves of levels up to `upto`, from the coarsest
   level up (a coarser neighbour's tile is complete when a finer leaf
   interpolates from it), with the interior values of the view */
static int fill_levels3(const fco3 *s, const view3 *v, int upto, double *tiles)
{
    int m = s->p.m, lmin = 99, lmax = -1;
    for (int p = 0; p < s->n; ++p) { if (s->lv[p] < lmin) lmin = s->lv[p]; if (s->lv[p] > lmax) lmax = s->lv[p]; }
    if (upto < lmax) lmax = upto;
    for (int l = lmin; l <= lmax; ++l)
        for (int p = 0; p < s->n; ++p) {
            if (s->lv[p] != l) continue;
            double *T = tiles + (size_t)p * P3(s);
            long long N = (long long)m << l;
            for (int k = -2; k < m + 2; ++k)
                for (int j = -2; j < m + 2; ++j)
                    for (int i = -2; i < m + 2; ++i) {
                        if (i >= 0 && i < m && j >= 0 && j < m && k >= 0 && k < m) {
                            T[tix(s, i, j, k)] = vval(s, v, p, cix(s, i, j, k));
                            continue;
                        }
                        long long gi = wrap((long long)s->x[p] * m + i, N), gj = wrap((long long)s->y[p] * m + j, N),
                                  gk = wrap((long long)s->z[p] * m + k, N);
                        int r = locate(s, l, (int32_t)(gi / m), (int32_t)(gj / m), (int32_t)(gk / m));
                        if (r < 0) { seterr("ghost cell without a leaf"); return FCO3_ERR_ARG; }
                        double val;
                        if (s->lv[r] == l) {
                            val = vval(s, v, r, cix(s, (int)(gi - (long long)s->x[r] * m), (int)(gj - (long long)s->y[r] * m),
                                                    (int)(gk - (long long)s->z[r] * m)));
                        } else if (s->lv[r] == l - 1) {
                            val = interp_child(s, r, tiles + (size_t)r * P3(s), gi, gj, gk);
                        } else if (s->lv[r] < l - 1) {
                            seterr("unbalanced neighbour");
                            return FCO3_ERR_UNBALANCED;
                        } else {
                            int f = locate(s, l + 1, (int32_t)(2 * gi / m), (int32_t)(2 * gj / m), (int32_t)(2 * gk / m));
                            if (f < 0 || s->lv[f] != l + 1) { seterr("unbalanced neighbour"); return FCO3_ERR_UNBALANCED; }
                            val = average_children(s, v, f, gi, gj, gk);
                        }
                        T[tix(s, i, j, k)] = val;
                    }
        }
    return FCO3_OK;
}

static int fill_all(const fco3 *s, const double *q, double *tiles)
{
    view3 v;
    view_now(s, q, &v);
    return fill_levels3(s, &v, 99, tiles);
}

int fco3_fill_tiles(fco3 *s, double *tiles)
{
    return fill_all(s, s->q, tiles);
}

/* -------------------------------------------------------- patch update */
static double mc(double th)
{
    double a = (1.0 + th) / 2.0, r = a < 2.0 ? a : 2.0;
    r = r < 2.0 * th ? r : 2.0 * th;
    return r > 0.0 ? r : 0.0;
}

/* one step of one patch from its complete tile T: new interior values and
   the flux through each boundary face cell as seen from the patch (side
   2d + hi, cells [b][a] over the two other axes in increasing order) */
static void patch_step(const fco3 *s, const double *T, double dt, double dx, double *qn, double *flux)
{
    int m = s->p.m, P = m + 4, N = P * P * P;
    const double vel[3] = {s->p.u, s->p.v, s->p.w};
    const double k = dt / dx;
    double *W = malloc(sizeof(double) * 3 * N), *am = malloc(sizeof(double) * 3 * N), *ap = malloc(sizeof(double) * 3 * N),
           *F = calloc(3 * (size_t)N, sizeof(double));
    int st[3] = {1, P, P * P};
    /* waves and fluctuations at face c - 1/2 along d, stored at cell c */
    for (int d = 0; d < 3; ++d)
        for (int c = 0; c < N; ++c) {
            int cc[3] = {c % P - 2, (c / P) % P - 2, c / (P * P) - 2};
            if (cc[d] < -1) { W[d * N + c] = am[d * N + c] = ap[d * N + c] = 0.0; continue; }
            double w = T[c] - T[c - st[d]];
            W[d * N + c] = w;
            am[d * N + c] = (vel[d] < 0.0 ? vel[d] : 0.0) * w;
            ap[d * N + c] = (vel[d] > 0.0 ? vel[d] : 0.0) * w;
        }
    /* own MC-limited corrections first */
    if (s->p.limiter)
        for (int d = 0; d < 3; ++d)
            for (int c = 0; c < N; ++c) {
                int cc[3] = {c % P - 2, (c / P) % P - 2, c / (P * P) - 2};
                if (cc[d] < 0 || cc[d] > m) continue;
                double w = W[d * N + c], sd = vel[d];
                if (w == 0.0) continue;
                double wu = sd >= 0.0 ? W[d * N + c - st[d]] : W[d * N + c + st[d]];
                double as = fabs(sd);
                F[d * N + c] += 0.5 * as * (1.0 - k * as) * mc(wu / w) * w;
            }
    /* transverse and corner terms of the fluctuations entering cells with
       index in 0..m-1 along their own direction and -1..m along the others */
    if (s->p.transverse)
        for (int d = 0; d < 3; ++d)
            for (int c = 0; c < N; ++c) {
                int cc[3] = {c % P - 2, (c / P) % P - 2, c / (P * P) - 2};
                for (int side = 0; side < 2; ++side) {
                    int X = side == 0 ? c : c - st[d];                      /* cell the fluctuation enters */
                    double A = side == 0 ? ap[d * N + c] : am[d * N + c];
                    int xd = cc[d] - side;
                    if (cc[d] < -1 || xd < 0 || xd > m - 1) continue;
                    int ok = 1;
                    for (int e = 0; e < 3; ++e)
                        if (e != d && (cc[e] < -1 || cc[e] > m)) ok = 0;
                    if (!ok) continue;
                    for (int e = 0; e < 3; ++e) {
                        if (e == d) continue;
                        double se = vel[e], sp = se > 0.0 ? se : 0.0, sm = se < 0.0 ? se : 0.0;
                        F[e * N + X + st[e]] -= 0.5 * k * sp * A;        /* upper e-face of X */
                        F[e * N + X] -= 0.5 * k * sm * A;                /* lower e-face of X */
                        if (s->p.transverse < 2) continue;
                        int f = 3 - d - e;
                        double sf = vel[f], fp = sf > 0.0 ? sf : 0.0, fm = sf < 0.0 ? sf : 0.0;
                        for (int dir = 0; dir < 2; ++dir) {
                            double sg = dir == 0 ? 1.0 : -1.0;
                            double B = (dir == 0 ? sp : sm) * A;           /* part moving towards +e / -e */
                            int Y = dir == 0 ? X + st[e] : X - st[e];       /* cell it moves into */
                            double cm = -sg * k * k / 6.0, co = sg * k * k / 6.0;
                            int ye = cc[e] + (dir == 0 ? 1 : -1);
                            if (ye >= -2 && ye <= m + 1) {
                                if (cc[f] + 1 <= m + 1) F[f * N + Y + st[f]] += cm * fp * B;
                                F[f * N + Y] += cm * fm * B;
                            }
                            if (cc[f] + 1 <= m + 1) F[f * N + X + st[f]] += co * fp * B;
                            F[f * N + X] += co * fm * B;
                        }
                    }
                }
            }
    /* conservative update, x then y then z parts */
    for (int kk = 0; kk < m; ++kk)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                int c = tix(s, i, j, kk);
                double v = T[c];
                for (int d = 0; d < 3; ++d) {
                    double fl = ap[d * N + c] + am[d * N + c + st[d]];
                    double dF = F[d * N + c + st[d]] - F[d * N + c];
                    v = v - k * (fl + dF);
                }
                qn[cix(s, i, j, kk)] = v;
            }
    /* boundary face fluxes as the patch sees them */
    for (int d = 0; d < 3; ++d) {
        int e = d == 0 ? 1 : 0, f = d == 2 ? 1 : 2;
        for (int hi = 0; hi < 2; ++hi)
            for (int b = 0; b < m; ++b)
                for (int a = 0; a < m; ++a) {
                    int cc[3];
                    cc[d] = hi ? m - 1 : 0; cc[e] = a; cc[f] = b;
                    int c = tix(s, cc[0], cc[1], cc[2]);
                    double val;
                    if (hi) val = vel[d] * T[c] + am[d * N + c + st[d]] + F[d * N + c + st[d]];
                    else val = vel[d] * T[c] - ap[d * N + c] + F[d * N + c];
                    flux[(2 * d + hi) * m * m + b * m + a] = val;
                }
    }
    free(W); free(am); free(ap); free(F);
}

/* ------------------------------------------------------------ stepping */
static int finest(const fco3 *s)
{
    int l = 0;
    for (int p = 0; p < s->n; ++p) if (s->lv[p] > l) l = s->lv[p];
    return l;
}
static double smax(const fco3 *s)
{
    double a = fabs(s->p.u), b = fabs(s->p.v), c = fabs(s->p.w);
    double r = a > b ? a : b;
    return r > c ? r : c;
}

static int coarsest(const fco3 *s)
{
    int l = 99;
    for (int p = 0; p < s->n; ++p) if (s->lv[p] < l) l = s->lv[p];
    return l;
}

/* CFL step: one global dt limited by the finest level; under sub-cycling the
   coarse step, every level then at the same Courant number */
double fco3_next_dt(const fco3 *s)
{
    double sm = smax(s);
    if (!(sm > 0.0)) return 0.0;
    int l = s->p.subcycle ? coarsest(s) : finest(s);
    return s->p.cfl * (1.0 / ((double)s->p.m * (double)(1 << l))) / sm;
}

/* kind of the leaf across side `side` of leaf p: 1 same level, 2 coarser, 3 finer */
static int side_kind(const fco3 *s, int p, int side)
{
    int d = side / 2, hi = side & 1, l = s->lv[p], w = 1 << l;
    int c[3] = {s->x[p], s->y[p], s->z[p]};
    c[d] = wrap(c[d] + (hi ? 1 : -1), w);
    int r = locate(s, l, c[0], c[1], c[2]);
    if (r < 0) return 0;
    return s->lv[r] == l ? 1 : (s->lv[r] < l ? 2 : 3);
}

typedef struct {
    int lo, hi;
    long long tick_old[FCO3_L + 1], tick_new[FCO3_L + 1];
    double dtc;
    double *qold, *tiles, *flux, *rec;   /* rec: dt * face flux per side of each leaf */
} step3;

/* update the leaves of level lev (every level if lev < 0) from their tiles
   with step dt, in place; records: sides facing a finer leaf take dt * flux,
   sides facing a coarser leaf add it (summed over the leaf's substeps) */
static void update_level(fco3 *s, step3 *st, int lev, double dt)
{
    int m = s->p.m, M2 = m * m;
    double *qn = malloc(sizeof(double) * mm3(s));
    for (int p = 0; p < s->n; ++p) {
        if (lev >= 0 && s->lv[p] != lev) continue;
        double dx = 1.0 / ((double)m * (double)(1 << s->lv[p]));
        double *fx = st->flux + (size_t)p * 6 * M2;
        patch_step(s, st->tiles + (size_t)p * P3(s), dt, dx, qn, fx);
        memcpy(s->q + (size_t)p * mm3(s), qn, sizeof(double) * mm3(s));
        for (int side = 0; side < 6; ++side) {
            int kind = side_kind(s, p, side);
            double *r = st->rec + ((size_t)p * 6 + side) * M2;
            for (int c = 0; c < M2; ++c) {
                if (kind == 3) r[c] = dt * fx[side * M2 + c];
                else if (kind == 2) r[c] += dt * fx[side * M2 + c];
            }
        }
    }
    free(qn);
}

static void zero_coarse_facing(fco3 *s, step3 *st, int lev)
{
    int M2 = s->p.m * s->p.m;
    for (int p = 0; p < s->n; ++p) {
        if (lev >= 0 && s->lv[p] != lev) continue;
        for (int side = 0; side < 6; ++side)
            if (side_kind(s, p, side) == 2) memset(st->rec + ((size_t)p * 6 + side) * M2, 0, sizeof(double) * M2);
    }
}

/* coarse-fine correction of leaf p: each coarse face cell next to finer
   leaves takes (its record - mean of the four fine records) / dx */
static int reflux_leaf(fco3 *s, const step3 *st, int p)
{
    int m = s->p.m, M2 = m * m, l = s->lv[p];
    long long N = (long long)m << l;
    double idx = (double)m * (double)(1 << l);
    for (int side = 0; side < 6; ++side) {
        int d = side / 2, hi = side & 1;
        int e = d == 0 ? 1 : 0, f = d == 2 ? 1 : 2;
        for (int b = 0; b < m; ++b)
            for (int a = 0; a < m; ++a) {
                long long g[3];
                g[0] = (long long)s->x[p] * m; g[1] = (long long)s->y[p] * m; g[2] = (long long)s->z[p] * m;
                g[d] += hi ? m : -1;                                 /* the cell across the face */
                g[e] += a; g[f] += b;
                for (int t = 0; t < 3; ++t) g[t] = wrap(g[t], N);
                int r = locate(s, l, (int32_t)(g[0] / m), (int32_t)(g[1] / m), (int32_t)(g[2] / m));
                if (r < 0 || s->lv[r] <= l) continue;             /* not a finer neighbour */
                long long fg[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
                if (!hi) fg[d] += 1;                                 /* the fine layer next to the face */
                int fr = locate(s, l + 1, (int32_t)(fg[0] / m), (int32_t)(fg[1] / m), (int32_t)(fg[2] / m));
                if (fr < 0 || s->lv[fr] != l + 1) { seterr("unbalanced face"); return FCO3_ERR_UNBALANCED; }
                long long o[3] = {(long long)s->x[fr] * m, (long long)s->y[fr] * m, (long long)s->z[fr] * m};
                const double *fx = st->rec + ((size_t)fr * 6 + 2 * d + (hi ? 0 : 1)) * M2;
                double ff[4];
                for (int t = 0; t < 4; ++t) {
                    int fa = (int)(fg[e] + (t & 1) - o[e]), fb = (int)(fg[f] + (t >> 1) - o[f]);
                    ff[t] = fx[fb * m + fa];
                }
                double fc = st->rec[((size_t)p * 6 + side) * M2 + b * m + a];
                double mean = 0.25 * ((ff[0] + ff[1]) + (ff[2] + ff[3]));
                int cc[3];
                cc[d] = hi ? m - 1 : 0; cc[e] = a; cc[f] = b;
                double delta = idx * (fc - mean);
                s->q[(size_t)p * mm3(s) + cix(s, cc[0], cc[1], cc[2])] += hi ? delta : -delta;
            }
    }
    return FCO3_OK;
}

/* level lev's next substep, then (for a level with finer leaves) the two
   substeps of the next level and the correction of lev's coarse cells */
static int advance_level3(fco3 *s, step3 *st, int lev)
{
    double dt = st->dtc / (double)(1LL << (lev - st->lo));
    long long T = st->tick_new[lev], ticks = 1LL << (st->hi - lev);
    view3 v;
    v.cur = s->q; v.old = st->qold;
    for (int l = 0; l <= FCO3_L; ++l) {
        long long a = st->tick_old[l], b = st->tick_new[l];
        v.alpha[l] = (b == a) ? 1.0 : (double)(T - a) / (double)(b - a);
    }
    int rc = fill_levels3(s, &v, lev, st->tiles);
    if (rc) return rc;
    for (int p = 0; p < s->n; ++p)
        if (s->lv[p] == lev) memcpy(st->qold + (size_t)p * mm3(s), s->q + (size_t)p * mm3(s), sizeof(double) * mm3(s));
    st->tick_old[lev] = T;
    st->tick_new[lev] = T + ticks;
    update_level(s, st, lev, dt);
    if (lev < st->hi) {
        zero_coarse_facing(s, st, lev + 1);
        if ((rc = advance_level3(s, st, lev + 1))) return rc;
        if ((rc = advance_level3(s, st, lev + 1))) return rc;
        if (s->p.refluxing)
            for (int p = 0; p < s->n; ++p)
                if (s->lv[p] == lev && (rc = reflux_leaf(s, st, p))) return rc;
    }
    return FCO3_OK;
}

static int one_step(fco3 *s, double dt)
{
    int M2 = s->p.m * s->p.m;
    step3 st;
    memset(&st, 0, sizeof st);
    st.lo = coarsest(s);
    st.hi = finest(s);
    st.dtc = dt;
    st.tiles = malloc(sizeof(double) * (size_t)s->n * P3(s));
    st.qold = malloc(sizeof(double) * (size_t)s->n * mm3(s));
    st.flux = malloc(sizeof(double) * (size_t)s->n * 6 * M2);
    st.rec = calloc((size_t)s->n * 6 * M2, sizeof(double));
    int rc;
    if (s->p.subcycle) {
        rc = advance_level3(s, &st, st.lo);
    } else {
        view3 v;
        view_now(s, s->q, &v);
        rc = fill_levels3(s, &v, 99, st.tiles);
        if (!rc) {
            zero_coarse_facing(s, &st, -1);
            update_level(s, &st, -1, dt);
            if (s->p.refluxing)
                for (int p = 0; p < s->n && !rc; ++p) rc = reflux_leaf(s, &st, p);
        }
    }
    if (!rc) s->t += dt;
    free(st.tiles); free(st.qold); free(st.flux); free(st.rec);
    return rc;
}

int fco3_advance(fco3 *s, int nsteps, double dt, double *t_out, double *dt_out)
{
    double sm = smax(s);
    double dxr = 1.0 / ((double)s->p.m * (double)(1 << (s->p.subcycle ? coarsest(s) : finest(s))));
    if (dt <= 0.0) dt = fco3_next_dt(s);
    if (!(dt > 0.0)) { seterr("no time step (zero velocity)"); return FCO3_ERR_ARG; }
    if (dt * sm / dxr > 1.0) { seterr("Courant number %g above 1", dt * sm / dxr); return FCO3_ERR_CFL; }
    for (int n = 0; n < nsteps; ++n) {
        int rc = one_step(s, dt);
        if (rc) return rc;
    }
    if (t_out) *t_out = s->t;
    if (dt_out) *dt_out = dt;
    return FCO3_OK;
}

/* sum of q dx^3 with Neumaier's compensated summation: a plain running sum
   over ~10^5..10^6 cells carries a rounding error near 1e-12 relative, which
   would hide the conservation (to round-off) that the method has */
int fco3_sum(const fco3 *s, double *sum)
{
    double acc = 0.0, comp = 0.0;
    int m = s->p.m;
    for (int p = 0; p < s->n; ++p) {
        double dx = 1.0 / ((double)m * (double)(1 << s->lv[p]));
        double v = dx * dx * dx;
        for (int c = 0; c < mm3(s); ++c) {
            double x = s->q[(size_t)p * mm3(s) + c] * v, t = acc + x;
            comp += fabs(acc) >= fabs(x) ? (acc - t) + x : (x - t) + acc;
            acc = t;
        }
    }
    *sum = acc + comp;
    return FCO3_OK;
}

/* --------------------------------------------------- tagging and regrid */
static double maxmin(const double *Q, int n)
{
    double lo = Q[0], hi = Q[0];
    for (int c = 1; c < n; ++c) { if (Q[c] < lo) lo = Q[c]; if (Q[c] > hi) hi = Q[c]; }
    return hi - lo;
}

/* 8 consecutive leaves starting at i forming one family */
static int is_family(const fco3 *s, int i)
{
    if (i + 8 > s->n || s->lv[i] == 0) return 0;
    int l = s->lv[i];
    if ((s->x[i] & 1) || (s->y[i] & 1) || (s->z[i] & 1)) return 0;
    for (int c = 0; c < 8; ++c) {
        int j = i + c;
        if (s->lv[j] != l || s->x[j] != s->x[i] + (c & 1) || s->y[j] != s->y[i] + ((c >> 1) & 1) ||
            s->z[j] != s->z[i] + (c >> 2))
            return 0;
    }
    return 1;
}

/* parent values of the family starting at leaf i: mean of 2x2x2 children */
static void family_parent(const fco3 *s, const double *q, int i, double *par)
{
    int m = s->p.m, h = m / 2;
    for (int K = 0; K < m; ++K)
        for (int J = 0; J < m; ++J)
            for (int I = 0; I < m; ++I) {
                int c = (I >= h) + 2 * (J >= h) + 4 * (K >= h);
                const double *Q = q + (size_t)(i + c) * mm3(s);
                int fi = 2 * (I % h), fj = 2 * (J % h), fk = 2 * (K % h);
                double a = Q[cix(s, fi, fj, fk)] + Q[cix(s, fi + 1, fj, fk)];
                double b = Q[cix(s, fi, fj + 1, fk)] + Q[cix(s, fi + 1, fj + 1, fk)];
                double cc = Q[cix(s, fi, fj, fk + 1)] + Q[cix(s, fi + 1, fj, fk + 1)];
                double d = Q[cix(s, fi, fj + 1, fk + 1)] + Q[cix(s, fi + 1, fj + 1, fk + 1)];
                par[cix(s, I, J, K)] = 0.125 * ((a + b) + (cc + d));
            }
}

int fco3_tag(fco3 *s, int8_t *flags)
{
    double thr = s->p.tag_threshold;
    double *par = malloc(sizeof(double) * mm3(s));
    for (int i = 0; i < s->n; ++i) {
        double v = maxmin(s->q + (size_t)i * mm3(s), mm3(s));
        flags[i] = (v > thr && s->lv[i] < s->p.max_level) ? 1 : 0;
    }
    for (int i = 0; i < s->n; ++i) {
        if (!is_family(s, i) || s->lv[i] <= s->p.min_level) continue;
        int any = 0;
        for (int c = 0; c < 8; ++c) any |= flags[i + c] != 0 || maxmin(s->q + (size_t)(i + c) * mm3(s), mm3(s)) > thr;
        if (any) { i += 7; continue; }
        family_parent(s, s->q, i, par);
        if (!(maxmin(par, mm3(s)) > thr))
            for (int c = 0; c < 8; ++c) flags[i + c] = -1;
        i += 7;
    }
    free(par);
    return FCO3_OK;
}

int fco3_regrid(fco3 *s, const int8_t *flags)
{
    int m = s->p.m;
    /* old forest, fields and complete tiles */
    fco3 old = *s;
    old.lv = malloc(s->n); old.x = malloc(4 * (size_t)s->n); old.y = malloc(4 * (size_t)s->n);
    old.z = malloc(4 * (size_t)s->n); old.key = malloc(8 * (size_t)s->n);
    old.q = malloc(sizeof(double) * (size_t)s->n * mm3(s));
    memcpy(old.lv, s->lv, s->n); memcpy(old.x, s->x, 4 * (size_t)s->n); memcpy(old.y, s->y, 4 * (size_t)s->n);
    memcpy(old.z, s->z, 4 * (size_t)s->n); memcpy(old.key, s->key, 8 * (size_t)s->n);
    memcpy(old.q, s->q, sizeof(double) * (size_t)s->n * mm3(s));
    double *otiles = malloc(sizeof(double) * (size_t)old.n * P3(s));
    int rc = fill_all(&old, old.q, otiles);
    if (rc) { free(otiles); free_forest(&old); return rc; }

    /* refine wins; a family coarsens when all eight are flagged -1 */
    Leaf *L = malloc(sizeof(Leaf) * (size_t)old.n * 8);
    int k = 0;
    for (int i = 0; i < old.n; ++i) {
        if (is_family(&old, i) && old.lv[i] > s->p.min_level) {
            int all = 1;
            for (int c = 0; c < 8; ++c) all &= flags[i + c] == -1;
            if (all) {
                L[k].l = (int8_t)(old.lv[i] - 1); L[k].x = old.x[i] >> 1; L[k].y = old.y[i] >> 1; L[k].z = old.z[i] >> 1;
                ++k; i += 7;
                continue;
            }
        }
        if (flags[i] == 1 && old.lv[i] < s->p.max_level) {
            for (int c = 0; c < 8; ++c) {
                L[k].l = (int8_t)(old.lv[i] + 1);
                L[k].x = 2 * old.x[i] + (c & 1); L[k].y = 2 * old.y[i] + ((c >> 1) & 1); L[k].z = 2 * old.z[i] + (c >> 2);
                ++k;
            }
        } else {
            L[k].l = old.lv[i]; L[k].x = old.x[i]; L[k].y = old.y[i]; L[k].z = old.z[i]; ++k;
        }
    }
    install(s, L, k);
    free(L);
    rc = balance_forest(s);
    if (rc) { free(otiles); free_forest(&old); return rc; }

    /* transfer: copy, interpolate from the old parent, or average the old children */
    view3 ov;
    view_now(&old, old.q, &ov);
    for (int p = 0; p < s->n; ++p) {
        int l = s->lv[p];
        int r = locate(&old, l, s->x[p], s->y[p], s->z[p]);
        double *Q = s->q + (size_t)p * mm3(s);
        if (r < 0) { seterr("transfer without a source"); rc = FCO3_ERR_ARG; break; }
        if (old.lv[r] == l) {
            memcpy(Q, old.q + (size_t)r * mm3(s), sizeof(double) * mm3(s));
        } else if (old.lv[r] == l - 1) {
            for (int kk = 0; kk < m; ++kk)
                for (int j = 0; j < m; ++j)
                    for (int i = 0; i < m; ++i)
                        Q[cix(s, i, j, kk)] = interp_child(&old, r, otiles + (size_t)r * P3(s), (long long)s->x[p] * m + i,
                                                           (long long)s->y[p] * m + j, (long long)s->z[p] * m + kk);
        } else if (old.lv[r] == l + 1) {
            for (int kk = 0; kk < m; ++kk)
                for (int j = 0; j < m; ++j)
                    for (int i = 0; i < m; ++i) {
                        long long gi = (long long)s->x[p] * m + i, gj = (long long)s->y[p] * m + j, gk = (long long)s->z[p] * m + kk;
                        int f = locate(&old, l + 1, (int32_t)(2 * gi / m), (int32_t)(2 * gj / m), (int32_t)(2 * gk / m));
                        Q[cix(s, i, j, kk)] = average_children(&old, &ov, f, gi, gj, gk);
                    }
        } else {
            seterr("a new leaf more than one level from its old leaves");
            rc = FCO3_ERR_ARG;
            break;
        }
    }
    free(otiles);
    free_forest(&old);
    return rc;
}

int fco3_init_refine(fco3 *s, int kind, const double *prm, int np)
{
    int rc = fco3_forest_uniform(s, s->p.min_level);
    for (int r = 0; r < s->p.max_level - s->p.min_level && rc == FCO3_OK; ++r) {
        rc = fco3_init(s, kind, prm, np);
        if (rc) break;
        int8_t *fl = malloc(s->n);
        fco3_tag(s, fl);
        char *mark = calloc(s->n, 1);
        int any = 0;
        for (int i = 0; i < s->n; ++i) if (fl[i] == 1) { mark[i] = 1; any = 1; }
        free(fl);
        if (any) refine_marked(s, mark);
        free(mark);
        rc = balance_forest(s);
    }
    if (rc == FCO3_OK) rc = fco3_init(s, kind, prm, np);
    return rc;
}
