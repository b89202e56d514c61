/*
 * fco_sim.c -- ghost fill, patch update, coarse-fine correction, time
 * stepping, tagging and regrid for the oracle (TEST INFRASTRUCTURE).
 *
 * Sec. 3 of the paper: each patch has two ghost layers; ghost values come from
 * a same-level neighbour (copy), a finer neighbour (average of its cells) or a
 * coarser neighbour (conservative, limited interpolation), with time-accurate
 * coarse data under sub-cycling; regrid interpolates to new fine patches and
 * averages to new coarse ones.  Sec. 4: one global dt, or a per-level dt with
 * a coarse-to-fine recursion followed by fine-to-coarse correction.
 *
 * Readings where the paper is silent (each is a numbered reading in the design
 * notes and is shared by both implementations):
 *  - ghost fill runs level by level, coarsest first; a coarser neighbour's
 *    complete ghost-filled array (interior + two ghost layers) is the source
 *    of coarse-to-fine interpolation;
 *  - fine-to-coarse value = 0.25 ((SW + SE) + (NW + NE)) in the receiving
 *    patch's axes;
 *  - coarse-to-fine value = Qc + sx*sigx + sy*sigy, sigma = +-1/4, slopes
 *    minmod of the one-sided coarse differences;
 *  - reflecting walls mirror the two nearest interior layers and negate the
 *    normal momentum, x walls first, then y walls over the full padded width;
 *  - the correction flux at an edge is its own MC-limited correction followed
 *    by the transverse parts of the four neighbouring perpendicular edges in
 *    the order below-left, below-right, above-left, above-right;
 *  - the coarse-fine correction uses the effective edge flux seen by each
 *    boundary cell: f(Q_cell) + (fluctuation toward that cell across the edge,
 *    with sign) + correction flux, integrated over each patch's own steps.
 */
#include "fco_internal.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>


static char g_err[256];
static void set_err(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char *fco_last_error(void) { return g_err; }

static double minv(double a, double b) { return a < b ? a : b; }

/* mapped spheres: the six-tree cubed sphere and the two-tree sphere share
 * the capacity-form advection; only the map differs */
static int is_sphere(int conn) { return conn == FCO_CONN_SPHERE || conn == FCO_CONN_PILLOW; }

static void map_point(const fco_sim *s, int t, long long U, long long V, double p[3])
{
    if (s->p.conn == FCO_CONN_PILLOW) fco_pillow_point(t, U, V, p);
    else fco_sphere_point(t, U, V, p);
}

static double map_area(const fco_sim *s, int t, long long U0, long long U1, long long V0, long long V1)
{
    return s->p.conn == FCO_CONN_PILLOW ? fco_pillow_cell_area(t, U0, U1, V0, V1)
                                        : fco_sphere_cell_area(t, U0, U1, V0, V1);
}
static double maxv(double a, double b) { return a > b ? a : b; }

/* ---------------------------------------------------------------------- */
fco_sim *fco_create(const fco_params *p)
{
    if (!p || p->m < 4 || (p->m & 1) || p->m > 64 || p->min_level < 0 ||
        p->max_level < p->min_level || p->max_level > 14) { set_err("bad params"); return NULL; }
    if (p->conn < FCO_CONN_SQUARE || p->conn > FCO_CONN_TABLE) { set_err("bad connectivity"); return NULL; }
    if (is_sphere(p->conn) && p->equation != FCO_EQ_ADV) { set_err("sphere needs advection"); return NULL; }
    if (p->transverse < 0 || p->transverse > 2 || p->entropy_fix < 0 || p->entropy_fix > 1) {
        set_err("bad transverse / entropy_fix"); return NULL;
    }
    if (p->transverse == 2 && is_sphere(p->conn)) { set_err("T2 is for the square"); return NULL; }
    if (p->velocity < 0 || p->velocity > 1 || (p->velocity == FCO_VEL_SWIRL && p->equation != FCO_EQ_ADV)) {
        set_err("bad velocity field"); return NULL;
    }
    fco_sim *s = (fco_sim *)calloc(1, sizeof(fco_sim));
    s->p = *p;
    s->F = p->equation == FCO_EQ_SWE ? 3 : 1;
    s->dt_from_cells = 1;
    s->ntab = 1;                 /* a table connectivity: one tree until its table is set */
    fco_forest_uniform(s, p->min_level);
    return s;
}

void fco_destroy(fco_sim *s)
{
    if (!s) return;
    free(s->leaves);
    free(s->q);
    free(s->table);
    free(s);
}

int fco_set_connectivity(fco_sim *s, int ntrees, const int32_t *table)
{
    if (s->p.conn != FCO_CONN_TABLE || ntrees < 1 || ntrees > FCO_MAX_TREES || !table) {
        set_err("fco_set_connectivity: bad arguments");
        return FCO_ERR_ARG;
    }
    for (int k = 0; k < ntrees * 4; ++k) {
        const int32_t *e = table + 3 * k;
        if (e[0] < -1 || e[0] >= ntrees || (e[0] >= 0 && (e[1] < 0 || e[1] > 3 || e[2] < 0 || e[2] > 1))) {
            set_err("fco_set_connectivity: bad table entry");
            return FCO_ERR_ARG;
        }
    }
    free(s->table);
    s->table = (int32_t *)malloc(sizeof(int32_t) * 12 * (size_t)ntrees);
    memcpy(s->table, table, sizeof(int32_t) * 12 * (size_t)ntrees);
    s->ntab = ntrees;
    return fco_forest_uniform(s, s->p.min_level);
}

int fco_num_fields(const fco_sim *s) { return s->F; }

static size_t patch_cells(const fco_sim *s) { return (size_t)s->p.m * s->p.m; }
static size_t patch_pad(const fco_sim *s) { return (size_t)FCO_PAD(s->p.m) * FCO_PAD(s->p.m); }

static void realloc_fields(fco_sim *s)
{
    free(s->q);
    s->q = (double *)calloc((size_t)s->n * s->F * patch_cells(s) + 1, sizeof(double));
}

int fco_forest_uniform(fco_sim *s, int level)
{
    int rc = fco_forest_uniform_topology(s, level);
    if (rc) return rc;
    realloc_fields(s);
    s->dt_from_cells = 1;
    return FCO_OK;
}

int fco_forest_set_leaves(fco_sim *s, int n, const int32_t *tree, const int32_t *level,
                          const int32_t *x, const int32_t *y)
{
    int rc = fco_forest_set_leaves_topology(s, n, tree, level, x, y);
    if (rc) { set_err("leaves do not tile the domain"); return rc; }
    realloc_fields(s);
    s->dt_from_cells = 1;
    return FCO_OK;
}

int fco_balance(fco_sim *s)
{
    int rc = fco_balance_topology(s);
    realloc_fields(s);
    return rc;
}

int fco_adapt_topology(fco_sim *s, const int8_t *flags)
{
    int rc = fco_adapt(s, flags, NULL);
    realloc_fields(s);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* geometry of the unit square: cell size and cell centre                  */
static double cell_dx(const fco_sim *s, int level) { return 1.0 / ((double)(1 << level) * s->p.m); }

static void cell_center(const fco_sim *s, const fco_leaf *l, int i, int j, double *x, double *y)
{
    double dx = cell_dx(s, l->level);
    *x = ((double)l->x * s->p.m + i + 0.5) * dx;
    *y = ((double)l->y * s->p.m + j + 0.5) * dx;
}

/* ---------------------------------------------------------------------- */
/* initial data: point samples at cell centres                             */
int fco_init_fields(fco_sim *s, int kind, const double *p, int np)
{
    if (s->p.conn == FCO_CONN_TABLE) { set_err("fco_init_fields: a table connectivity has no fields"); return FCO_ERR_ARG; }
    int m = s->p.m, F = s->F;
    if (s->p.equation == FCO_EQ_SWE && kind != FCO_INIT_DAMBREAK && kind != FCO_INIT_HUMPS) return FCO_ERR_ARG;
    if (s->p.equation == FCO_EQ_ADV && kind != FCO_INIT_ADV_BOX && kind != FCO_INIT_ADV_SINE && kind != FCO_INIT_HILL &&
        kind != FCO_INIT_HALF)
        return FCO_ERR_ARG;
    if ((kind == FCO_INIT_HILL || kind == FCO_INIT_HALF) != is_sphere(s->p.conn)) return FCO_ERR_ARG;
    if (kind == FCO_INIT_HILL && np < 3) return FCO_ERR_ARG;
    if (kind == FCO_INIT_HALF && np < 2) return FCO_ERR_ARG;
    if (kind == FCO_INIT_DAMBREAK && np < 5) return FCO_ERR_ARG;
    if (kind == FCO_INIT_HUMPS && (np < 1 || (np - 1) % 4)) return FCO_ERR_ARG;
    if (kind == FCO_INIT_ADV_BOX && np < 6) return FCO_ERR_ARG;
    if (kind == FCO_INIT_ADV_SINE && np < 4) return FCO_ERR_ARG;
    for (int k = 0; k < s->n; ++k) {
        const fco_leaf *l = &s->leaves[k];
        double *q = s->q + (size_t)k * F * m * m;
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                double x, y;
                cell_center(s, l, i, j, &x, &y);
                int c = j * m + i;
                if (kind == FCO_INIT_DAMBREAK) {
                    double dxx = x - p[0], dyy = y - p[1];
                    q[c] = (dxx * dxx + dyy * dyy < p[2]) ? p[3] : p[4];
                    q[m * m + c] = 0.0; q[2 * m * m + c] = 0.0;
                } else if (kind == FCO_INIT_HUMPS) {
                    double h = p[0];
                    for (int b = 0; b < (np - 1) / 4; ++b) {
                        const double *hp = p + 1 + 4 * b;
                        double dxx = x - hp[2], dyy = y - hp[3];
                        h += hp[0] * exp(-(dxx * dxx + dyy * dyy) / (hp[1] * hp[1]));
                    }
                    q[c] = h; q[m * m + c] = 0.0; q[2 * m * m + c] = 0.0;
                } else if (kind == FCO_INIT_HALF) {
                    /* Example 2: 0 on one half of the sphere, 1 on the other */
                    const long long N = 1LL << FCO_MAXLEVEL;
                    long long w2 = 2 * ((1LL << (FCO_MAXLEVEL - l->level)) / m);
                    long long U = ((long long)l->x * m + i) * w2 + w2 / 2 - N;
                    long long V = ((long long)l->y * m + j) * w2 + w2 / 2 - N;
                    double pt[3], ce[3] = {cos(p[1]) * cos(p[0]), cos(p[1]) * sin(p[0]), sin(p[1])};
                    map_point(s, l->tree, U, V, pt);
                    q[c] = ((pt[0] * ce[0] + pt[1] * ce[1]) + pt[2] * ce[2]) > 0.0 ? 1.0 : 0.0;
                } else if (kind == FCO_INIT_HILL) {
                    /* Gaussian of the great-circle distance to the centre */
                    const long long N = 1LL << FCO_MAXLEVEL;
                    long long w2 = 2 * ((1LL << (FCO_MAXLEVEL - l->level)) / m);
                    long long U = ((long long)l->x * m + i) * w2 + w2 / 2 - N;
                    long long V = ((long long)l->y * m + j) * w2 + w2 / 2 - N;
                    double pt[3], ce[3] = {cos(p[1]) * cos(p[0]), cos(p[1]) * sin(p[0]), sin(p[1])};
                    map_point(s, l->tree, U, V, pt);
                    double ch = sqrt(((pt[0] - ce[0]) * (pt[0] - ce[0]) + (pt[1] - ce[1]) * (pt[1] - ce[1])) +
                                     (pt[2] - ce[2]) * (pt[2] - ce[2]));
                    double d = 2.0 * asin(ch < 2.0 ? 0.5 * ch : 1.0);
                    q[c] = exp(-(d * d) / (p[2] * p[2]));
                } else if (kind == FCO_INIT_ADV_BOX) {
                    q[c] = (x >= p[0] && x < p[1] && y >= p[2] && y < p[3]) ? p[4] : p[5];
                } else {
                    q[c] = p[0] + p[1] * sin(2.0 * M_PI * (p[2] * x + p[3] * y));
                }
            }
    }
    s->dt_from_cells = 1;
    return FCO_OK;
}

int fco_get_fields(const fco_sim *s, double *out)
{
    memcpy(out, s->q, sizeof(double) * (size_t)s->n * s->F * patch_cells(s));
    return FCO_OK;
}

int fco_set_fields(fco_sim *s, const double *in)
{
    memcpy(s->q, in, sizeof(double) * (size_t)s->n * s->F * patch_cells(s));
    s->dt_from_cells = 1;
    return FCO_OK;
}

/* sum over cells of (cell area) * q, per field; leaves in SFC order */
int fco_conservation_sums(const fco_sim *s, double *sums)
{
    int m = s->p.m;
    for (int f = 0; f < s->F; ++f) {
        double tot = 0.0;
        for (int k = 0; k < s->n; ++k) {
            const fco_leaf *l = &s->leaves[k];
            double dx = cell_dx(s, l->level), acc = 0.0;
            const double *q = s->q + ((size_t)k * s->F + f) * m * m;
            if (is_sphere(s->p.conn)) {
                /* sum of cell area * q on the unit sphere */
                const long long N = 1LL << FCO_MAXLEVEL;
                long long w2 = 2 * ((1LL << (FCO_MAXLEVEL - l->level)) / m);
                for (int c = 0; c < m * m; ++c) {
                    long long U0 = ((long long)l->x * m + c % m) * w2 - N, V0 = ((long long)l->y * m + c / m) * w2 - N;
                    acc += map_area(s, l->tree, U0, U0 + w2, V0, V0 + w2) * q[c];
                }
                tot += acc;
                continue;
            }
            for (int c = 0; c < m * m; ++c) acc += q[c];
            tot += acc * (dx * dx);
        }
        sums[f] = tot;
    }
    return FCO_OK;
}

/* ---------------------------------------------------------------------- */
/* time view: interior values of every level at the time of a fill          */
typedef struct {
    const double *cur, *old;
    double alpha[FCO_MAXLEVEL + 1];  /* weight of the newer state per level */
} view_t;

static double vval(const fco_sim *s, const view_t *v, int k, int f, int i, int j)
{
    int m = s->p.m;
    size_t o = ((size_t)k * s->F + f) * m * m + (size_t)j * m + i;
    double a = v->alpha[s->leaves[k].level];
    if (a == 1.0) return v->cur[o];
    if (a == 0.0) return v->old[o];
    return (1.0 - a) * v->old[o] + a * v->cur[o];
}

static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return minv(a, b);
    if (a < 0.0 && b < 0.0) return maxv(a, b);
    return 0.0;
}

/* reflecting-wall ghost layers of a padded patch on the unit square */
static void fill_walls(const fco_sim *s, const fco_leaf *l, double *P)
{
    int m = s->p.m, F = s->F, side = 1 << l->level;
    size_t PP = patch_pad(s);
    if (s->p.conn != FCO_CONN_SQUARE) return;
    for (int f = 0; f < F; ++f) {
        double *A = P + f * PP;
        double sg = (s->p.equation == FCO_EQ_SWE && f == 1) ? -1.0 : 1.0;
        for (int j = -2; j < m + 2; ++j)
            for (int k = 0; k < 2; ++k) {
                if (l->x == 0) A[FCO_IDX(m, -1 - k, j)] = sg * A[FCO_IDX(m, k, j)];
                if (l->x == side - 1) A[FCO_IDX(m, m + k, j)] = sg * A[FCO_IDX(m, m - 1 - k, j)];
            }
    }
    for (int f = 0; f < F; ++f) {
        double *A = P + f * PP;
        double sg = (s->p.equation == FCO_EQ_SWE && f == 2) ? -1.0 : 1.0;
        for (int i = -2; i < m + 2; ++i)
            for (int k = 0; k < 2; ++k) {
                if (l->y == 0) A[FCO_IDX(m, i, -1 - k)] = sg * A[FCO_IDX(m, i, k)];
                if (l->y == side - 1) A[FCO_IDX(m, i, m + k)] = sg * A[FCO_IDX(m, i, m - 1 - k)];
            }
    }
}

/*
 * Fill the padded array of patch k: interior from the time view, every ghost
 * cell from the leaf that contains the ghost cell's centre.  Coarser sources
 * must already hold their complete padded arrays in pad.
 */
static int fill_patch(const fco_sim *s, const view_t *v, int k, double *pad)
{
    const fco_leaf *l = &s->leaves[k];
    int m = s->p.m, F = s->F;
    size_t PP = patch_pad(s);
    double *P = pad + (size_t)k * F * PP;
    for (size_t c = 0; c < (size_t)F * PP; ++c) P[c] = 0.0;
    for (int f = 0; f < F; ++f)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) P[f * PP + FCO_IDX(m, i, j)] = vval(s, v, k, f, i, j);
    long long w = (1LL << (FCO_MAXLEVEL - l->level)) / m;   /* finest units per cell */
    for (int j = -2; j < m + 2; ++j)
        for (int i = -2; i < m + 2; ++i) {
            if (i >= 0 && i < m && j >= 0 && j < m) continue;
            long long gi = (long long)l->x * m + i, gj = (long long)l->y * m + j;
            long long X = gi * w + w / 2, Y = gj * w + w / 2, Xm, Ym;
            int t2 = fco_map_point(s->p.conn, l->tree, X, Y, &Xm, &Ym);
            if (t2 < 0) continue;                       /* wall: filled below */
            int nb = fco_find_leaf(s, t2, Xm, Ym);
            if (nb < 0) { set_err("point location failed"); return FCO_ERR_ARG; }
            const fco_leaf *N = &s->leaves[nb];
            int dl = N->level - l->level;
            if (dl == 0) {
                int ci = (int)(Xm / w - (long long)N->x * m), cj = (int)(Ym / w - (long long)N->y * m);
                for (int f = 0; f < F; ++f) P[f * PP + FCO_IDX(m, i, j)] = vval(s, v, nb, f, ci, cj);
            } else if (dl == 1) {
                long long wf = w / 2;
                double val[3][2][2];
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        long long Xf = (2 * gi + a) * wf + wf / 2, Yf = (2 * gj + b) * wf + wf / 2, Xfm, Yfm;
                        int t3 = fco_map_point(s->p.conn, l->tree, Xf, Yf, &Xfm, &Yfm);
                        int nf = t3 < 0 ? -1 : fco_find_leaf(s, t3, Xfm, Yfm);
                        if (nf < 0 || s->leaves[nf].level != l->level + 1) return FCO_ERR_UNBALANCED;
                        int ci = (int)(Xfm / wf - (long long)s->leaves[nf].x * m);
                        int cj = (int)(Yfm / wf - (long long)s->leaves[nf].y * m);
                        for (int f = 0; f < F; ++f) val[f][b][a] = vval(s, v, nf, f, ci, cj);
                    }
                for (int f = 0; f < F; ++f)
                    P[f * PP + FCO_IDX(m, i, j)] =
                        0.25 * ((val[f][0][0] + val[f][0][1]) + (val[f][1][0] + val[f][1][1]));
            } else if (dl == -1) {
                long long wc = 2 * w;
                int ci = (int)(Xm / wc - (long long)N->x * m), cj = (int)(Ym / wc - (long long)N->y * m);
                long long cx = ((long long)N->x * m + ci) * wc + wc / 2;
                long long cy = ((long long)N->y * m + cj) * wc + wc / 2;
                double sgx = Xm > cx ? 0.25 : -0.25, sgy = Ym > cy ? 0.25 : -0.25;
                const double *C = pad + (size_t)nb * F * PP;
                for (int f = 0; f < F; ++f) {
                    const double *A = C + f * PP;
                    double qc = A[FCO_IDX(m, ci, cj)];
                    double sx = minmod(A[FCO_IDX(m, ci + 1, cj)] - qc, qc - A[FCO_IDX(m, ci - 1, cj)]);
                    double sy = minmod(A[FCO_IDX(m, ci, cj + 1)] - qc, qc - A[FCO_IDX(m, ci, cj - 1)]);
                    P[f * PP + FCO_IDX(m, i, j)] = (qc + sgx * sx) + sgy * sy;
                }
            } else return FCO_ERR_UNBALANCED;
        }
    if (s->p.conn == FCO_CONN_SPHERE) {
        /* cells beyond a cube corner (three trees meet, no fourth): average of
         * the two adjacent face-ghost values of the same row and column */
        for (int j = -2; j < m + 2; ++j)
            for (int i = -2; i < m + 2; ++i) {
                if ((i >= 0 && i < m) || (j >= 0 && j < m)) continue;
                long long gi = (long long)l->x * m + i, gj = (long long)l->y * m + j;
                long long X = gi * w + w / 2, Y = gj * w + w / 2, Xm, Ym;
                if (fco_map_point(s->p.conn, l->tree, X, Y, &Xm, &Ym) >= 0) continue;
                int ic = i < 0 ? 0 : m - 1, jc = j < 0 ? 0 : m - 1;
                for (int f = 0; f < F; ++f)
                    P[f * PP + FCO_IDX(m, i, j)] =
                        0.5 * (P[f * PP + FCO_IDX(m, i, jc)] + P[f * PP + FCO_IDX(m, ic, j)]);
            }
    }
    fill_walls(s, l, P);
    return FCO_OK;
}

/* fill every patch of level <= lmax, coarsest level first */
static int fill_levels(const fco_sim *s, const view_t *v, int lmax, double *pad)
{
    int lo = 99, hi = -1;
    for (int k = 0; k < s->n; ++k) {
        lo = s->leaves[k].level < lo ? s->leaves[k].level : lo;
        hi = s->leaves[k].level > hi ? s->leaves[k].level : hi;
    }
    if (lmax < hi) hi = lmax;
    for (int lev = lo; lev <= hi; ++lev)
        for (int k = 0; k < s->n; ++k)
            if (s->leaves[k].level == lev) {
                int rc = fill_patch(s, v, k, pad);
                if (rc) return rc;
            }
    return FCO_OK;
}

static void view_current(const fco_sim *s, view_t *v)
{
    v->cur = s->q; v->old = s->q;
    for (int l = 0; l <= FCO_MAXLEVEL; ++l) v->alpha[l] = 1.0;
}

int fco_fill_ghosts(fco_sim *s, double *out)
{
    if (s->p.conn == FCO_CONN_TABLE) { set_err("fco_fill_ghosts: a table connectivity has no fields"); return FCO_ERR_ARG; }
    view_t v;
    view_current(s, &v);
    return fill_levels(s, &v, 99, out);
}

/* ---------------------------------------------------------------------- */
/* geometry of one padded patch: capacity of every cell of the padded tile,  */
/* speeds of every x-edge (i = -1..m+1, rows j = -2..m+1) and y-edge        */
/* (j = -1..m+1, columns i = -2..m+1), and which patch corners are cube      */
/* corners.  On the square: capacity 1, the constant advection velocity.     */
typedef struct {
    double *kap, *sx, *sy;
    int cube_corner;      /* bit 0 SW, 1 SE, 2 NW, 3 NE */
} geom_t;

#define GK(g, m, i, j) (g)->kap[((j) + 2) * ((m) + 4) + ((i) + 2)]
#define GSX(g, m, i, j) (g)->sx[((j) + 2) * ((m) + 3) + ((i) + 1)]
#define GSY(g, m, i, j) (g)->sy[((j) + 1) * ((m) + 4) + ((i) + 2)]


static void geom_alloc(int m, geom_t *g)
{
    g->kap = (double *)malloc(sizeof(double) * (size_t)(m + 4) * (m + 4));
    g->sx = (double *)malloc(sizeof(double) * (size_t)(m + 4) * (m + 3));
    g->sy = (double *)malloc(sizeof(double) * (size_t)(m + 3) * (m + 4));
    g->cube_corner = 0;
}

static void geom_free(geom_t *g) { free(g->kap); free(g->sx); free(g->sy); }

/* stream function of the swirl on the square (R27; the paper's Example 1
 * prescribes a distorting flow without giving it) */
static double swirl_psi(const fco_sim *s, double x, double y)
{
    const double sx = sin(M_PI * x), sy = sin(M_PI * y);
    return s->p.adv_u * ((sx * sx) * (sy * sy)) / M_PI;
}

static void geom_build(const fco_sim *s, const fco_leaf *l, geom_t *g)
{
    int m = s->p.m;
    g->cube_corner = 0;
    if (!is_sphere(s->p.conn)) {
        for (int k = 0; k < (m + 4) * (m + 4); ++k) g->kap[k] = 1.0;
        if (s->p.velocity != FCO_VEL_SWIRL) {
            for (int k = 0; k < (m + 4) * (m + 3); ++k) { g->sx[k] = s->p.adv_u; g->sy[k] = s->p.adv_v; }
            return;
        }
        /* swirl (R27): normal velocity of an edge = difference of the stream
         * function between its ends over the edge length, so that every
         * cell's edge fluxes sum to zero */
        const double dx = cell_dx(s, l->level);
        const long long i0 = (long long)l->x * m, j0 = (long long)l->y * m;
        for (int j = -2; j < m + 2; ++j)
            for (int i = -1; i <= m + 1; ++i) {          /* u = (psi(top) - psi(bottom)) / dy */
                double x = (double)(i0 + i) * dx, y0 = (double)(j0 + j) * dx, y1 = (double)(j0 + j + 1) * dx;
                GSX(g, m, i, j) = (swirl_psi(s, x, y1) - swirl_psi(s, x, y0)) / dx;
            }
        for (int j = -1; j <= m + 1; ++j)
            for (int i = -2; i < m + 2; ++i) {          /* v = (psi(left) - psi(right)) / dx */
                double y = (double)(j0 + j) * dx, x0 = (double)(i0 + i) * dx, x1 = (double)(i0 + i + 1) * dx;
                GSY(g, m, i, j) = (swirl_psi(s, x0, y) - swirl_psi(s, x1, y)) / dx;
            }
        return;
    }
    const long long N = 1LL << FCO_MAXLEVEL;
    long long w2 = 2 * ((1LL << (FCO_MAXLEVEL - l->level)) / m);      /* doubled units per cell */
    double dxi = 1.0 / ((double)(1 << l->level) * m);
    long long Ub = (long long)l->x * m * w2 - N, Vb = (long long)l->y * m * w2 - N;
    for (int j = -2; j < m + 2; ++j)
        for (int i = -2; i < m + 2; ++i) {
            long long U0 = Ub + i * w2, V0 = Vb + j * w2;
            GK(g, m, i, j) = map_area(s, l->tree, U0, U0 + w2, V0, V0 + w2) / (dxi * dxi);
        }
    double pa[3], pb[3];
    for (int j = -2; j < m + 2; ++j)
        for (int i = -1; i <= m + 1; ++i) {          /* flux toward +xi: psi(top) - psi(bottom) */
            long long U = Ub + i * w2, V0 = Vb + j * w2;
            map_point(s, l->tree, U, V0, pa);
            map_point(s, l->tree, U, V0 + w2, pb);
            GSX(g, m, i, j) = (fco_sphere_psi(&s->p, pb) - fco_sphere_psi(&s->p, pa)) / dxi;
        }
    for (int j = -1; j <= m + 1; ++j)
        for (int i = -2; i < m + 2; ++i) {          /* flux toward +eta: psi(left) - psi(right) */
            long long U0 = Ub + i * w2, V = Vb + j * w2;
            map_point(s, l->tree, U0, V, pa);
            map_point(s, l->tree, U0 + w2, V, pb);
            GSY(g, m, i, j) = (fco_sphere_psi(&s->p, pa) - fco_sphere_psi(&s->p, pb)) / dxi;
        }
    int last = (1 << l->level) - 1;
    if (l->x == 0 && l->y == 0) g->cube_corner |= 1;
    if (l->x == last && l->y == 0) g->cube_corner |= 2;
    if (l->x == 0 && l->y == last) g->cube_corner |= 4;
    if (l->x == last && l->y == last) g->cube_corner |= 8;
}

/* is x-edge (i, j) / y-edge (i, j) a patch-boundary edge ending at a cube corner */
static int xedge_at_cube_corner(const geom_t *g, int m, int i, int j)
{
    return ((g->cube_corner & 1) && i == 0 && j == 0) || ((g->cube_corner & 2) && i == m && j == 0) ||
           ((g->cube_corner & 4) && i == 0 && j == m - 1) || ((g->cube_corner & 8) && i == m && j == m - 1);
}
static int yedge_at_cube_corner(const geom_t *g, int m, int i, int j)
{
    return ((g->cube_corner & 1) && i == 0 && j == 0) || ((g->cube_corner & 2) && i == m - 1 && j == 0) ||
           ((g->cube_corner & 4) && i == 0 && j == m) || ((g->cube_corner & 8) && i == m - 1 && j == m);
}

/* ---------------------------------------------------------------------- */
/* wave-propagation update of one padded patch (capacity form)              */
typedef struct {
    double dx, dy, dt;
    double smax;           /* largest |s| / capacity over edges touching the interior */
    double *reg;           /* [4][m][F] effective side flux * dt, or NULL  */
    const geom_t *geo;
} upd_t;

/* limited second-order correction of an edge, summed over its waves:
 * |s| (1 - dt / (kappa_up dx) |s|) phi W, with theta = (W_up . W) / (W . W)
 * (the upwind edge eL for s >= 0, else eR; kappa_up the capacity of the
 * upwind cell).  The correction flux is half of it. */
static void edge_correction(const fco_edge *e, const fco_edge *eL, const fco_edge *eR, double kapL, double kapR,
                            double dt, double dx, int F, double *acc)
{
    for (int f = 0; f < 3; ++f) acc[f] = 0.0;
    for (int p = 0; p < e->nw; ++p) {
        int left = e->s[p] >= 0.0;
        const fco_edge *eu = left ? eL : eR;
        double ww = 0.0, wu = 0.0;
        for (int f = 0; f < F; ++f) { ww += e->W[p][f] * e->W[p][f]; wu += eu->W[p][f] * e->W[p][f]; }
        double phi = ww == 0.0 ? 0.0 : fco_mc_limiter(wu / ww);
        double dtdx = dt / ((left ? kapL : kapR) * dx);
        double as = fabs(e->s[p]), c = as * (1.0 - dtdx * as);
        for (int f = 0; f < F; ++f) acc[f] += c * (phi * e->W[p][f]);
    }
}

static int patch_update(const fco_sim *s, const double *P, double *qout, upd_t *u)
{
    const int m = s->p.m, F = s->F, swe = s->p.equation == FCO_EQ_SWE;
    const size_t PP = patch_pad(s);
    const geom_t *geo = u->geo;
    const int nxr = m + 2, nxc = m + 3;      /* x-edges: rows -1..m, edges -1..m+1 */
    const int nyr = m + 3, nyc = m + 2;      /* y-edges: rows -1..m+1, cols -1..m  */
    fco_edge *ex = (fco_edge *)malloc(sizeof(fco_edge) * (size_t)nxr * nxc);
    fco_edge *ey = (fco_edge *)malloc(sizeof(fco_edge) * (size_t)nyr * nyc);
    double *Ft = (double *)calloc((size_t)m * (m + 1) * 3, sizeof(double)); /* [j][i] i=0..m */
    double *Gt = (double *)calloc((size_t)(m + 1) * m * 3, sizeof(double)); /* [j][i] j=0..m */
#define EX(i, j) ex[((j) + 1) * nxc + ((i) + 1)]
#define EY(i, j) ey[((j) + 1) * nyc + ((i) + 1)]
#define QP(f, i, j) P[(f) * PP + FCO_IDX(m, i, j)]
#define FT(i, j) (Ft + (((size_t)(j) * (m + 1) + (i)) * 3))
#define GT(i, j) (Gt + (((size_t)(j) * m + (i)) * 3))
#define KAP(i, j) GK(geo, m, i, j)
    int rc = FCO_OK;
    if (swe)
        for (int j = -2; j < m + 2 && !rc; ++j)
            for (int i = -2; i < m + 2; ++i)
                if (!(QP(0, i, j) > 0.0)) { rc = FCO_ERR_DRY; break; }
    if (rc) goto done;
    /* Riemann problems: x-edge (i, j) between cells (i-1, j) and (i, j) */
    for (int j = -1; j <= m; ++j)
        for (int i = -1; i <= m + 1; ++i) {
            double qL[3], qR[3];
            for (int f = 0; f < F; ++f) { qL[f] = QP(f, i - 1, j); qR[f] = QP(f, i, j); }
            if (swe) fco_riemann_swe(0, qL, qR, s->p.g, &EX(i, j));
            else fco_riemann_adv(GSX(geo, m, i, j), qL, qR, &EX(i, j));
            if (swe && s->p.entropy_fix) fco_entropy_fix_swe(0, qL, qR, s->p.g, &EX(i, j));
        }
    /* y-edge (i, j) between cells (i, j-1) and (i, j) */
    for (int j = -1; j <= m + 1; ++j)
        for (int i = -1; i <= m; ++i) {
            double qL[3], qR[3];
            for (int f = 0; f < F; ++f) { qL[f] = QP(f, i, j - 1); qR[f] = QP(f, i, j); }
            if (swe) fco_riemann_swe(1, qL, qR, s->p.g, &EY(i, j));
            else fco_riemann_adv(GSY(geo, m, i, j), qL, qR, &EY(i, j));
            if (swe && s->p.entropy_fix) fco_entropy_fix_swe(1, qL, qR, s->p.g, &EY(i, j));
        }
    /* CFL: edges that touch an interior cell, speed over the smaller capacity */
    u->smax = 0.0;
    for (int j = 0; j < m; ++j)
        for (int i = 0; i <= m; ++i) {
            double kmin = minv(KAP(i - 1, j), KAP(i, j));
            for (int p = 0; p < EX(i, j).nw; ++p) u->smax = maxv(u->smax, fabs(EX(i, j).s[p]) / kmin);
        }
    for (int j = 0; j <= m; ++j)
        for (int i = 0; i < m; ++i) {
            double kmin = minv(KAP(i, j - 1), KAP(i, j));
            for (int p = 0; p < EY(i, j).nw; ++p) u->smax = maxv(u->smax, fabs(EY(i, j).s[p]) / kmin);
        }

    const double dt = u->dt;
    /* own MC-limited correction fluxes; the upwind cell's capacity scales the
     * Courant factor */
    for (int j = 0; j < m; ++j)
        for (int i = 0; i <= m; ++i) {
            double acc[3];
            edge_correction(&EX(i, j), &EX(i - 1, j), &EX(i + 1, j), KAP(i - 1, j), KAP(i, j), dt, u->dx, F, acc);
            for (int f = 0; f < F; ++f) FT(i, j)[f] = 0.5 * acc[f];
        }
    for (int j = 0; j <= m; ++j)
        for (int i = 0; i < m; ++i) {
            double acc[3];
            edge_correction(&EY(i, j), &EY(i, j - 1), &EY(i, j + 1), KAP(i, j - 1), KAP(i, j), dt, u->dy, F, acc);
            for (int f = 0; f < F; ++f) GT(i, j)[f] = 0.5 * acc[f];
        }
    /* T2: the full limited corrections of every edge whose fluctuations are
     * split transversely (x-edges i = 0..m, rows -1..m; y-edges i = -1..m,
     * rows 0..m) */
    const int t2 = s->p.transverse == 2;
    double *cqx = NULL, *cqy = NULL;
#define CQX(i, j) (cqx + (((size_t)((j) + 1) * (m + 1) + (i)) * 3))
#define CQY(i, j) (cqy + (((size_t)(j) * (m + 2) + ((i) + 1)) * 3))
    if (t2) {
        cqx = (double *)calloc((size_t)(m + 2) * (m + 1) * 3, sizeof(double));
        cqy = (double *)calloc((size_t)(m + 1) * (m + 2) * 3, sizeof(double));
        for (int j = -1; j <= m; ++j)
            for (int i = 0; i <= m; ++i)
                edge_correction(&EX(i, j), &EX(i - 1, j), &EX(i + 1, j), KAP(i - 1, j), KAP(i, j), dt, u->dx, F,
                                CQX(i, j));
        for (int j = 0; j <= m; ++j)
            for (int i = -1; i <= m; ++i)
                edge_correction(&EY(i, j), &EY(i, j - 1), &EY(i, j + 1), KAP(i, j - 1), KAP(i, j), dt, u->dy, F,
                                CQY(i, j));
    }
    /* transverse propagation of the normal fluctuations; the factor is half
     * dt / (capacity dx) of the cell the fluctuation enters.  Edges of the
     * patch boundary that end at a cube corner receive none. */
    {
        /* into F~ at x-edge (i, j) from y-edges: below-left (i-1, j) up-going,
         * below-right (i, j) up-going, above-left (i-1, j+1) down-going,
         * above-right (i, j+1) down-going; the part moving toward +x from the
         * left column, toward -x from the right column. */
        for (int j = 0; j < m; ++j)
            for (int i = 0; i <= m; ++i) {
                if (xedge_at_cube_corner(geo, m, i, j)) continue;
                double *Fe = FT(i, j);
                const fco_edge *src[4] = {&EY(i - 1, j), &EY(i, j), &EY(i - 1, j + 1), &EY(i, j + 1)};
                const int up[4] = {1, 1, 0, 0}, right[4] = {1, 0, 1, 0};
                const int si[4] = {i - 1, i, i - 1, i}, sj[4] = {j, j, j + 1, j + 1};
                for (int q = 0; q < 4; ++q) {
                    const fco_edge *e = src[q];
                    const double *d = up[q] ? e->apdq : e->amdq;
                    double d2[3];
                    if (t2) {         /* fluctuation with the correction wave: A+dQ - cq, A-dQ + cq */
                        const double *cq = CQY(si[q], sj[q]);
                        for (int f = 0; f < F; ++f) d2[f] = up[q] ? d[f] - cq[f] : d[f] + cq[f];
                        d = d2;
                    }
                    int ci = right[q] ? i - 1 : i;       /* cell the fluctuation enters */
                    double bm[3], bp[3];
                    if (swe) fco_transverse_swe(1, e, d, bm, bp);
                    else {
                        double sxe = GSX(geo, m, i, j);  /* the edge it crosses */
                        bp[0] = maxv(sxe, 0.0) * d[0];
                        bm[0] = minv(sxe, 0.0) * d[0];
                    }
                    const double *part = right[q] ? bp : bm;
                    double ky = 0.5 * (dt / (KAP(ci, j) * u->dy));
                    for (int f = 0; f < F; ++f) Fe[f] -= ky * part[f];
                }
            }
        /* into G~ at y-edge (i, j) from x-edges: below-left (i, j-1) right-going,
         * below-right (i+1, j-1) left-going, above-left (i, j) right-going,
         * above-right (i+1, j) left-going; up part from the row below, down
         * part from the row above. */
        for (int j = 0; j <= m; ++j)
            for (int i = 0; i < m; ++i) {
                if (yedge_at_cube_corner(geo, m, i, j)) continue;
                double *Ge = GT(i, j);
                const fco_edge *src[4] = {&EX(i, j - 1), &EX(i + 1, j - 1), &EX(i, j), &EX(i + 1, j)};
                const int rgo[4] = {1, 0, 1, 0}, upw[4] = {1, 1, 0, 0};
                const int si[4] = {i, i + 1, i, i + 1}, sj[4] = {j - 1, j - 1, j, j};
                for (int q = 0; q < 4; ++q) {
                    const fco_edge *e = src[q];
                    const double *d = rgo[q] ? e->apdq : e->amdq;
                    double d2[3];
                    if (t2) {
                        const double *cq = CQX(si[q], sj[q]);
                        for (int f = 0; f < F; ++f) d2[f] = rgo[q] ? d[f] - cq[f] : d[f] + cq[f];
                        d = d2;
                    }
                    int cj = upw[q] ? j - 1 : j;         /* cell the fluctuation enters */
                    double bm[3], bp[3];
                    if (swe) fco_transverse_swe(0, e, d, bm, bp);
                    else {
                        double sye = GSY(geo, m, i, j);
                        bp[0] = maxv(sye, 0.0) * d[0];
                        bm[0] = minv(sye, 0.0) * d[0];
                    }
                    const double *part = upw[q] ? bp : bm;
                    double kx = 0.5 * (dt / (KAP(i, cj) * u->dx));
                    for (int f = 0; f < F; ++f) Ge[f] -= kx * part[f];
                }
            }
    }
    /* conservative update (capacity form) */
    for (int f = 0; f < F; ++f)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                double X = (EX(i, j).apdq[f] + EX(i + 1, j).amdq[f]) + (FT(i + 1, j)[f] - FT(i, j)[f]);
                double Y = (EY(i, j).apdq[f] + EY(i, j + 1).amdq[f]) + (GT(i, j + 1)[f] - GT(i, j)[f]);
                double dtdx = dt / (KAP(i, j) * u->dx), dtdy = dt / (KAP(i, j) * u->dy);
                qout[((size_t)f * m + j) * m + i] = (QP(f, i, j) - dtdx * X) - dtdy * Y;
            }
    /* effective fluxes through the four sides, times dt */
    if (u->reg) {
        for (int c = 0; c < m; ++c) {
            double qc[3], fl[3];
            double *r;
            /* -x side: cell (0, c), edge (0, c) */
            for (int f = 0; f < F; ++f) qc[f] = QP(f, 0, c);
            if (swe) fco_flux_swe(0, qc, s->p.g, fl); else fl[0] = GSX(geo, m, 0, c) * qc[0];
            r = u->reg + ((size_t)0 * m + c) * F;
            for (int f = 0; f < F; ++f) r[f] = u->dt * ((fl[f] - EX(0, c).apdq[f]) + FT(0, c)[f]);
            /* +x side: cell (m-1, c), edge (m, c) */
            for (int f = 0; f < F; ++f) qc[f] = QP(f, m - 1, c);
            if (swe) fco_flux_swe(0, qc, s->p.g, fl); else fl[0] = GSX(geo, m, m, c) * qc[0];
            r = u->reg + ((size_t)1 * m + c) * F;
            for (int f = 0; f < F; ++f) r[f] = u->dt * ((fl[f] + EX(m, c).amdq[f]) + FT(m, c)[f]);
            /* -y side: cell (c, 0), edge (c, 0) */
            for (int f = 0; f < F; ++f) qc[f] = QP(f, c, 0);
            if (swe) fco_flux_swe(1, qc, s->p.g, fl); else fl[0] = GSY(geo, m, c, 0) * qc[0];
            r = u->reg + ((size_t)2 * m + c) * F;
            for (int f = 0; f < F; ++f) r[f] = u->dt * ((fl[f] - EY(c, 0).apdq[f]) + GT(c, 0)[f]);
            /* +y side: cell (c, m-1), edge (c, m) */
            for (int f = 0; f < F; ++f) qc[f] = QP(f, c, m - 1);
            if (swe) fco_flux_swe(1, qc, s->p.g, fl); else fl[0] = GSY(geo, m, c, m) * qc[0];
            r = u->reg + ((size_t)3 * m + c) * F;
            for (int f = 0; f < F; ++f) r[f] = u->dt * ((fl[f] + EY(c, m).amdq[f]) + GT(c, m)[f]);
        }
    }
#undef EX
#undef EY
#undef QP
#undef FT
#undef GT
#undef KAP
#undef CQX
#undef CQY
    free(cqx); free(cqy);
done:
    free(ex); free(ey); free(Ft); free(Gt);
    return rc;
}

int fco_patch_step(int equation, int m, double g, double dx, double dy, double dt,
                   double adv_u, double adv_v, const double *qpad, double *qout, double *smax)
{
    fco_sim s;
    memset(&s, 0, sizeof s);
    s.p.m = m; s.p.equation = equation; s.p.g = g; s.p.adv_u = adv_u; s.p.adv_v = adv_v;
    s.F = equation == FCO_EQ_SWE ? 3 : 1;
    geom_t geo;
    geom_alloc(m, &geo);
    fco_leaf l0 = {0, 0, 0, 0};
    geom_build(&s, &l0, &geo);
    upd_t u = {dx, dy, dt, 0.0, NULL, &geo};
    int rc = patch_update(&s, qpad, qout, &u);
    geom_free(&geo);
    if (smax) *smax = u.smax;
    return rc;
}

/* ---------------------------------------------------------------------- */
/* coarse-fine correction of coarse boundary cells                          */
/* reg: [n][4][m][F].  Coarse side values = dt_c * F_c, fine side values    */
/* = sum over its substeps of dt_f * F_f.                                    */
/* cubed sphere: fine cells across coarse boundary cell c of side `side` are
 * found by locating their centres; the fine side is the one whose coarser
 * neighbour is patch k; fluxes are compared as outward from the coarse cell */
static void reflux_patch_sphere(const fco_sim *s, const int32_t *nbr, int k, const double *reg, double *q)
{
    int m = s->p.m, F = s->F;
    const fco_leaf *l = &s->leaves[k];
    double dx = cell_dx(s, l->level);
    long long wc = (1LL << (FCO_MAXLEVEL - l->level)) / m, wf = wc / 2;
    geom_t g;
    geom_alloc(m, &g);
    geom_build(s, l, &g);
    for (int side = 0; side < 4; ++side) {
        if (nbr[((size_t)k * 8 + side) * 4] != FCO_NB_FINER) continue;
        double sgc = (side & 1) ? 1.0 : -1.0;
        for (int c = 0; c < m; ++c) {
            int ci = side == 0 ? 0 : (side == 1 ? m - 1 : c);
            int cj = side == 2 ? 0 : (side == 3 ? m - 1 : c);
            long long X0 = ((long long)l->x * m + ci) * wc, Y0 = ((long long)l->y * m + cj) * wc;
            double rin[3] = {0.0, 0.0, 0.0};
            for (int q2 = 0; q2 < 2; ++q2) {
                long long X, Y;
                long long a = q2 == 0 ? wf / 2 : wf + wf / 2;
                if (side == 0) { X = X0 - wf / 2; Y = Y0 + a; }
                else if (side == 1) { X = X0 + wc + wf / 2; Y = Y0 + a; }
                else if (side == 2) { X = X0 + a; Y = Y0 - wf / 2; }
                else { X = X0 + a; Y = Y0 + wc + wf / 2; }
                long long Xm, Ym;
                int t2 = fco_map_point(s->p.conn, l->tree, X, Y, &Xm, &Ym);
                int nf = fco_find_leaf(s, t2, Xm, Ym);
                const fco_leaf *L = &s->leaves[nf];
                int fi = (int)(Xm / wf - (long long)L->x * m), fj = (int)(Ym / wf - (long long)L->y * m);
                /* the fine leaf's side facing this coarse side: the one whose
                 * outward normal is opposite to the image of this side's
                 * outward normal (on the two-tree sphere a fine corner patch
                 * faces the same coarse patch across two of its sides) */
                long long Xn = X + (side == 0 ? -1 : side == 1 ? 1 : 0), Yn = Y + (side == 2 ? -1 : side == 3 ? 1 : 0);
                long long Xnm, Ynm;
                fco_map_point(s->p.conn, l->tree, Xn, Yn, &Xnm, &Ynm);
                long long ddx = Xnm - Xm, ddy = Ynm - Ym;
                int sf = ddx > 0 ? 0 : ddx < 0 ? 1 : ddy > 0 ? 2 : 3;
                int along = sf < 2 ? fj : fi;
                double sgf = (sf & 1) ? -1.0 : 1.0;        /* inward through side sf */
                const double *rf = reg + (((size_t)nf * 4 + sf) * m + along) * F;
                for (int f = 0; f < F; ++f) rin[f] += sgf * rf[f];
            }
            const double *rc = reg + (((size_t)k * 4 + side) * m + c) * F;
            for (int f = 0; f < F; ++f) {
                double corr = (sgc * rc[f] - 0.5 * rin[f]) / (GK(&g, m, ci, cj) * dx);
                q[((size_t)k * F + f) * m * m + (size_t)cj * m + ci] += corr;
            }
        }
    }
    geom_free(&g);
}

static void reflux_patch(const fco_sim *s, const int32_t *nbr, int k, const double *reg, double *q)
{
    if (is_sphere(s->p.conn)) { reflux_patch_sphere(s, nbr, k, reg, q); return; }
    int m = s->p.m, F = s->F, h = m / 2;
    double dx = cell_dx(s, s->leaves[k].level);
    for (int side = 0; side < 4; ++side) {
        const int32_t *e = nbr + ((size_t)k * 8 + side) * 4;
        if (e[0] != FCO_NB_FINER) continue;
        int opp = side ^ 1;
        double sg = (side & 1) ? 1.0 : -1.0;   /* + side: (Rc - Rf), - side: (Rf - Rc) */
        for (int c = 0; c < m; ++c) {
            int fine = c < h ? e[1] : e[2];
            int kf = 2 * (c % h);
            const double *rc = reg + (((size_t)k * 4 + side) * m + c) * F;
            const double *r0 = reg + (((size_t)fine * 4 + opp) * m + kf) * F;
            const double *r1 = reg + (((size_t)fine * 4 + opp) * m + kf + 1) * F;
            int ci = side == 0 ? 0 : (side == 1 ? m - 1 : c);
            int cj = side == 2 ? 0 : (side == 3 ? m - 1 : c);
            for (int f = 0; f < F; ++f) {
                double corr = (rc[f] - 0.5 * (r0[f] + r1[f])) / dx;
                q[((size_t)k * F + f) * m * m + (size_t)cj * m + ci] += sg * corr;
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* time stepping                                                            */
static void level_range(const fco_sim *s, int *lo, int *hi)
{
    *lo = 99; *hi = -1;
    for (int k = 0; k < s->n; ++k) {
        if (s->leaves[k].level < *lo) *lo = s->leaves[k].level;
        if (s->leaves[k].level > *hi) *hi = s->leaves[k].level;
    }
}

/* R10 first-step rule: largest characteristic speed over cells, per level */
static double cell_rate(const fco_sim *s)
{
    int m = s->p.m, lo, hi;
    level_range(s, &lo, &hi);
    double rate = 0.0;
    for (int k = 0; k < s->n; ++k) {
        int lev = s->leaves[k].level;
        double cmax = 0.0;
        const double *q = s->q + (size_t)k * s->F * m * m;
        if (is_sphere(s->p.conn) || (s->p.equation == FCO_EQ_ADV && s->p.velocity == FCO_VEL_SWIRL)) {
            /* advection speeds of the edges touching the interior over the
             * smaller adjacent capacity */
            geom_t g;
            geom_alloc(m, &g);
            geom_build(s, &s->leaves[k], &g);
            for (int j = 0; j < m; ++j)
                for (int i = 0; i <= m; ++i) {
                    cmax = maxv(cmax, fabs(GSX(&g, m, i, j)) / minv(GK(&g, m, i - 1, j), GK(&g, m, i, j)));
                    cmax = maxv(cmax, fabs(GSY(&g, m, j, i)) / minv(GK(&g, m, j, i - 1), GK(&g, m, j, i)));
                }
            geom_free(&g);
        } else
        for (int c = 0; c < m * m; ++c) {
            double sp;
            if (s->p.equation == FCO_EQ_SWE) {
                double h = q[c], u = q[m * m + c] / h, v = q[2 * m * m + c] / h, cc = sqrt(s->p.g * h);
                sp = maxv(fabs(u) + cc, fabs(v) + cc);
            } else sp = maxv(fabs(s->p.adv_u), fabs(s->p.adv_v));
            cmax = maxv(cmax, sp);
        }
        double r = cmax / cell_dx(s, s->p.subcycle ? lo : lev);
        rate = maxv(rate, r);
    }
    return rate;
}

typedef struct {
    int lo, hi;
    long long tick_old[FCO_MAXLEVEL + 1], tick_new[FCO_MAXLEVEL + 1];
    double *qold, *pad, *reg;
    int32_t *nbr;
    double dtc;
    double smax_lev[FCO_MAXLEVEL + 1];
} step_t;

static void sub_view(const fco_sim *s, const step_t *st, long long T, view_t *v)
{
    v->cur = s->q; v->old = st->qold;
    for (int l = 0; l <= FCO_MAXLEVEL; ++l) {
        long long a = st->tick_old[l], b = st->tick_new[l];
        v->alpha[l] = (b == a) ? 1.0 : (double)(T - a) / (double)(b - a);
    }
}

/* update all patches of level lev (or every level if lev < 0) with step dt */
static int update_patches(fco_sim *s, step_t *st, int lev, double dt)
{
    int m = s->p.m, F = s->F;
    size_t PP = patch_pad(s), pc = (size_t)F * m * m;
    double *tmp = (double *)malloc(sizeof(double) * pc);
    for (int k = 0; k < s->n; ++k) {
        int l = s->leaves[k].level;
        if (lev >= 0 && l != lev) continue;
        double dx = cell_dx(s, l);
        double regk[4 * 64 * 3];
        geom_t g;
        geom_alloc(m, &g);
        geom_build(s, &s->leaves[k], &g);
        upd_t u = {dx, dx, dt, 0.0, regk, &g};
        int rc = patch_update(s, st->pad + (size_t)k * F * PP, tmp, &u);
        geom_free(&g);
        if (rc) { free(tmp); set_err("dry state (h <= 0)"); return rc; }
        for (size_t c = 0; c < pc; ++c)
            if (!isfinite(tmp[c])) { free(tmp); set_err("non-finite state"); return FCO_ERR_NONFINITE; }
        memcpy(s->q + (size_t)k * pc, tmp, sizeof(double) * pc);
        /* registers: sides facing a finer neighbour are set, sides facing a
         * coarser neighbour accumulate over the patch's substeps */
        for (int side = 0; side < 4; ++side) {
            int kind = st->nbr[((size_t)k * 8 + side) * 4];
            double *r = st->reg + ((size_t)k * 4 + side) * m * F;
            for (int c = 0; c < m * F; ++c) {
                if (kind == FCO_NB_FINER) r[c] = regk[side * m * F + c];
                else if (kind == FCO_NB_COARSER) r[c] += regk[side * m * F + c];
            }
        }
        st->smax_lev[l] = maxv(st->smax_lev[l], u.smax);
        s->cell_updates += (int64_t)m * m;
    }
    free(tmp);
    return FCO_OK;
}

static void zero_fine_registers(const fco_sim *s, step_t *st, int lev)
{
    int m = s->p.m, F = s->F;
    for (int k = 0; k < s->n; ++k) {
        if (lev >= 0 && s->leaves[k].level != lev) continue;
        for (int side = 0; side < 4; ++side)
            if (st->nbr[((size_t)k * 8 + side) * 4] == FCO_NB_COARSER)
                memset(st->reg + ((size_t)k * 4 + side) * m * F, 0, sizeof(double) * m * F);
    }
}

static int advance_level(fco_sim *s, step_t *st, int lev)
{
    int m = s->p.m, F = s->F;
    size_t pc = (size_t)F * m * m;
    double dt = st->dtc / (double)(1LL << (lev - st->lo));
    long long T = st->tick_new[lev], ticks = 1LL << (st->hi - lev);
    if (s->hook && s->hook(s->hook_ctx, lev, s->q, st->qold, s->n)) { set_err("substep hook failed"); return FCO_ERR_ARG; }
    view_t v;
    sub_view(s, st, T, &v);
    int rc = fill_levels(s, &v, lev, st->pad);
    if (rc) return rc;
    for (int k = 0; k < s->n; ++k)
        if (s->leaves[k].level == lev) memcpy(st->qold + k * pc, s->q + k * pc, sizeof(double) * pc);
    st->tick_old[lev] = T;
    st->tick_new[lev] = T + ticks;
    rc = update_patches(s, st, lev, dt);
    if (rc) return rc;
    if (lev < st->hi) {
        zero_fine_registers(s, st, lev + 1);
        if ((rc = advance_level(s, st, lev + 1))) return rc;
        if ((rc = advance_level(s, st, lev + 1))) return rc;
        if (s->p.refluxing)
            for (int k = 0; k < s->n; ++k)
                if (s->leaves[k].level == lev) reflux_patch(s, st->nbr, k, st->reg, s->q);
    }
    return FCO_OK;
}

/* one (coarse) step with step size dt; returns the Courant number */
static int one_step(fco_sim *s, step_t *st, double dt, double *courant, double *rate_out)
{
    int rc;
    st->dtc = dt;
    for (int l = 0; l <= FCO_MAXLEVEL; ++l) { st->tick_old[l] = st->tick_new[l] = 0; st->smax_lev[l] = 0.0; }
    if (s->p.subcycle) {
        rc = advance_level(s, st, st->lo);
    } else {
        view_t v;
        view_current(s, &v);
        if (s->hook && s->hook(s->hook_ctx, -1, s->q, s->q, s->n)) { set_err("substep hook failed"); return FCO_ERR_ARG; }
        rc = fill_levels(s, &v, 99, st->pad);
        if (!rc) {
            zero_fine_registers(s, st, -1);
            rc = update_patches(s, st, -1, dt);
        }
        if (!rc && s->p.refluxing)
            for (int k = 0; k < s->n; ++k) reflux_patch(s, st->nbr, k, st->reg, s->q);
    }
    if (rc) return rc;
    /* Courant number: global dt -> dt * max_l smax_l / dx_l; sub-cycling ->
     * max_l dt_l smax_l / dx_l = dt * max_l smax_l / dx_lmin */
    double rate = 0.0;
    for (int l = st->lo; l <= st->hi; ++l)
        rate = maxv(rate, st->smax_lev[l] / cell_dx(s, s->p.subcycle ? st->lo : l));
    *courant = dt * rate;
    *rate_out = rate;
    return FCO_OK;
}

/*
 * R10: the step size comes from the previous step's wave speeds
 * (dt = cfl / rate), or from cell speeds after initialisation or regrid.  A
 * step whose Courant number exceeds 1 is undone and retaken with
 * dt <- 0.9 dt cfl / nu, at most three times.
 */
void fco_set_substep_hook(fco_sim *s, fco_substep_hook hook, void *ctx)
{
    s->hook = hook;
    s->hook_ctx = ctx;
}

int fco_advance(fco_sim *s, double dt_fixed, int nsteps, double *t_out, double *dt_out)
{
    if (s->p.conn == FCO_CONN_TABLE) { set_err("fco_advance: a table connectivity has no fields"); return FCO_ERR_ARG; }
    int m = s->p.m, F = s->F;
    size_t PP = patch_pad(s), pc = (size_t)F * m * m;
    step_t st;
    memset(&st, 0, sizeof st);
    level_range(s, &st.lo, &st.hi);
    st.pad = (double *)malloc(sizeof(double) * (size_t)s->n * F * PP);
    st.qold = (double *)malloc(sizeof(double) * (size_t)s->n * pc);
    st.reg = (double *)calloc((size_t)s->n * 4 * m * F, sizeof(double));
    st.nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->n * 32);
    double *save = (double *)malloc(sizeof(double) * (size_t)s->n * pc);
    int rc = fco_build_neighbors(s, st.nbr);
    double dt = 0.0;
    int64_t cu0 = 0;
    for (int step = 0; step < nsteps && !rc; ++step) {
        if (dt_fixed > 0.0) dt = dt_fixed;
        else {
            if (s->dt_from_cells || !(s->dt_next > 0.0)) s->dt_next = s->p.cfl / cell_rate(s);
            dt = s->dt_next;
        }
        memcpy(save, s->q, sizeof(double) * (size_t)s->n * pc);
        cu0 = s->cell_updates;
        double nu = 0.0, rate = 0.0;
        for (int attempt = 0;; ++attempt) {
            rc = one_step(s, &st, dt, &nu, &rate);
            if (rc || nu <= 1.0 || dt_fixed > 0.0 || attempt == 3) break;
            memcpy(s->q, save, sizeof(double) * (size_t)s->n * pc);
            s->cell_updates = cu0;
            dt = 0.9 * dt * (s->p.cfl / nu);
        }
        if (rc) break;
        s->last_courant = nu;
        if (rate > 0.0) s->dt_next = s->p.cfl / rate;
        s->dt_from_cells = 0;
        s->t += dt;
        if (nu > 1.0) { set_err("Courant number above 1"); rc = FCO_ERR_CFL; }
    }
    free(st.pad); free(st.qold); free(st.reg); free(st.nbr); free(save);
    if (t_out) *t_out = s->t;
    if (dt_out) *dt_out = dt;
    return rc;
}

double fco_time(const fco_sim *s) { return s->t; }
double fco_next_dt(const fco_sim *s) { return s->dt_from_cells ? s->p.cfl / cell_rate(s) : s->dt_next; }
double fco_last_courant(const fco_sim *s) { return s->last_courant; }
int64_t fco_cell_updates(const fco_sim *s) { return s->cell_updates; }

/* ---------------------------------------------------------------------- */
/* tagging (Sec. 5): refine a patch if its criterion exceeds the threshold; */
/* flag a family of four for coarsening if their averaged parent would not  */
/* be refined.                                                              */
static double crit_padded(const fco_sim *s, const double *A, int lo, int hi)
{
    int m = s->p.m;
    double c = 0.0;
    if (s->p.tag_crit == FCO_TAG_GRAD) {
        for (int j = lo; j < hi; ++j)
            for (int i = lo; i < hi; ++i) {
                double gx = (A[FCO_IDX(m, i + 1, j)] - A[FCO_IDX(m, i - 1, j)]) * 0.5;
                double gy = (A[FCO_IDX(m, i, j + 1)] - A[FCO_IDX(m, i, j - 1)]) * 0.5;
                double g = sqrt(gx * gx + gy * gy);
                if (g > c) c = g;
            }
        return c;
    }
    double mn = A[FCO_IDX(m, lo, lo)], mx = mn;
    for (int j = lo; j < hi; ++j)
        for (int i = lo; i < hi; ++i) {
            double v = A[FCO_IDX(m, i, j)];
            mn = minv(mn, v); mx = maxv(mx, v);
        }
    return mx - mn;
}

int fco_tag(fco_sim *s, int8_t *flags)
{
    if (s->p.conn == FCO_CONN_TABLE) { set_err("fco_tag: a table connectivity has no fields"); return FCO_ERR_ARG; }
    int m = s->p.m, F = s->F, h = m / 2;
    size_t PP = patch_pad(s);
    double *pad = (double *)malloc(sizeof(double) * (size_t)s->n * F * PP);
    int rc = fco_fill_ghosts(s, pad);
    if (rc) { free(pad); return rc; }
    double thr = s->p.tag_threshold;
    for (int k = 0; k < s->n; ++k) {
        const double *A = pad + (size_t)k * F * PP;          /* field 0 */
        int lo = s->p.tag_crit == FCO_TAG_GRAD ? 0 : 0;
        flags[k] = crit_padded(s, A, lo, m) > thr ? 1 : 0;
    }
    /* families: four consecutive sibling leaves above min_level */
    double *par = (double *)calloc(PP, sizeof(double));
    for (int k = 0; k + 3 < s->n; ++k) {
        const fco_leaf *l = &s->leaves[k];
        if (l->level <= s->p.min_level || (l->x & 1) || (l->y & 1)) continue;
        int fam = 1;
        for (int c = 0; c < 4; ++c) {
            const fco_leaf *o = &s->leaves[k + c];
            if (o->tree != l->tree || o->level != l->level || o->x != l->x + (c & 1) || o->y != l->y + (c >> 1)) fam = 0;
        }
        if (!fam) continue;
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                int c = (i >= h) + 2 * (j >= h);
                const double *q = s->q + (size_t)(k + c) * F * m * m;     /* field 0 */
                int fi = 2 * (i % h), fj = 2 * (j % h);
                double a00 = q[fj * m + fi], a10 = q[fj * m + fi + 1];
                double a01 = q[(fj + 1) * m + fi], a11 = q[(fj + 1) * m + fi + 1];
                par[FCO_IDX(m, i, j)] = 0.25 * ((a00 + a10) + (a01 + a11));
            }
        int lo = s->p.tag_crit == FCO_TAG_GRAD ? 1 : 0, hi = s->p.tag_crit == FCO_TAG_GRAD ? m - 1 : m;
        if (!(crit_padded(s, par, lo, hi) > thr))
            for (int c = 0; c < 4; ++c)
                if (flags[k + c] == 0) flags[k + c] = -1;
    }
    free(par);
    free(pad);
    return FCO_OK;
}

int fco_tag_patch_f32(int crit, int m, float threshold, const float *hpad)
{
    float c = 0.0f;
    if (crit == FCO_TAG_GRAD) {
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                float gx = (hpad[FCO_IDX(m, i + 1, j)] - hpad[FCO_IDX(m, i - 1, j)]) * 0.5f;
                float gy = (hpad[FCO_IDX(m, i, j + 1)] - hpad[FCO_IDX(m, i, j - 1)]) * 0.5f;
                float g = sqrtf(gx * gx + gy * gy);
                if (g > c) c = g;
            }
    } else {
        float mn = hpad[FCO_IDX(m, 0, 0)], mx = mn;
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                float v = hpad[FCO_IDX(m, i, j)];
                if (v < mn) mn = v;
                if (v > mx) mx = v;
            }
        c = mx - mn;
    }
    return c > threshold ? 1 : 0;
}

/* ---------------------------------------------------------------------- */
/* regrid (Sec. 3, last paragraph): new fine patches by limited linear      */
/* interpolation from the old patch's ghost-filled array (evaluated at the  */
/* new cell centres, any depth), new coarse patches by 2x2 averaging.       */
int fco_regrid(fco_sim *s, const int8_t *flags)
{
    if (s->p.conn == FCO_CONN_TABLE) { set_err("fco_regrid: a table connectivity has no fields"); return FCO_ERR_ARG; }
    int m = s->p.m, F = s->F, h = m / 2;
    size_t PP = patch_pad(s), pc = (size_t)F * m * m;
    int nold = s->n;
    fco_leaf *oldl = (fco_leaf *)malloc(sizeof(fco_leaf) * (size_t)nold);
    memcpy(oldl, s->leaves, sizeof(fco_leaf) * (size_t)nold);
    double *pad = (double *)malloc(sizeof(double) * (size_t)nold * F * PP);
    int rc = fco_fill_ghosts(s, pad);
    if (rc) { free(pad); free(oldl); return rc; }
    double *oldq = s->q;
    s->q = NULL;
    int32_t *org = NULL;
    fco_adapt(s, flags, &org);
    s->q = (double *)calloc((size_t)s->n * pc + 1, sizeof(double));
    for (int k = 0; k < s->n; ++k) {
        const fco_leaf *l = &s->leaves[k];
        int kind = org[3 * k], o = org[3 * k + 1], dl = org[3 * k + 2];
        double *q = s->q + (size_t)k * pc;
        if (kind == 0) { memcpy(q, oldq + (size_t)o * pc, sizeof(double) * pc); continue; }
        if (kind == 1) {
            const fco_leaf *L = &oldl[o];
            const double *A0 = pad + (size_t)o * F * PP;
            int r = 1 << dl;
            for (int j = 0; j < m; ++j)
                for (int i = 0; i < m; ++i) {
                    long long gi = (long long)l->x * m + i, gj = (long long)l->y * m + j;
                    int ci = (int)(gi / r - (long long)L->x * m), cj = (int)(gj / r - (long long)L->y * m);
                    double sgx = ((double)(gi % r) + 0.5) / r - 0.5;
                    double sgy = ((double)(gj % r) + 0.5) / r - 0.5;
                    for (int f = 0; f < F; ++f) {
                        const double *A = A0 + f * PP;
                        double qc = A[FCO_IDX(m, ci, cj)];
                        double sx = minmod(A[FCO_IDX(m, ci + 1, cj)] - qc, qc - A[FCO_IDX(m, ci - 1, cj)]);
                        double sy = minmod(A[FCO_IDX(m, ci, cj + 1)] - qc, qc - A[FCO_IDX(m, ci, cj - 1)]);
                        q[(size_t)f * m * m + j * m + i] = (qc + sgx * sx) + sgy * sy;
                    }
                }
            if (is_sphere(s->p.conn) && r <= m) {
                /* capacity-weighted correction per old cell: the new cells
                 * inside old cell (ci, cj) carry its mass kappa_c dxi_c^2 q_c
                 * exactly (the old cell lies inside one new leaf for r <= m;
                 * deeper refinement keeps the plain interpolation) */
                geom_t gn, go;
                geom_alloc(m, &gn); geom_alloc(m, &go);
                geom_build(s, l, &gn);
                geom_build(s, L, &go);
                int cells = m / r;
                for (int bj = 0; bj < cells; ++bj)
                    for (int bi = 0; bi < cells; ++bi) {
                        long long gi0 = (long long)l->x * m + bi * r, gj0 = (long long)l->y * m + bj * r;
                        int ci = (int)(gi0 / r - (long long)L->x * m), cj = (int)(gj0 / r - (long long)L->y * m);
                        double ksum = 0.0;
                        for (int jj = 0; jj < r; ++jj)
                            for (int ii = 0; ii < r; ++ii) ksum += GK(&gn, m, bi * r + ii, bj * r + jj);
                        for (int f = 0; f < F; ++f) {
                            double mass = 0.0;
                            for (int jj = 0; jj < r; ++jj)
                                for (int ii = 0; ii < r; ++ii)
                                    mass += GK(&gn, m, bi * r + ii, bj * r + jj) *
                                            q[(size_t)f * m * m + (bj * r + jj) * m + bi * r + ii];
                            double want = GK(&go, m, ci, cj) * (double)(r * r) *
                                          A0[f * PP + FCO_IDX(m, ci, cj)];
                            double d = (want - mass) / ksum;
                            for (int jj = 0; jj < r; ++jj)
                                for (int ii = 0; ii < r; ++ii) q[(size_t)f * m * m + (bj * r + jj) * m + bi * r + ii] += d;
                        }
                    }
                geom_free(&gn); geom_free(&go);
            }
            continue;
        }
        if (is_sphere(s->p.conn)) {  /* capacity-weighted 2x2 average */
            geom_t gc[4];
            for (int c = 0; c < 4; ++c) { geom_alloc(m, &gc[c]); geom_build(s, &oldl[o + c], &gc[c]); }
            for (int j = 0; j < m; ++j)
                for (int i = 0; i < m; ++i) {
                    int c = (i >= h) + 2 * (j >= h);
                    int fi = 2 * (i % h), fj = 2 * (j % h);
                    const geom_t *g = &gc[c];
                    double k00 = GK(g, m, fi, fj), k10 = GK(g, m, fi + 1, fj);
                    double k01 = GK(g, m, fi, fj + 1), k11 = GK(g, m, fi + 1, fj + 1);
                    double ks = (k00 + k10) + (k01 + k11);
                    for (int f = 0; f < F; ++f) {
                        const double *a = oldq + (size_t)(o + c) * pc + (size_t)f * m * m;
                        q[(size_t)f * m * m + j * m + i] =
                            ((k00 * a[fj * m + fi] + k10 * a[fj * m + fi + 1]) +
                             (k01 * a[(fj + 1) * m + fi] + k11 * a[(fj + 1) * m + fi + 1])) / ks;
                    }
                }
            for (int c = 0; c < 4; ++c) geom_free(&gc[c]);
            continue;
        }
        for (int j = 0; j < m; ++j)          /* parent of old leaves o..o+3 */
            for (int i = 0; i < m; ++i) {
                int c = (i >= h) + 2 * (j >= h);
                int fi = 2 * (i % h), fj = 2 * (j % h);
                for (int f = 0; f < F; ++f) {
                    const double *a = oldq + (size_t)(o + c) * pc + (size_t)f * m * m;
                    q[(size_t)f * m * m + j * m + i] =
                        0.25 * ((a[fj * m + fi] + a[fj * m + fi + 1]) + (a[(fj + 1) * m + fi] + a[(fj + 1) * m + fi + 1]));
                }
            }
    }
    free(org); free(oldq); free(pad); free(oldl);
    s->dt_from_cells = 1;
    return FCO_OK;
}

/* R15: uniform at min_level, then (max - min) rounds of {initialise, tag,
 * refine, balance}, then a final initialisation. */
int fco_init_refine(fco_sim *s, int kind, const double *p, int np)
{
    if (s->p.conn == FCO_CONN_TABLE) { set_err("fco_init_refine: a table connectivity has no fields"); return FCO_ERR_ARG; }
    int rc = fco_forest_uniform(s, s->p.min_level);
    if (rc) return rc;
    for (int r = 0; r < s->p.max_level - s->p.min_level; ++r) {
        if ((rc = fco_init_fields(s, kind, p, np))) return rc;
        int8_t *fl = (int8_t *)malloc((size_t)s->n);
        if ((rc = fco_tag(s, fl))) { free(fl); return rc; }
        for (int k = 0; k < s->n; ++k) if (fl[k] < 0) fl[k] = 0;
        fco_adapt(s, fl, NULL);
        free(fl);
        realloc_fields(s);
    }
    rc = fco_init_fields(s, kind, p, np);
    s->dt_from_cells = 1;
    return rc;
}
