/*
 * fco_pillow.c -- two-tree sphere geometry for the oracle (TEST INFRASTRUCTURE).
 *
 * Sec. 5, Example 2: two quadtrees, each on the reference square [-1,1]^2,
 * each mapped onto one hemisphere; solid-body rotation carries a field that
 * is 0 on one half of the sphere and 1 on the other.  The paper cites the
 * mapping without giving it.  The reading used here (one logically
 * rectangular 2N x N strip folded onto the sphere):
 *   - tree 0 is the northern hemisphere, tree 1 the southern one with its
 *     x coordinate mirrored, so that the two trees side by side (tree 0's
 *     right border against tree 1's left border) form one strip that is
 *     periodic in x; a y border of one tree meets the y border of the other
 *     with a half turn (x -> -x);
 *   - square to disc by concentric squares: the square of half-width
 *     r = max(|x|, |y|) goes to the circle of colatitude theta = r pi / 2,
 *     the longitude phi running linearly in the ratio of the smaller to the
 *     larger coordinate along each of the four sides (pi/2 per side);
 *   - the area element is then (pi^2 / 8) sin(pi r / 2) / r dx dy (one
 *     hemisphere integrates to 2 pi); a cell's area is that integral over
 *     the cell, evaluated piece by piece where r is one of |x|, |y|, so that
 *     areas are additive under refinement to rounding;
 *   - the four corners of each square lie on the equator, where two cells
 *     meet with an angle of pi each: a corner patch faces the same patch of
 *     the other tree across both of its border sides, and the point beyond
 *     both borders at once is the patch's own corner reflected through the
 *     corner point.
 * Coordinates: doubled centred, as for the cubed sphere: a point of tree t
 * is (U, V) with x = U / N, y = V / N, N = 2^FCO_MAXLEVEL.
 */
#include "fco_internal.h"
#include <math.h>

/* fold a doubled-coordinate point beyond tree t's border onto the tree that
 * holds it; border points stay on tree t */
int fco_pillow_fold(int t, long long U, long long V, long long *Uo, long long *Vo)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    if (U > N) { U -= 2 * N; t = 1 - t; }
    else if (U < -N) { U += 2 * N; t = 1 - t; }
    if (V > N) { V = 2 * N - V; U = -U; t = 1 - t; }
    else if (V < -N) { V = -2 * N - V; U = -U; t = 1 - t; }
    *Uo = U; *Vo = V;
    return t;
}

int fco_pillow_point(int t, long long U, long long V, double p[3])
{
    const long long N = 1LL << FCO_MAXLEVEL;
    long long Uf, Vf;
    t = fco_pillow_fold(t, U, V, &Uf, &Vf);
    double x = (double)Uf / (double)N, y = (double)Vf / (double)N;
    if (t == 1) x = -x;
    double ax = fabs(x), ay = fabs(y), r = ax > ay ? ax : ay, phi = 0.0;
    if (r > 0.0) {
        if (ax >= ay) phi = x > 0.0 ? (M_PI / 4.0) * (y / x) : M_PI + (M_PI / 4.0) * (y / x);
        else phi = y > 0.0 ? M_PI / 2.0 - (M_PI / 4.0) * (x / y) : 1.5 * M_PI - (M_PI / 4.0) * (x / y);
    }
    double st = 1.0, ct = 0.0;               /* the equator exactly, from either tree */
    if (r < 1.0) { st = sin((M_PI / 2.0) * r); ct = cos((M_PI / 2.0) * r); }
    p[0] = st * cos(phi);
    p[1] = st * sin(phi);
    p[2] = t == 0 ? ct : -ct;
    return 1;
}

/* Gauss-Legendre nodes and weights on [-1, 1], from Newton's method on the
 * three-term recurrence of the Legendre polynomials */
#define GL_N 12
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void)
{
    for (int i = 0; i < GL_N; ++i) {
        double z = cos(M_PI * (i + 0.75) / (GL_N + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= GL_N; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    gl_ready = 1;
}

/* g(u) = sin(pi u / 2) / u: the area element's radial factor */
static double g_rad(double u) { return sin((M_PI / 2.0) * u) / u; }

/* integral over [a, b] of g(u) * (c0 + c1 u) (Gauss-Legendre; the integrand
 * is entire, so GL_N nodes reach rounding on any sub-interval of [0, 1]) */
static double gl_lin(double a, double b, double c0, double c1)
{
    if (!(b > a)) return 0.0;
    double h = 0.5 * (b - a), c = 0.5 * (b + a), s = 0.0;
    for (int i = 0; i < GL_N; ++i) {
        double u = c + h * gl_x[i];
        s += gl_w[i] * (g_rad(u) * (c0 + c1 * u));
    }
    return h * s;
}

/* K = integral over u in [a0, a1] of g(u) * |[b0, min(b1, u)]| (the part of
 * the rectangle [a0, a1] x [b0, b1], 0 <= a0, 0 <= b0, where u = r is the
 * first coordinate); the weight is piecewise linear with kinks at b0, b1 */
static double k_part(double a0, double a1, double b0, double b1)
{
    double lo = a0 > b0 ? a0 : b0;            /* below b0 the weight is 0 */
    double mid = a1 < b1 ? a1 : b1;           /* between b0 and b1: u - b0 */
    double s = 0.0;
    if (mid > lo) s += gl_lin(lo, mid, -b0, 1.0);
    double lo2 = a0 > b1 ? a0 : b1;           /* above b1: b1 - b0 */
    if (a1 > lo2) s += gl_lin(lo2, a1, b1 - b0, 0.0);
    return s;
}

/* integral of g(max(x, y)) over [a0, a1] x [b0, b1] in the first quadrant */
static double quad_part(double a0, double a1, double b0, double b1)
{
    return k_part(a0, a1, b0, b1) + k_part(b0, b1, a0, a1);
}

/* the same over any rectangle: split at the axes, reflect into the first
 * quadrant (g depends on |x|, |y| only) */
static double rect_integral(double x0, double x1, double y0, double y1)
{
    double xs[2][2], ys[2][2];
    int nx = 0, ny = 0;
    if (x0 < 0.0) { xs[nx][0] = x1 < 0.0 ? -x1 : 0.0; xs[nx][1] = -x0; ++nx; }
    if (x1 > 0.0) { xs[nx][0] = x0 > 0.0 ? x0 : 0.0; xs[nx][1] = x1; ++nx; }
    if (y0 < 0.0) { ys[ny][0] = y1 < 0.0 ? -y1 : 0.0; ys[ny][1] = -y0; ++ny; }
    if (y1 > 0.0) { ys[ny][0] = y0 > 0.0 ? y0 : 0.0; ys[ny][1] = y1; ++ny; }
    double s = 0.0;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j) s += quad_part(xs[i][0], xs[i][1], ys[j][0], ys[j][1]);
    return s;
}

/* spherical area of the cell [U0, U1] x [V0, V1] of tree t (doubled
 * coordinates; a cell beyond the border is measured in the tree that holds
 * it -- the area element is the same in both trees and even in x and y) */
double fco_pillow_cell_area(int t, long long U0, long long U1, long long V0, long long V1)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    if (!gl_ready) gl_init();
    long long a, b, c, d;
    /* fold the cell through its centre's tree */
    long long Uc = (U0 + U1) / 2, Vc = (V0 + V1) / 2, Ucf, Vcf;
    fco_pillow_fold(t, Uc, Vc, &Ucf, &Vcf);
    long long hu = (U1 - U0) / 2, hv = (V1 - V0) / 2;
    a = Ucf - hu; b = Ucf + hu; c = Vcf - hv; d = Vcf + hv;
    double x0 = (double)a / (double)N, x1 = (double)b / (double)N;
    double y0 = (double)c / (double)N, y1 = (double)d / (double)N;
    return (M_PI * M_PI / 8.0) * rect_integral(x0, x1, y0, y1);
}
