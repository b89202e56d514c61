/*
 * fco_sphere.c -- cubed-sphere geometry for the oracle (TEST INFRASTRUCTURE).
 *
 * Fig. 1 (right) of the paper shows a forest of six quadtrees forming the
 * cubed sphere; Sec. 2 identifies each tree with a mapped reference square and
 * Sec. 4 describes neighbour access across trees with coordinate
 * transformations; Sec. 5 Eq. (1) is scalar advection by a prescribed velocity.
 * The mapping is not given in the paper; the readings used here:
 *   - equiangular gnomonic faces: a point of tree t with doubled centred
 *     coordinates (U, V) (cube point N n + U a + V b) lies on the unit sphere at
 *     p / |p|, p_k = tan(pi/4 c_k / N) for the integer cube coordinates c_k,
 *     with p_k = +-1 exactly where |c_k| = N (so points on cube edges are
 *     computed identically from every tree that shares them);
 *   - solid-body rotation with angular speed omega about the axis tilted by
 *     `tilt` from z in the x-z plane has streamfunction psi(p) = omega k . p;
 *     the flux through an edge is the difference of psi at its end nodes, so
 *     the discrete velocity is divergence free;
 *   - cell area = exact spherical area of the cell between its four great-circle
 *     edges, in the coordinates of the tree that contains the cell.
 */
#include "fco_internal.h"
#include <math.h>

extern const int fco_cube_n[6][3], fco_cube_a[6][3], fco_cube_b[6][3];

/* fold a doubled-coordinate point of tree t onto the face that contains it;
 * points exactly on a face border stay on tree t.  Returns the face's tree or
 * -1 beyond a cube corner. */
int fco_sphere_fold(int t, long long U, long long V, long long *Uo, long long *Vo)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    int outU = U > N || U < -N, outV = V > N || V < -N;
    if (!outU && !outV) { *Uo = U; *Vo = V; return t; }
    if (outU && outV) return -1;
    long long s = outU ? (U > 0 ? 1 : -1) : (V > 0 ? 1 : -1);
    long long E = outU ? s * U - N : s * V - N;
    const int *ax = outU ? fco_cube_a[t] : fco_cube_b[t];
    long long c[3];
    for (int k = 0; k < 3; ++k)
        c[k] = (N - E) * fco_cube_n[t][k] + s * N * ax[k] + (outU ? 0 : U * fco_cube_a[t][k]) +
               (outV ? 0 : V * fco_cube_b[t][k]);
    int t2 = -1;
    for (int q = 0; q < 6; ++q)
        if (fco_cube_n[q][0] == s * ax[0] && fco_cube_n[q][1] == s * ax[1] && fco_cube_n[q][2] == s * ax[2]) t2 = q;
    *Uo = c[0] * fco_cube_a[t2][0] + c[1] * fco_cube_a[t2][1] + c[2] * fco_cube_a[t2][2];
    *Vo = c[0] * fco_cube_b[t2][0] + c[1] * fco_cube_b[t2][1] + c[2] * fco_cube_b[t2][2];
    return t2;
}

/* unit-sphere point of doubled coordinates (U, V) in tree t (folded first);
 * returns 0 beyond a cube corner */
int fco_sphere_point(int t, long long U, long long V, double p[3])
{
    const long long N = 1LL << FCO_MAXLEVEL;
    long long Uf, Vf;
    int tf = fco_sphere_fold(t, U, V, &Uf, &Vf);
    if (tf < 0) {   /* beyond a cube corner: extend tree t's gnomonic map */
        tf = t; Uf = U; Vf = V;
    }
    double q[3];
    for (int k = 0; k < 3; ++k) {
        long long c = N * fco_cube_n[tf][k] + Uf * fco_cube_a[tf][k] + Vf * fco_cube_b[tf][k];
        if (c == N) q[k] = 1.0;
        else if (c == -N) q[k] = -1.0;
        else q[k] = tan((M_PI / 4.0) * ((double)c / (double)N));
    }
    double r = sqrt((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]);
    for (int k = 0; k < 3; ++k) p[k] = q[k] / r;
    return 1;
}

double fco_sphere_psi(const fco_params *pr, const double p[3])
{
    double kx = sin(pr->omega_axis_tilt), kz = cos(pr->omega_axis_tilt);
    return pr->omega * ((kx * p[0] + 0.0 * p[1]) + kz * p[2]);
}

/* area of the face-coordinate rectangle [a1, a2] x [b1, b2] (angles) */
static double omega_corner(double a, double b)
{
    double ta = tan(a), tb = tan(b);
    return atan(ta * tb / sqrt(1.0 + ta * ta + tb * tb));
}

/* exact area of the cell with doubled-coordinate corners U0 < U1, V0 < V1 of
 * tree t, computed in the tree that contains the cell centre */
double fco_sphere_cell_area(int t, long long U0, long long U1, long long V0, long long V1)
{
    const long long N = 1LL << FCO_MAXLEVEL;
    long long Uc = (U0 + U1) / 2, Vc = (V0 + V1) / 2, Ua, Va, Ub, Vb, tmp;
    int tf = fco_sphere_fold(t, Uc, Vc, &tmp, &tmp);
    if (tf < 0) tf = t;
    if (tf == t) { Ua = U0; Ub = U1; Va = V0; Vb = V1; }
    else {
        fco_sphere_fold(t, U0, V0, &Ua, &Va);
        fco_sphere_fold(t, U1, V1, &Ub, &Vb);
        /* a corner exactly on the border stays in t: fold a point just inside */
        long long e = (U1 - U0) / 4;
        long long x0, y0, x1, y1;
        fco_sphere_fold(t, U0 + e, V0 + e, &x0, &y0);
        fco_sphere_fold(t, U1 - e, V1 - e, &x1, &y1);
        long long lo_u = x0 < x1 ? x0 : x1, hi_u = x0 < x1 ? x1 : x0;
        long long lo_v = y0 < y1 ? y0 : y1, hi_v = y0 < y1 ? y1 : y0;
        Ua = lo_u - e; Ub = hi_u + e; Va = lo_v - e; Vb = hi_v + e;
    }
    double k = M_PI / 4.0 / (double)N;
    double a1 = k * (double)Ua, a2 = k * (double)Ub, b1 = k * (double)Va, b2 = k * (double)Vb;
    return ((omega_corner(a2, b2) - omega_corner(a1, b2)) - omega_corner(a2, b1)) + omega_corner(a1, b1);
}
