// fc_sphere.cuh -- the cubed sphere: six trees on the faces of a cube
// (Fig. 1 right of the paper), neighbour access across trees by coordinate
// transformation (Sec. 4), and the mapped geometry of scalar advection by
// solid-body rotation (Sec. 5, Eq. (1), written in capacity form).
//
// Conventions (they fix tree numbering and the neighbour table, so they are
// part of the library's interface):
//   * tree t covers the face with outward normal n_t; its x axis runs along
//     a_t and its y axis along b_t, with a_t x b_t = n_t:
//         t  n    a    b
//         0  +x   +y   +z
//         1  +y   -x   +z
//         2  -x   -y   +z
//         3  -y   +x   +z
//         4  +z   +y   -x
//         5  -z   +y   +x
//   * doubled centred coordinates: the point (U, V) of tree t is the cube
//     point N n_t + U a_t + V b_t, N = 2^30; the finest-level coordinate X of
//     a point centred in finest cell X is U = 2X + 1 - N;
//   * the sphere point of a cube point c is q / |q| with q_k = tan(pi/4 c_k/N)
//     (equiangular gnomonic map), q_k = +-1 exactly where |c_k| = N, so points
//     on cube edges are computed identically from both trees;
//   * streamfunction of rotation with angular speed omega about the unit axis
//     k = (sin tilt, 0, cos tilt): psi = omega k . p; the flux through an edge
//     is the difference of psi at its end points, so every cell's net flux
//     telescopes to zero (discretely divergence-free velocity);
//   * cell area: exact spherical area of the cell between its four
//     great-circle edges, evaluated in the tree that holds the cell.
#pragma once
#include "fc_internal.cuh"

namespace fc {

struct CubeFace { signed char n[3], a[3], b[3]; };

static __constant__ CubeFace c_cube[6] = {
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
    {{-1, 0, 0}, {0, -1, 0}, {0, 0, 1}},
    {{0, -1, 0}, {1, 0, 0}, {0, 0, 1}},
    {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}},
    {{0, 0, -1}, {0, 1, 0}, {1, 0, 0}},
};

constexpr long long kCubeN = 1LL << kMaxBits;

__device__ inline int cube_tree_of_normal(long long v0, long long v1, long long v2)
{
    for (int t = 0; t < 6; ++t)
        if (c_cube[t].n[0] == v0 && c_cube[t].n[1] == v1 && c_cube[t].n[2] == v2) return t;
    return -1;
}

// Fold a doubled-coordinate point of tree t that lies beyond exactly one of
// the tree's borders onto the neighbouring face.  `strict`: a point exactly on
// the border stays in t (geometry); otherwise |U| = N counts as beyond (never
// met for cell centres, whose doubled coordinates are odd).  Returns the
// tree, or -1 beyond a cube corner.
__device__ inline int cube_fold(int t, long long U, long long V, bool strict, long long *Uo, long long *Vo)
{
    const long long N = kCubeN;
    const bool outU = strict ? (U > N || U < -N) : (U >= N || U <= -N);
    const bool outV = strict ? (V > N || V < -N) : (V >= N || V <= -N);
    if (!outU && !outV) { *Uo = U; *Vo = V; return t; }
    if (outU && outV) return -1;
    const CubeFace &f = c_cube[t];
    const long long s = outU ? (U > 0 ? 1 : -1) : (V > 0 ? 1 : -1);
    const long long E = (outU ? s * U : s * V) - N;            // distance beyond the edge
    const signed char *ax = outU ? f.a : f.b;
    long long P[3];
    for (int k = 0; k < 3; ++k)                                // fold the overhang down along -n
        P[k] = (N - E) * f.n[k] + s * N * ax[k] + (outU ? 0 : U * f.a[k]) + (outV ? 0 : V * f.b[k]);
    const int t2 = cube_tree_of_normal(s * ax[0], s * ax[1], s * ax[2]);
    const CubeFace &g = c_cube[t2];
    *Uo = P[0] * g.a[0] + P[1] * g.a[1] + P[2] * g.a[2];
    *Vo = P[0] * g.b[0] + P[1] * g.b[1] + P[2] * g.b[2];
    return t2;
}

// finest-level point (X, Y) of tree t, possibly just outside [0, N)^2, to
// the tree holding it; -1 beyond a cube corner
__device__ inline int cube_map_point(int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    const long long N = kCubeN;
    long long Uo, Vo;
    const int t2 = cube_fold(t, 2 * X + 1 - N, 2 * Y + 1 - N, false, &Uo, &Vo);
    if (t2 < 0) return -1;
    *Xo = (Uo + N - 1) / 2;
    *Yo = (Vo + N - 1) / 2;
    return t2;
}

// Orientation of the offset map from tree t into the tree holding the probe
// point (X, Y) outside t: 1 + 4 swap + 2 (image of +x negative) + (image of
// +y negative), from the images of unit steps that stay on the probe's side
// of the crossed edge; 0 when the point is inside t or beyond a corner.
__device__ inline int cube_orientation(int t, long long X, long long Y)
{
    const long long N = kCubeN;
    if (X >= 0 && X < N && Y >= 0 && Y < N) return 0;
    long long X0, Y0, X1, Y1, X2, Y2;
    if (cube_map_point(t, X, Y, &X0, &Y0) < 0) return 0;
    long long sx = (X < 0 || X >= N) ? (X < 0 ? -1 : 1) : 1;
    long long sy = (Y < 0 || Y >= N) ? (Y < 0 ? -1 : 1) : 1;
    if (X >= 0 && X < N && X + sx >= N) sx = -1;
    if (Y >= 0 && Y < N && Y + sy >= N) sy = -1;
    cube_map_point(t, X + sx, Y, &X1, &Y1);
    cube_map_point(t, X, Y + sy, &X2, &Y2);
    const long long ix = (X1 - X0) * sx, iy = (Y1 - Y0) * sx;   // image of +x
    const long long jx = (X2 - X0) * sy, jy = (Y2 - Y0) * sy;   // image of +y
    const int swap = ix == 0;
    const int r0 = swap ? (jx < 0) : (ix < 0);
    const int r1 = swap ? (iy < 0) : (jy < 0);
    return 1 + 4 * swap + 2 * r0 + r1;
}

// ---------------------------------------------------------------------------
// mapped geometry, FP64 with explicit rounding (evaluated once per forest)
constexpr double kQuarterPi = 0.78539816339744830962;

// unit-sphere point of doubled coordinates (U, V) of tree t; beyond a cube
// corner tree t's own map is extended
__device__ inline void sph_point(int t, long long U, long long V, double p[3])
{
    const long long N = kCubeN;
    long long Uf, Vf;
    int tf = cube_fold(t, U, V, true, &Uf, &Vf);
    if (tf < 0) { tf = t; Uf = U; Vf = V; }
    const CubeFace &f = c_cube[tf];
    double q[3];
    for (int k = 0; k < 3; ++k) {
        const long long c = N * f.n[k] + Uf * f.a[k] + Vf * f.b[k];
        q[k] = c == N ? 1.0 : (c == -N ? -1.0 : tan(__dmul_rn(kQuarterPi, (double)c / (double)N)));
    }
    const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])), __dmul_rn(q[2], q[2])));
    for (int k = 0; k < 3; ++k) p[k] = q[k] / r;
}

__device__ inline double sph_psi(double omega, double tilt, const double p[3])
{
    const double kx = sin(tilt), kz = cos(tilt);
    return __dmul_rn(omega, __dadd_rn(__dadd_rn(__dmul_rn(kx, p[0]), __dmul_rn(0.0, p[1])), __dmul_rn(kz, p[2])));
}

// signed area of the face-angle rectangle [0, a] x [0, b]
__device__ inline double sph_corner(double a, double b)
{
    const double ta = tan(a), tb = tan(b);
    return atan(__dmul_rn(ta, tb) / sqrt(__dadd_rn(__dadd_rn(1.0, __dmul_rn(ta, ta)), __dmul_rn(tb, tb))));
}

// area of the cell [U0, U1] x [V0, V1] of tree t (U0 < U1, V0 < V1, equal
// widths), computed in the tree that holds the cell centre: the fold is an
// isometry of the cube surface, so the cell stays an axis-aligned square of
// the same width there
__device__ inline double sph_cell_area(int t, long long U0, long long U1, long long V0, long long V1)
{
    const long long h = (U1 - U0) / 2;
    long long Uc, Vc;
    int tf = cube_fold(t, U0 + h, V0 + (V1 - V0) / 2, true, &Uc, &Vc);
    long long Ua = U0, Ub = U1, Va = V0, Vb = V1;
    if (tf >= 0 && tf != t) { Ua = Uc - h; Ub = Uc + h; Va = Vc - h; Vb = Vc + h; }
    const double k = kQuarterPi / (double)kCubeN;
    const double a1 = __dmul_rn(k, (double)Ua), a2 = __dmul_rn(k, (double)Ub);
    const double b1 = __dmul_rn(k, (double)Va), b2 = __dmul_rn(k, (double)Vb);
    return __dadd_rn(__dadd_rn(__dadd_rn(sph_corner(a2, b2), -sph_corner(a1, b2)), -sph_corner(a2, b1)),
                     sph_corner(a1, b1));
}

// ---------------------------------------------------------------------------
// Two-tree sphere (Sec. 5, Example 2: two quadtrees on [-1, 1]^2, one per
// hemisphere).  The paper cites the map without giving it; the library's
// reading (part of its interface, like the cube's conventions above):
//   * tree 0 covers the northern hemisphere, tree 1 the southern one with its
//     x axis mirrored; side by side (tree 0's +x border against tree 1's -x
//     border) they form one strip of 2N x N finest cells, periodic in x; a y
//     border of one tree meets the same y border of the other with a half
//     turn (x -> -x);
//   * beyond both borders at a tree corner lies the patch's own corner,
//     reflected through the corner point (the corner is a point of the
//     equator where only two cells meet);
//   * the point (x, y) = (U, V) / N goes to colatitude (pi / 2) max(|x|, |y|)
//     (from the south pole for tree 1, after mirroring x) and to a longitude
//     linear in the ratio of the smaller to the larger coordinate along each
//     side of the concentric square, pi / 2 per side;
//   * cell area: the integral of the map's area element
//     (pi^2 / 8) sin(pi r / 2) / r over the cell, r = max(|x|, |y|), so that
//     areas add up under refinement.

// doubled coordinates beyond tree t's borders to the tree holding them
// (`strict`: a point exactly on a border stays in t)
__device__ inline int pillow_fold(int t, long long U, long long V, bool strict, long long *Uo, long long *Vo)
{
    const long long N = kCubeN;
    const bool xp = strict ? U > N : U >= N, xm = strict ? U < -N : U <= -N;
    const bool yp = strict ? V > N : V >= N, ym = strict ? V < -N : V <= -N;
    if (xp || xm) { U += xp ? -2 * N : 2 * N; t ^= 1; }
    if (yp || ym) { V = (yp ? 2 * N : -2 * N) - V; U = -U; t ^= 1; }
    *Uo = U;
    *Vo = V;
    return t;
}

__device__ inline int pillow_map_point(int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    const long long N = kCubeN;
    long long Uo, Vo;
    const int t2 = pillow_fold(t, 2 * X + 1 - N, 2 * Y + 1 - N, false, &Uo, &Vo);
    *Xo = (Uo + N - 1) / 2;
    *Yo = (Vo + N - 1) / 2;
    return t2;
}

// finest-level point of either sphere to the tree holding it
__device__ inline int sphere_map_point(int conn, int t, long long X, long long Y, long long *Xo, long long *Yo)
{
    return conn == FC_CONN_PILLOW ? pillow_map_point(t, X, Y, Xo, Yo) : cube_map_point(t, X, Y, Xo, Yo);
}

// cube_orientation's code for either sphere
__device__ inline int sphere_orientation(int conn, int t, long long X, long long Y)
{
    if (conn != FC_CONN_PILLOW) return cube_orientation(t, X, Y);
    const long long N = kCubeN;
    if (X >= 0 && X < N && Y >= 0 && Y < N) return 0;
    long long X0, Y0, X1, Y1, X2, Y2;
    const long long sx = X < 0 ? -1 : (X >= N ? 1 : (X + 1 >= N ? -1 : 1));
    const long long sy = Y < 0 ? -1 : (Y >= N ? 1 : (Y + 1 >= N ? -1 : 1));
    pillow_map_point(t, X, Y, &X0, &Y0);
    pillow_map_point(t, X + sx, Y, &X1, &Y1);
    pillow_map_point(t, X, Y + sy, &X2, &Y2);
    const long long ix = (X1 - X0) * sx, iy = (Y1 - Y0) * sx;
    const long long jx = (X2 - X0) * sy, jy = (Y2 - Y0) * sy;
    const int swap = ix == 0;
    const int r0 = swap ? (jx < 0) : (ix < 0);
    const int r1 = swap ? (iy < 0) : (jy < 0);
    return 1 + 4 * swap + 2 * r0 + r1;
}

__device__ inline void pil_point(int t, long long U, long long V, double p[3])
{
    long long Uf, Vf;
    t = pillow_fold(t, U, V, true, &Uf, &Vf);
    const double x = (t ? -(double)Uf : (double)Uf) / (double)kCubeN, y = (double)Vf / (double)kCubeN;
    const double ax = fabs(x), ay = fabs(y), r = fmax(ax, ay);
    double lon = 0.0;
    if (r > 0.0) {
        if (ax >= ay) lon = __dadd_rn(x > 0.0 ? 0.0 : 2.0 * (2.0 * kQuarterPi), __dmul_rn(kQuarterPi, y / x));
        else lon = __dadd_rn(y > 0.0 ? 2.0 * kQuarterPi : 6.0 * kQuarterPi, -__dmul_rn(kQuarterPi, x / y));
    }
    double sn = 1.0, cs = 0.0;                   // the equator exactly, from either tree
    if (r < 1.0) { const double th = __dmul_rn(2.0 * kQuarterPi, r); sn = sin(th); cs = cos(th); }
    p[0] = __dmul_rn(sn, cos(lon));
    p[1] = __dmul_rn(sn, sin(lon));
    p[2] = t ? -cs : cs;
}

// Gauss-Legendre rule of kGl points on [-1, 1]: node i by Newton's method on
// P_n from the three-term recurrence, weight 2 / ((1 - x^2) P_n'(x)^2)
constexpr int kGl = 12;
__device__ inline void gl_node(int i, double *x, double *w)
{
    double z = cos(3.14159265358979323846 * ((double)i + 0.75) / ((double)kGl + 0.5)), dp = 1.0;
    for (int it = 0; it < 8; ++it) {
        double a = 1.0, b = z;
        for (int k = 2; k <= kGl; ++k) {
            const double c = ((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / (double)k;
            a = b;
            b = c;
        }
        dp = (double)kGl * (z * b - a) / (z * z - 1.0);
        z -= b / dp;
    }
    double a = 1.0, b = z;
    for (int k = 2; k <= kGl; ++k) {
        const double c = ((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / (double)k;
        a = b;
        b = c;
    }
    dp = (double)kGl * (z * b - a) / (z * z - 1.0);
    *x = z;
    *w = 2.0 / ((1.0 - z * z) * dp * dp);
}

// integral over [a, b] of sin(pi u / 2) / u * (c0 + c1 u)
__device__ inline double pil_seg(const double *gx, const double *gw, double a, double b, double c0, double c1)
{
    if (!(b > a)) return 0.0;
    const double h = 0.5 * (b - a), c = 0.5 * (b + a);
    double s = 0.0;
    for (int i = 0; i < kGl; ++i) {
        const double u = c + h * gx[i];
        s += gw[i] * (sin(2.0 * kQuarterPi * u) / u * (c0 + c1 * u));
    }
    return h * s;
}

// the part of [a0, a1] x [b0, b1] (first quadrant) where the first
// coordinate is the larger: weight |[b0, min(b1, u)]|, linear between kinks
__device__ inline double pil_half(const double *gx, const double *gw, double a0, double a1, double b0, double b1)
{
    double s = 0.0;
    const double lo = fmax(a0, b0), hi = fmin(a1, b1);
    if (hi > lo) s += pil_seg(gx, gw, lo, hi, -b0, 1.0);
    const double lo2 = fmax(a0, b1);
    if (a1 > lo2) s += pil_seg(gx, gw, lo2, a1, b1 - b0, 0.0);
    return s;
}

__device__ inline double pil_rect(const double *gx, const double *gw, double x0, double x1, double y0, double y1)
{
    double xa[2][2], ya[2][2];
    int nx = 0, ny = 0;
    if (x0 < 0.0) { xa[nx][0] = x1 < 0.0 ? -x1 : 0.0; xa[nx][1] = -x0; ++nx; }
    if (x1 > 0.0) { xa[nx][0] = fmax(x0, 0.0); xa[nx][1] = x1; ++nx; }
    if (y0 < 0.0) { ya[ny][0] = y1 < 0.0 ? -y1 : 0.0; ya[ny][1] = -y0; ++ny; }
    if (y1 > 0.0) { ya[ny][0] = fmax(y0, 0.0); ya[ny][1] = y1; ++ny; }
    double s = 0.0;
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < ny; ++b)
            s += pil_half(gx, gw, xa[a][0], xa[a][1], ya[b][0], ya[b][1]) +
                 pil_half(gx, gw, ya[b][0], ya[b][1], xa[a][0], xa[a][1]);
    return s;
}

// area of the cell [U0, U1] x [V0, V1] of tree t, measured in the tree that
// holds its centre (the fold keeps the cell a square of the same width)
__device__ inline double pil_cell_area(const double *gx, const double *gw, int t, long long U0, long long U1,
                                       long long V0, long long V1)
{
    const long long h = (U1 - U0) / 2;
    long long Uc, Vc;
    pillow_fold(t, U0 + h, V0 + h, true, &Uc, &Vc);
    const double N = (double)kCubeN;
    return (2.0 * kQuarterPi) * (2.0 * kQuarterPi) * 0.5 *
           pil_rect(gx, gw, (double)(Uc - h) / N, (double)(Uc + h) / N, (double)(Vc - h) / N, (double)(Vc + h) / N);
}

}  // namespace fc
