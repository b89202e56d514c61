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

}  // namespace fc
