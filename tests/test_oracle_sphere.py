"""Pins of the oracle's cubed sphere (Fig. 1 right, Sec. 4, Sec. 5 Eq. (1) in
capacity form) against facts that do not come from the oracle's formulas:

* spherical geometry: each cell is a geodesic quadrilateral (the gnomonic map
  sends straight face lines to great circles), so its area is its spherical
  excess by Girard's theorem, computed here from the corner points alone; the
  cells of all six trees tile the sphere (total area 4 pi); the map is
  equiangular (equal steps of U are equal angles along a face's centre line);
  every tree's frame is right-handed and outward; a point on a cube edge has
  bitwise the same sphere point from both trees;
* mass: the sum of area x q is conserved to roundoff by stepping (uniform,
  adaptive, subcycled, with refluxing) and by regridding;
* solid-body rotation: after one period the hill is back where it started, with
  an error that shrinks under refinement; after a quarter period the hill sits a
  quarter turn further counterclockwise about the axis (right-hand rule);
* ghost cells across tree borders hold the neighbouring tree's cell values.
"""
import math

import numpy as np
import pytest

from fc_inputs import SplitMix64
from oracle import fco
from oracle.fco import Oracle, OracleParams

N = fco.SPHERE_N


def _girard(P):
    """area of the geodesic polygon with unit-vector corners P (in order)"""
    k = len(P)
    tot = 0.0
    for i in range(k):
        v, a, b = P[i], P[(i + 1) % k], P[(i - 1) % k]
        ta = a - np.dot(a, v) * v
        tb = b - np.dot(b, v) * v
        ta /= np.linalg.norm(ta)
        tb /= np.linalg.norm(tb)
        tot += math.acos(max(-1.0, min(1.0, float(np.dot(ta, tb)))))
    return tot - (k - 2) * math.pi


def _frames():
    """(n, a, b) of each tree recovered from mapped points"""
    out = []
    for t in range(6):
        n = fco.sphere_point(t, 0, 0)
        a = np.sqrt(2.0) * fco.sphere_point(t, N, 0) - n
        b = np.sqrt(2.0) * fco.sphere_point(t, 0, N) - n
        out.append(tuple(np.rint(v).astype(int) for v in (n, a, b)))
    return out


def test_frames_are_right_handed_and_cover_the_cube():
    fr = _frames()
    normals = {tuple(n) for n, _, _ in fr}
    assert len(normals) == 6 and all(sum(abs(c) for c in n) == 1 for n in normals)
    for n, a, b in fr:
        assert tuple(np.cross(a, b)) == tuple(n)


def test_equiangular_centre_lines():
    for t in range(6):
        p0 = fco.sphere_point(t, 0, 0)
        for k in range(-4, 5):
            U = k * (N // 4)
            for p in (fco.sphere_point(t, U, 0), fco.sphere_point(t, 0, U)):
                ang = math.atan2(np.linalg.norm(np.cross(p0, p)), float(np.dot(p0, p)))
                assert abs(ang - math.pi / 4 * abs(U) / N) < 1e-14


def test_points_on_cube_edges_agree_bitwise():
    fr = _frames()
    rng = SplitMix64(17)
    for t in range(6):
        n, a, b = fr[t]
        for _ in range(40):
            s = 1 if rng.next_u64() & 1 else -1
            V = int(rng.next_u64() % (2 * N + 1)) - N
            for U, W in ((s * N, V), (V, s * N)):
                c = N * n + U * a + W * b
                p = fco.sphere_point(t, U, W)
                for t2 in range(6):
                    n2, a2, b2 = fr[t2]
                    if t2 != t and int(np.dot(c, n2)) == N:   # the point lies on tree t2 too
                        q = fco.sphere_point(t2, int(np.dot(c, a2)), int(np.dot(c, b2)))
                        assert np.array_equal(p, q)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_cell_area_is_spherical_excess(level):
    m = 8
    w2 = 2 * ((1 << (30 - level)) // m)
    ncell = (1 << level) * m
    rng = SplitMix64(level + 5)
    for t in range(6):
        # interior cells and ghost cells beyond a border (cells beyond a cube
        # corner have no place on the sphere and their capacity is never used)
        picks = [(int(rng.next_u64() % ncell), int(rng.next_u64() % ncell)) for _ in range(6)]
        picks += [(-1, 0), (-2, ncell - 1), (ncell, 2 % ncell), (1 % ncell, -2), (0, ncell + 1)]
        for i, j in picks:
            U0, V0 = i * w2 - N, j * w2 - N
            P = [fco.sphere_point(t, U0, V0), fco.sphere_point(t, U0 + w2, V0),
                 fco.sphere_point(t, U0 + w2, V0 + w2), fco.sphere_point(t, U0, V0 + w2)]
            ref = _girard(P)
            got = fco.sphere_cell_area(t, U0, U0 + w2, V0, V0 + w2)
            assert abs(got - ref) <= 1e-9 * ref, (t, i, j, got, ref)


def _sphere(level_lo, level_hi, m=8, tilt=math.pi / 4, omega=2 * math.pi, subcycle=0, refluxing=1,
            threshold=0.02):
    return Oracle(OracleParams(conn=fco.CONN_SPHERE, equation=fco.EQ_ADV, m=m, min_level=level_lo,
                               max_level=level_hi, omega=omega, omega_axis_tilt=tilt, cfl=0.9,
                               subcycle=subcycle, refluxing=refluxing, tag_threshold=threshold))


def test_areas_tile_the_sphere():
    for lev in (0, 2):
        o = _sphere(lev, lev)
        o.uniform(lev)
        o.set_fields(np.ones((o.n, 1, o.m, o.m)))
        assert abs(o.sums()[0] - 4 * math.pi) < 1e-12


def _cell_points(o):
    tr, lv, xs, ys = o.leaves()
    m = o.m
    P = np.zeros((o.n, m, m, 3))
    for k in range(o.n):
        w2 = 2 * ((1 << (30 - int(lv[k]))) // m)
        for j in range(m):
            for i in range(m):
                U = (int(xs[k]) * m + i) * w2 + w2 // 2 - N
                V = (int(ys[k]) * m + j) * w2 + w2 // 2 - N
                P[k, j, i] = fco.sphere_point(int(tr[k]), U, V)
    return P


def _cell_areas(o):
    tr, lv, xs, ys = o.leaves()
    m = o.m
    A = np.zeros((o.n, m, m))
    for k in range(o.n):
        w2 = 2 * ((1 << (30 - int(lv[k]))) // m)
        for j in range(m):
            for i in range(m):
                U0 = (int(xs[k]) * m + i) * w2 - N
                V0 = (int(ys[k]) * m + j) * w2 - N
                A[k, j, i] = fco.sphere_cell_area(int(tr[k]), U0, U0 + w2, V0, V0 + w2)
    return A


def _hill(P, lon0, lat0, width):
    c = np.array([math.cos(lat0) * math.cos(lon0), math.cos(lat0) * math.sin(lon0), math.sin(lat0)])
    d = 2.0 * np.arcsin(np.minimum(np.linalg.norm(P - c, axis=-1) / 2.0, 1.0))
    return np.exp(-(d / width) ** 2)


def test_hill_initial_values():
    o = _sphere(1, 1)
    o.uniform(1)
    o.init_fields(fco.INIT_HILL, [0.3, 0.2, 0.4])
    np.testing.assert_allclose(o.fields()[:, 0], _hill(_cell_points(o), 0.3, 0.2, 0.4), rtol=0, atol=1e-14)


def test_ghosts_across_tree_borders_hold_neighbour_cells():
    o = _sphere(1, 1)
    o.uniform(1)
    o.init_fields(fco.INIT_HILL, [0.3, 0.2, 0.9])
    pad = o.fill_ghosts()
    tr, lv, xs, ys = o.leaves()
    m = o.m
    checked = 0
    for k in range(o.n):
        w2 = 2 * ((1 << (30 - int(lv[k]))) // m)
        for j in range(-2, m + 2):
            for i in range(-2, m + 2):
                if 0 <= i < m and 0 <= j < m:
                    continue
                U = (int(xs[k]) * m + i) * w2 + w2 // 2 - N
                V = (int(ys[k]) * m + j) * w2 + w2 // 2 - N
                if abs(U) > N and abs(V) > N:
                    continue                      # beyond a cube corner: averaged rule
                ref = _hill(fco.sphere_point(int(tr[k]), U, V)[None], 0.3, 0.2, 0.9)[0]
                assert abs(pad[k, 0, j + 2, i + 2] - ref) < 1e-14
                checked += 1
    assert checked > 1000


def _mass_rel(o, s0):
    return abs(o.sums()[0] - s0) / abs(s0)


@pytest.mark.parametrize("subcycle", [0, 1])
def test_mass_conserved_adaptive(subcycle):
    o = _sphere(1, 3, subcycle=subcycle)
    o.init_refine(fco.INIT_HILL, [0.5, 0.3, 0.35])
    levels = set(o.leaves()[1].tolist())
    assert len(levels) >= 2
    s0 = o.sums()[0]
    for _ in range(3):
        o.advance(2)
        assert _mass_rel(o, s0) < 1e-13
        assert o.last_courant <= 0.9 * (1 + 1e-12)
        o.regrid(o.tag())
        assert _mass_rel(o, s0) < 1e-13


def test_regrid_conserves_mass_both_ways():
    o = _sphere(1, 3)
    o.uniform(2)
    o.init_fields(fco.INIT_HILL, [1.0, -0.4, 0.5])
    s0 = o.sums()[0]
    rng = SplitMix64(3)
    for _ in range(4):
        fl = np.array([(int(rng.next_u64() % 3) - 1) for _ in range(o.n)], np.int8)
        o.regrid(fl)
        assert _mass_rel(o, s0) < 1e-13


def _revolution(level, width=0.5, tilt=math.pi / 4, T=1.0):
    o = _sphere(level, level, tilt=tilt)
    o.uniform(level)
    o.init_fields(fco.INIT_HILL, [0.3, 0.2, width])
    q0 = o.fields()[:, 0].copy()
    while o.time < T - 1e-12:
        o.advance(1, min(o.next_dt, T - o.time))
    return o, q0


def test_one_revolution_returns_and_converges():
    errs = []
    for lev in (1, 2):
        o, q0 = _revolution(lev)
        A = _cell_areas(o)
        errs.append(float((np.abs(o.fields()[:, 0] - q0) * A).sum() / (np.abs(q0) * A).sum()))
    assert errs[1] < 0.15 and errs[1] < errs[0] / 2.5, errs


def test_quarter_turn_is_counterclockwise_about_the_axis():
    o, _ = _revolution(1, width=0.4, tilt=0.0, T=0.25)
    q = o.fields()[:, 0]
    P = _cell_points(o)
    A = _cell_areas(o)
    c = (P * (q * A)[..., None]).sum(axis=(0, 1, 2))
    lon = math.atan2(c[1], c[0])
    assert abs(lon - (0.3 + math.pi / 2)) < 0.05, lon


def test_freestream_exact_without_correction():
    """a constant stays exactly constant: every fluctuation vanishes, every
    ghost rule (copy, 2x2 average, limited interpolation, corner mean) returns
    the constant"""
    o = _sphere(1, 3, subcycle=1, refluxing=0)
    o.init_refine(fco.INIT_HILL, [0.5, 0.3, 0.35])     # adaptive forest from the hill
    o.set_fields(np.full((o.n, 1, o.m, o.m), 1.25))
    o.advance(6)
    assert np.all(o.fields() == 1.25)


def test_freestream_to_roundoff_with_correction_and_regrid():
    o = _sphere(1, 3, subcycle=1)
    o.init_refine(fco.INIT_HILL, [0.5, 0.3, 0.35])
    o.set_fields(np.full((o.n, 1, o.m, o.m), 1.25))
    o.advance(4)
    o.regrid(SplitMix64_flags(o.n, 9))
    o.advance(2)
    assert np.max(np.abs(o.fields() - 1.25)) < 1e-13


def SplitMix64_flags(n, seed):
    rng = SplitMix64(seed)
    return np.array([(int(rng.next_u64() % 3) - 1) for _ in range(n)], np.int8)
