"""Pins of the oracle's two-tree sphere (Sec. 5, Example 2: two quadtrees on
[-1,1]^2, one per hemisphere; solid-body rotation of a field that is 0 on one
half of the sphere and 1 on the other).

The map is the oracle's reading (concentric squares to circles of colatitude
pi r / 2; tree 1 mirrored in x; x borders continue into the other tree, y
borders meet the other tree with a half turn).  Pinned against what the
geometry and the mathematics fix: the sphere's area, a closed form of a
cell's area through the sine integral (scipy), additivity under refinement,
brute-force triangulation, bitwise-shared border points, the neighbour
relation against the shared edges' end points, and for the solver: an exactly
steady case, freestream and mass through coarse-fine borders at every
singular corner (with the correction visibly needed), and convergence over
one revolution.
"""
import math

import numpy as np
import pytest

from oracle import fco
from oracle.fco import Oracle, OracleParams

N = 1 << 30


def _mk(lo, hi, m=8, subcycle=0, refluxing=1, tilt=math.pi / 4, thr=0.002):
    return Oracle(OracleParams(conn=fco.CONN_PILLOW, equation=fco.EQ_ADV, m=m, min_level=lo, max_level=hi,
                               omega=2 * math.pi, omega_axis_tilt=tilt, cfl=0.9, subcycle=subcycle,
                               refluxing=refluxing, tag_threshold=thr, tag_crit=fco.TAG_MAXMIN))


def _morton(x, y):
    return sum((((x >> b) & 1) << (2 * b)) | (((y >> b) & 1) << (2 * b + 1)) for b in range(16))


def _two_levels(o, l0, l1):
    """tree 0 uniform at level l0, tree 1 at level l1"""
    tr, lv, xs, ys = [], [], [], []
    for t, lev in ((0, l0), (1, l1)):
        w = 1 << lev
        for x, y in sorted(((x, y) for y in range(w) for x in range(w)), key=lambda c: _morton(*c)):
            tr.append(t); lv.append(lev); xs.append(x); ys.append(y)
    o.set_leaves(tr, lv, xs, ys)


def _areas(o):
    tr, lv, x, y = o.leaves()
    m = o.m
    A = np.zeros((o.n, m, m))
    for k in range(o.n):
        w2 = 2 * ((1 << (30 - int(lv[k]))) // m)
        for j in range(m):
            for i in range(m):
                U0 = int(x[k]) * m * w2 + i * w2 - N
                V0 = int(y[k]) * m * w2 + j * w2 - N
                A[k, j, i] = fco.pillow_cell_area(int(tr[k]), U0, U0 + w2, V0, V0 + w2)
    return A


# ---- geometry ---------------------------------------------------------------

def test_areas_sum_to_the_sphere_and_each_tree_to_a_hemisphere():
    for L in (0, 3):
        w = 2 * N >> L
        per_tree = []
        for t in (0, 1):
            s = math.fsum(fco.pillow_cell_area(t, -N + i * w, -N + (i + 1) * w, -N + j * w, -N + (j + 1) * w)
                          for j in range(1 << L) for i in range(1 << L))
            per_tree.append(s)
        assert abs(per_tree[0] - 2 * math.pi) < 1e-14 and abs(per_tree[1] - 2 * math.pi) < 1e-14
        assert abs(sum(per_tree) - 4 * math.pi) < 2e-14


def test_cell_area_inside_one_sector_is_the_sine_integral():
    """inside x >= |y| the area element is (pi^2/8) sin(pi x / 2) / x, so a
    cell's area is (pi^2/8) (y1 - y0) (Si(pi x1 / 2) - Si(pi x0 / 2))"""
    from scipy.special import sici
    for (x0, x1, y0, y1) in [(0.5, 0.625, -0.25, 0.125), (0.75, 1.0, 0.5, 0.75), (0.25, 0.5, -0.25, 0.25)]:
        want = math.pi ** 2 / 8 * (y1 - y0) * (sici(math.pi * x1 / 2)[0] - sici(math.pi * x0 / 2)[0])
        for t in (0, 1):
            got = fco.pillow_cell_area(t, int(x0 * N), int(x1 * N), int(y0 * N), int(y1 * N))
            assert got == pytest.approx(want, rel=2e-15)
        # the same cell turned a quarter (sector y >= |x|) has the same area
        got = fco.pillow_cell_area(0, int(y0 * N), int(y1 * N), int(x0 * N), int(x1 * N))
        assert got == pytest.approx(want, rel=2e-15)


def test_cell_areas_are_additive_under_refinement():
    rng = np.random.default_rng(3)
    for _ in range(40):
        L = int(rng.integers(0, 6))
        w = 2 * N >> L
        i, j, t = int(rng.integers(0, 1 << L)), int(rng.integers(0, 1 << L)), int(rng.integers(0, 2))
        U0, V0 = -N + i * w, -N + j * w
        parent = fco.pillow_cell_area(t, U0, U0 + w, V0, V0 + w)
        h = w // 2
        kids = math.fsum(fco.pillow_cell_area(t, U0 + a * h, U0 + (a + 1) * h, V0 + b * h, V0 + (b + 1) * h)
                         for a in (0, 1) for b in (0, 1))
        assert parent == pytest.approx(kids, rel=4e-16, abs=0)


def _tri(a, b, c):
    return 2 * math.atan2(abs(np.dot(a, np.cross(b, c))), 1 + a @ b + b @ c + c @ a)


def _brute_area(t, U0, U1, V0, V1, k):
    us = [U0 + (U1 - U0) * i // k for i in range(k + 1)]
    vs = [V0 + (V1 - V0) * j // k for j in range(k + 1)]
    P = [[fco.pillow_point(t, u, v) for u in us] for v in vs]
    return sum(_tri(P[j][i], P[j][i + 1], P[j + 1][i + 1]) + _tri(P[j][i], P[j + 1][i + 1], P[j + 1][i])
               for j in range(k) for i in range(k))


def test_cell_area_is_the_limit_of_triangulations_of_the_mapped_cell():
    """cells across a diagonal kink, at a tree corner, and across an axis"""
    for (t, U0, U1, V0, V1) in [(0, -N // 8, 3 * N // 8, -N // 8, 3 * N // 8), (1, N // 2, N, N // 2, N),
                                (0, -N, -N // 2, 0, N // 2)]:
        a = fco.pillow_cell_area(t, U0, U1, V0, V1)
        e1 = abs(_brute_area(t, U0, U1, V0, V1, 32) - a)
        e2 = abs(_brute_area(t, U0, U1, V0, V1, 64) - a)
        assert e2 < 2e-4 * a and e2 < 0.3 * e1          # second-order convergence onto the area


def test_points_on_the_sphere_and_border_points_shared_bitwise():
    for Y in range(-N, N + 1, N // 16):
        for X in range(-N, N + 1, N // 16):
            p0, p1 = fco.pillow_point(0, X, Y), fco.pillow_point(1, X, Y)
            assert abs(p0 @ p0 - 1) < 1e-15 and abs(p1 @ p1 - 1) < 1e-15
            assert p0[2] >= 0.0 and p1[2] <= 0.0
        # tree 0's x borders continue into tree 1's; y borders meet with a half turn
        assert np.array_equal(fco.pillow_point(0, N, Y), fco.pillow_point(1, -N, Y))
        assert np.array_equal(fco.pillow_point(0, -N, Y), fco.pillow_point(1, N, Y))
        assert np.array_equal(fco.pillow_point(0, Y, N), fco.pillow_point(1, -Y, N))
        assert np.array_equal(fco.pillow_point(0, Y, -N), fco.pillow_point(1, -Y, -N))
        assert fco.pillow_point(0, N, Y)[2] == 0.0
    assert np.array_equal(fco.pillow_point(0, 0, 0), [0.0, 0.0, 1.0])
    assert np.array_equal(fco.pillow_point(1, 0, 0), [0.0, 0.0, -1.0])


def test_crossing_a_border_mirrors_through_the_equator():
    """the map continued beyond a tree border (x border: the other tree, x
    continued; y border: the other tree with a half turn) lands on the mirror
    image, through the equatorial plane, of the point as far inside"""
    mirror = np.array([1.0, 1.0, -1.0])
    for t in (0, 1):
        for V in range(-N + N // 32, N, N // 16):
            for e in (1, N // 1024, N // 8):
                assert np.array_equal(fco.pillow_point(t, N + e, V), mirror * fco.pillow_point(t, N - e, V))
                assert np.array_equal(fco.pillow_point(t, -N - e, V), mirror * fco.pillow_point(t, -N + e, V))
                assert np.array_equal(fco.pillow_point(t, V, N + e), mirror * fco.pillow_point(t, V, N - e))
                assert np.array_equal(fco.pillow_point(t, V, -N - e), mirror * fco.pillow_point(t, V, -N + e))
    for (t, U, V) in [(0, N + N // 4, N // 3), (1, -N - N // 8, -N // 2), (0, N // 5, N + N // 16)]:
        t2, U2, V2 = fco.pillow_fold(t, U, V)
        assert t2 == 1 - t and -N <= U2 <= N and -N <= V2 <= N
    # beyond both borders at a corner: the same tree, reflected through the corner
    assert fco.pillow_fold(0, N + 6, N + 10) == (0, N - 6, N - 10)


def _edge_nodes(tr, lv, x, y, side):
    """sphere points of the two end nodes of a leaf's side"""
    w2 = 2 * N >> int(lv)
    U0, V0 = -N + int(x) * w2, -N + int(y) * w2
    ends = {0: [(U0, V0), (U0, V0 + w2)], 1: [(U0 + w2, V0), (U0 + w2, V0 + w2)],
            2: [(U0, V0), (U0 + w2, V0)], 3: [(U0, V0 + w2), (U0 + w2, V0 + w2)]}[side]
    return {tuple(fco.pillow_point(int(tr), U, V)) for U, V in ends}


@pytest.mark.parametrize("levels", [(2, 2), (1, 2), (2, 1)])
def test_neighbour_table_against_shared_edges(levels):
    """every same-level side neighbour shares the side's two end nodes (as
    sphere points, bit for bit) with one of its own sides that lists this
    leaf back; finer neighbours' sides lie on the side; no boundary"""
    o = _mk(1, 2)
    _two_levels(o, *levels)
    tr, lv, x, y = o.leaves()
    nb = o.neighbors()
    assert not np.any(nb[:, :, 0] == fco.NB_NONE)
    for k in range(o.n):
        for d in range(4):
            kind, a = nb[k, d, 0], nb[k, d, 1]
            mine = _edge_nodes(tr[k], lv[k], x[k], y[k], d)
            if kind == fco.NB_SAME:
                back = [d2 for d2 in range(4) if nb[a, d2, 0] == fco.NB_SAME and nb[a, d2, 1] == k and
                        _edge_nodes(tr[a], lv[a], x[a], y[a], d2) == mine]
                assert len(back) == 1, (k, d)
            elif kind == fco.NB_FINER:
                for f in (nb[k, d, 1], nb[k, d, 2]):
                    assert any(len(_edge_nodes(tr[f], lv[f], x[f], y[f], d2) & mine) == 1 and
                               nb[f, d2, 0] == fco.NB_COARSER and nb[f, d2, 1] == k for d2 in range(4)), (k, d)
            else:
                assert kind == fco.NB_COARSER and lv[a] == lv[k] - 1


# ---- the solver on the two-tree sphere -------------------------------------

def test_equator_split_under_rotation_about_the_pole_is_steady():
    """q = 1 on the northern tree, 0 on the southern one, rotation about z:
    no flux crosses the equator (both end nodes of every border edge have
    z = 0 exactly) and each tree is a constant state"""
    o = _mk(2, 2, tilt=0.0)
    o.uniform(2)
    o.init_fields(fco.INIT_HALF, [0.0, math.pi / 2])
    q0 = o.fields()
    tr = o.leaves()[0]
    assert np.all(q0[tr == 0] == 1.0) and np.all(q0[tr == 1] == 0.0)
    o.advance(6)
    assert np.abs(o.fields() - q0).max() <= 1e-15


@pytest.mark.parametrize("subcycle", [0, 1])
def test_coarse_fine_at_every_singular_corner(subcycle):
    """tree 0 one level coarser than tree 1: every border between the trees,
    the four singular corners included, is coarse-fine"""
    o = _mk(1, 2, subcycle=subcycle)
    _two_levels(o, 1, 2)
    o.set_fields(np.full((o.n, 1, o.m, o.m), 0.75))
    o.advance(5)
    assert np.abs(o.fields() - 0.75).max() <= 1e-15              # freestream
    o.init_fields(fco.INIT_HALF, [0.3, 0.4])
    s0 = o.sums()[0]
    o.advance(5)
    assert abs(o.sums()[0] - s0) <= 1e-14 * abs(s0)             # mass with the correction
    p = _mk(1, 2, subcycle=subcycle, refluxing=0)
    _two_levels(p, 1, 2)
    p.init_fields(fco.INIT_HALF, [0.3, 0.4])
    p.advance(5)
    assert abs(p.sums()[0] - s0) > 1e-6 * abs(s0)               # and without it, visibly not


@pytest.mark.parametrize("subcycle", [0, 1])
def test_example_2_mass_through_steps_and_regrids(subcycle):
    o = _mk(1, 3, subcycle=subcycle, thr=0.05)
    o.init_refine(fco.INIT_HALF, [0.4, 0.5])
    assert len(set(o.leaves()[1].tolist())) > 1
    s0 = o.sums()[0]
    forests = {o.n}
    for _ in range(3):
        o.advance(2)
        o.regrid(o.tag())
        forests.add(o.n)
        assert abs(o.sums()[0] - s0) <= 1e-14 * abs(s0)
    q = o.fields()
    assert q.min() > -0.2 and q.max() < 1.2                      # limited scheme, 0/1 data


def test_one_revolution_converges():
    errs = []
    for lev in (1, 2, 3):
        o = _mk(lev, lev)
        o.uniform(lev)
        o.init_fields(fco.INIT_HILL, [0.5, 0.3, 0.35])
        q0 = o.fields()[:, 0].copy()
        s0 = o.sums()[0]
        while o.time < 1.0 - 1e-12:
            o.advance(1, min(o.next_dt, 1.0 - o.time))
        assert abs(o.sums()[0] - s0) <= 1e-14 * abs(s0)
        A = _areas(o)
        errs.append(float((A * np.abs(o.fields()[:, 0] - q0)).sum() / (A * np.abs(q0)).sum()))
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 3.5 and errs[2] < 0.05
