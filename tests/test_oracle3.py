"""Pins of the three-dimensional oracle (octree of m^3 patches, scalar
advection with a constant velocity, periodic unit cube).

The paper states the method for d = 2 and 3 and shows only 2D results, so
the 3D scheme is the 2D one with transverse terms in both perpendicular
directions plus corner (double-transverse) terms.  What pins it:
  * with the limiter off it equals the tensor-product upwind step
    prod_d (1 - nu_d D_d) exactly, for every sign pattern of the velocity
    (the corner terms are what makes it so: without them it differs);
  * Courant number 1 along an axis translates the data by one cell, bit for
    bit; a constant state stays constant bit for bit on an adaptive forest;
  * planar data give the 1D scheme bit for bit whatever the transverse
    speeds; smooth data converge at second order;
  * permuting the axes (data, forest and velocity) permutes the result;
  * mass is conserved to round-off on adaptive forests with the coarse-fine
    correction and visibly not without it;
  * 2:1 balance against a brute-force ripple over all touching pairs; ghost
    cells reproduce a linear field; regrid conserves mass and a refine /
    coarsen round trip returns the data; max - min flags against numpy.
"""
import itertools

import numpy as np
import pytest

from oracle.fco3 import ERR_CFL, ERR_UNBALANCED, INIT_GAUSS, INIT_SINE, Oracle3, Oracle3Error, Oracle3Params

rng = np.random.default_rng(20240)


def _uniform(m, level, **kw):
    return Oracle3(Oracle3Params(m=m, min_level=level, max_level=level, **kw))


def _scatter(o, G):
    """global uniform grid (finest level of a uniform forest) -> leaf fields"""
    lv, x, y, z = o.leaves()
    m = o.m
    q = np.zeros((o.n, m, m, m))
    for k in range(o.n):
        q[k] = G[z[k] * m:(z[k] + 1) * m, y[k] * m:(y[k] + 1) * m, x[k] * m:(x[k] + 1) * m]
    return q


def _tensor_upwind(G, nu):
    """prod over axes of (1 - nu_d D_d), D_d the upwind difference; array axes (z, y, x)"""
    R = G.copy()
    for d, n in enumerate(nu):
        ax = 2 - d
        if n >= 0:
            R = (1 - n) * R + n * np.roll(R, 1, axis=ax)
        else:
            R = (1 + n) * R - n * np.roll(R, -1, axis=ax)
    return R


@pytest.mark.parametrize("vel", [(0.3, 0.5, 0.7), (-0.3, 0.5, -0.7), (0.6, -0.2, 0.9), (-0.8, -0.1, -0.4)])
def test_first_order_is_tensor_product_upwind(vel):
    m, lev = 4, 1
    o = _uniform(m, lev, limiter=0, transverse=2, u=vel[0], v=vel[1], w=vel[2])
    N = m << lev
    G = rng.standard_normal((N, N, N))
    o.set_fields(_scatter(o, G))
    dx = 1.0 / N
    dt = 0.9 * dx
    o.advance(1, dt)
    ref = _tensor_upwind(G, [v * dt / dx for v in vel])
    np.testing.assert_allclose(o.grid(), ref, rtol=0, atol=1e-14)


def test_corner_terms_are_needed():
    m, lev, vel = 4, 1, (0.3, 0.5, 0.7)
    o = _uniform(m, lev, limiter=0, transverse=1, u=vel[0], v=vel[1], w=vel[2])
    N = m << lev
    G = rng.standard_normal((N, N, N))
    o.set_fields(_scatter(o, G))
    o.advance(1, 0.9 / N)
    assert np.abs(o.grid() - _tensor_upwind(G, [0.9 * v for v in vel])).max() > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_courant_one_translates_bitexact(axis):
    m, lev = 4, 2
    vel = [0.0, 0.0, 0.0]
    vel[axis] = 1.0
    o = _uniform(m, lev, u=vel[0], v=vel[1], w=vel[2])
    N = m << lev
    G = 1.0 + rng.random((N, N, N))           # values in [1, 2): exact differences
    o.set_fields(_scatter(o, G))
    o.advance(1, 1.0 / N)
    assert np.array_equal(o.grid(), np.roll(G, 1, axis=2 - axis))


def _amr(m=4, lmin=2, lmax=4, **kw):
    """three levels: 37 / 189 / 216 leaves at levels 2 / 3 / 4 (on a level-1
    grid every patch touches every other through the periodic wrap, so one
    fine leaf would refine them all)"""
    o = Oracle3(Oracle3Params(m=m, min_level=lmin, max_level=lmax, tag_threshold=0.02, **kw))
    o.init_refine(INIT_GAUSS, [0.0, 1.0, 0.3, 0.3, 0.3, 0.08])
    return o


def test_constant_state_stays_constant_on_amr():
    o = _amr(u=0.6, v=-0.5, w=0.4)
    assert len(set(o.leaves()[0])) == 3
    o.set_fields(np.full((o.n, o.m, o.m, o.m), 1.25))
    o.advance(4)
    assert np.all(o.fields() == 1.25)


def _mc(th):
    return np.maximum(0.0, np.minimum(np.minimum((1.0 + th) / 2.0, 2.0), 2.0 * th))


def _step1d(q, u, k):
    """1D wave propagation with the MC limiter, periodic (the 1D form of the same method)"""
    W = q - np.roll(q, 1)                                  # wave at face i - 1/2
    ap, am = max(u, 0.0) * W, min(u, 0.0) * W
    Wu = np.roll(W, 1) if u >= 0 else np.roll(W, -1)
    with np.errstate(divide="ignore", invalid="ignore"):
        th = np.where(W != 0.0, Wu / np.where(W != 0.0, W, 1.0), 0.0)
    F = np.where(W != 0.0, 0.5 * abs(u) * (1.0 - k * abs(u)) * _mc(th) * W, 0.0)
    fl = ap + np.roll(am, -1)
    return q - k * (fl + (np.roll(F, -1) - F))


@pytest.mark.parametrize("vel", [(0.7, 0.4, -0.3), (-0.5, -0.6, 0.2)])
def test_planar_data_give_the_1d_scheme_bitexact(vel):
    m, lev = 4, 2
    o = _uniform(m, lev, u=vel[0], v=vel[1], w=vel[2])
    N = m << lev
    xc = (np.arange(N) + 0.5) / N
    q1 = 1.0 + 0.5 * np.sin(2 * np.pi * xc) + (xc > 0.5)
    o.set_fields(_scatter(o, np.broadcast_to(q1, (N, N, N)).copy()))
    dt = 0.8 / N
    o.advance(3, dt)
    ref = q1.copy()
    for _ in range(3):
        ref = _step1d(ref, vel[0], dt * N)
    assert np.array_equal(o.grid(), np.broadcast_to(ref, (N, N, N)))


def _sine_error(m, lev, T):
    vel = (1.0, 0.5, -0.5)
    o = _uniform(m, lev, u=vel[0], v=vel[1], w=vel[2])
    o.init(INIT_SINE, [1.0, 0.5, 1.0, 1.0, 1.0])
    N = m << lev
    steps = int(np.ceil(T / (0.8 / N)))
    o.advance(steps, T / steps)
    c = (np.arange(N) + 0.5) / N
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    ex = 1.0 + 0.5 * np.sin(2 * np.pi * ((X - vel[0] * T) + (Y - vel[1] * T) + (Z - vel[2] * T)))
    return np.abs(o.grid() - ex).mean()


def test_second_order_convergence_on_smooth_data():
    e = np.array([_sine_error(4, lev, 0.25) for lev in (2, 3, 4)])
    rates = np.log2(e[:-1] / e[1:])
    assert rates.min() > 1.8, (e, rates)


def test_axis_permutation_permutes_the_result():
    vel = (0.6, -0.3, 0.45)
    a = _amr(u=vel[0], v=vel[1], w=vel[2])
    lv, x, y, z = a.leaves()
    q = a.fields()
    # new axes: x' = y, y' = z, z' = x
    b = Oracle3(Oracle3Params(m=4, min_level=2, max_level=4, tag_threshold=0.02, u=vel[1], v=vel[2], w=vel[0]))
    order = sorted(range(len(lv)), key=lambda k: _key(lv[k], y[k], z[k], x[k]))
    b.set_leaves(lv[order], y[order], z[order], x[order])
    b.set_fields(np.stack([np.transpose(q[k], (2, 0, 1)) for k in order]))
    a.advance(3)
    b.advance(3)
    ga, gb = a.grid(), b.grid()
    np.testing.assert_allclose(np.transpose(ga, (2, 0, 1)), gb, rtol=0, atol=1e-14)


def _key(l, x, y, z, L=20):
    s = L - int(l)
    k = 0
    for b in range(L):
        k |= ((int(x) << s >> b) & 1) << (3 * b)
        k |= ((int(y) << s >> b) & 1) << (3 * b + 1)
        k |= ((int(z) << s >> b) & 1) << (3 * b + 2)
    return k


@pytest.mark.parametrize("refluxing", [1, 0])
def test_mass_conservation_on_amr(refluxing):
    o = _amr(u=0.7, v=0.4, w=-0.55, refluxing=refluxing)
    s0 = o.sum()
    for _ in range(2):
        o.advance(3)
        o.regrid(o.tag())
    drift = abs(o.sum() - s0) / abs(s0)
    if refluxing:
        assert drift < 2e-14, drift
    else:
        assert drift > 1e-8, drift


# ---------------------------------------------------------------- forest
def _touch(a, b):
    """leaves (l, x, y, z) touch (face, edge or corner; periodic) and are distinct"""
    la, lb = a[0], b[0]
    L = max(la, lb)
    n = 1 << L
    lo_a = [c << (L - la) for c in a[1:]]
    lo_b = [c << (L - lb) for c in b[1:]]
    wa, wb = 1 << (L - la), 1 << (L - lb)
    inside = True
    for d in range(3):
        ok = False
        for sh in (-n, 0, n):
            if lo_b[d] + sh <= lo_a[d] + wa and lo_a[d] <= lo_b[d] + sh + wb:
                ok = True
        inside &= ok
    return inside and a != b


def _brute_balance(leaves, lmax):
    leaves = set(leaves)
    while True:
        bad = None
        for a, b in itertools.combinations(sorted(leaves), 2):
            if abs(a[0] - b[0]) > 1 and _touch(a, b):
                bad = a if a[0] < b[0] else b
                break
        if bad is None:
            return leaves
        leaves.remove(bad)
        l, x, y, z = bad
        for c in range(8):
            leaves.add((l + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c >> 2)))


def _random_forest(seed, lmax=3):
    r = np.random.default_rng(seed)
    leaves = [(1, x, y, z) for z in range(2) for y in range(2) for x in range(2)]
    for _ in range(3):
        nxt = []
        for lf in leaves:
            if lf[0] < lmax and r.random() < 0.3:
                l, x, y, z = lf
                nxt += [(l + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c >> 2)) for c in range(8)]
            else:
                nxt.append(lf)
        leaves = nxt
    return leaves


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_balance_against_brute_force(seed):
    """the coarsest 2:1-balanced refinement is unique: the oracle's ripple
    (run by every regrid) must give the brute-force one"""
    leaves = _random_forest(seed)
    ref = _brute_balance(leaves, 4)
    srt = sorted(leaves, key=lambda t: _key(*t))
    lv, x, y, z = (np.array([t[i] for t in srt]) for i in range(4))
    o = Oracle3(Oracle3Params(m=4, min_level=0, max_level=4))
    if ref == set(leaves):
        o.set_leaves(lv, x, y, z)
    else:
        with pytest.raises(Oracle3Error) as ei:
            o.set_leaves(lv, x, y, z)
        assert ei.value.rc == ERR_UNBALANCED
    # reach the input by refining the ancestors of its leaves level by level
    o.uniform(1)
    for lev in (1, 2):
        lv3, x3, y3, z3 = o.leaves()
        inner = {(t[1] >> (t[0] - lev), t[2] >> (t[0] - lev), t[3] >> (t[0] - lev)) for t in leaves if t[0] > lev}
        flags = np.array([1 if lv3[k] == lev and (x3[k], y3[k], z3[k]) in inner else 0 for k in range(o.n)], np.int8)
        o.set_fields(np.zeros((o.n, 4, 4, 4)))
        o.regrid(flags)
    got = set(zip(*(a.tolist() for a in o.leaves())))
    assert got == ref
    assert o.is_balanced()


def test_linear_field_ghosts_exact():
    o = Oracle3(Oracle3Params(m=4, min_level=2, max_level=4, tag_threshold=0.02))
    o.init_refine(INIT_GAUSS, [0.0, 1.0, 0.5, 0.5, 0.5, 0.12])
    lv, x, y, z = o.leaves()
    assert len(set(lv)) == 3
    m = o.m
    a, b, c, d = 0.3, 1.1, -0.7, 0.45
    q = np.zeros((o.n, m, m, m))
    for k in range(o.n):
        dx = 1.0 / (m << lv[k])
        cc = (np.arange(m) + 0.5) * dx
        Z, Y, X = np.meshgrid(z[k] * m * dx + cc, y[k] * m * dx + cc, x[k] * m * dx + cc, indexing="ij")
        q[k] = a + b * X + c * Y + d * Z
    o.set_fields(q)
    T = o.tiles()
    checked = 0
    for k in range(o.n):
        w = 1 << lv[k]
        if min(x[k], y[k], z[k]) == 0 or max(x[k], y[k], z[k]) == w - 1:
            continue                           # periodic wrap breaks the linear field
        dx = 1.0 / (m << lv[k])
        cc = (np.arange(-2, m + 2) + 0.5) * dx
        Z, Y, X = np.meshgrid(z[k] * m * dx + cc, y[k] * m * dx + cc, x[k] * m * dx + cc, indexing="ij")
        np.testing.assert_allclose(T[k], a + b * X + c * Y + d * Z, rtol=0, atol=1e-13)
        checked += 1
    assert checked > 10


def test_regrid_conserves_and_round_trips():
    o = Oracle3(Oracle3Params(m=4, min_level=1, max_level=2))
    o.init(INIT_GAUSS, [0.2, 1.0, 0.5, 0.4, 0.6, 0.25])
    q0, s0 = o.fields(), o.sum()
    o.regrid(np.ones(o.n, np.int8))
    assert o.n == 64 and abs(o.sum() - s0) <= 1e-15 * abs(s0)
    o.regrid(-np.ones(o.n, np.int8))
    assert o.n == 8 and abs(o.sum() - s0) <= 1e-15 * abs(s0)
    np.testing.assert_allclose(o.fields(), q0, rtol=0, atol=1e-15)


def test_tag_flags_against_numpy():
    o = _amr()
    f = o.tag()
    lv, x, y, z = o.leaves()
    q = o.fields()
    mm = q.reshape(o.n, -1).max(1) - q.reshape(o.n, -1).min(1)
    thr = o.params.tag_threshold
    assert np.array_equal(f == 1, (mm > thr) & (lv < 4))
    assert np.any(f == -1)
    for k in np.nonzero(f == -1)[0]:
        assert mm[k] <= thr and lv[k] > 2


def test_courant_above_one_refused():
    o = _uniform(4, 1, u=1.0)
    with pytest.raises(Oracle3Error) as ei:
        o.advance(1, 1.01 / 8)
    assert ei.value.rc == ERR_CFL


# ------------------------------------------------------------ sub-cycling
def test_subcycling_on_one_level_is_the_global_step_bitexact():
    m, lev, vel = 4, 2, (0.6, -0.4, 0.5)
    a = _uniform(m, lev, u=vel[0], v=vel[1], w=vel[2])
    b = Oracle3(Oracle3Params(m=m, min_level=lev, max_level=lev, u=vel[0], v=vel[1], w=vel[2], subcycle=1))
    q = rng.standard_normal((a.n, m, m, m))
    a.set_fields(q)
    b.set_fields(q)
    a.advance(3)
    b.advance(3)
    assert np.array_equal(a.fields(), b.fields())


def test_subcycled_mass_conservation_and_constant_state():
    o = _amr(u=0.7, v=0.4, w=-0.55, subcycle=1)
    assert len(set(o.leaves()[0])) == 3
    s0 = o.sum()
    for _ in range(2):
        o.advance(2)
        o.regrid(o.tag())
    assert abs(o.sum() - s0) <= 2e-14 * abs(s0)
    o.set_fields(np.full((o.n, o.m, o.m, o.m), 1.25))
    o.advance(2)
    assert np.all(o.fields() == 1.25)


def test_subcycled_step_is_limited_by_the_coarsest_level():
    o = _amr(u=1.0, subcycle=1)
    g = _amr(u=1.0)
    lv = o.leaves()[0]
    assert o.next_dt == pytest.approx(0.9 / (4 << int(lv.min())), rel=1e-15)
    assert g.next_dt == pytest.approx(0.9 / (4 << int(lv.max())), rel=1e-15)
    with pytest.raises(Oracle3Error) as ei:
        o.advance(1, 1.01 / (4 << int(lv.min())))
    assert ei.value.rc == ERR_CFL


def test_subcycled_and_global_runs_agree_on_smooth_data():
    """same forest, same final time: the two time-stepping strategies differ
    by much less than either differs from the initial state"""
    vel = (0.5, 0.3, -0.4)
    a = _amr(u=vel[0], v=vel[1], w=vel[2])
    b = _amr(u=vel[0], v=vel[1], w=vel[2], subcycle=1)
    q0 = a.fields()
    T = 8 * a.next_dt
    a.advance(8)
    steps = int(round(T / b.next_dt))
    b.advance(steps, T / steps)
    assert abs(a.time - b.time) < 1e-15
    qa, qb = a.fields(), b.fields()
    moved = np.abs(qa - q0).sum()
    assert np.abs(qa - qb).sum() < 0.05 * moved
