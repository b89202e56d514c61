"""Pins of the oracle's patch numerics, ghost fill, regrid and time stepping.

Each pin is fixed by mathematics, not by the oracle itself:
  * lake at rest is preserved bit for bit, across coarse-fine faces and regrid;
  * mass is conserved to roundoff on AMR forests with the coarse-fine
    correction on (and visibly not without it: the correction is needed);
  * momentum too on the periodic square;
  * at Courant number 1 with u = 1, v = 0 the profile moves one cell per step
    exactly (the correction factor 1 - |s| dt/dx vanishes);
  * 16 patches at one level give bit for bit the same result as one patch
    covering the domain whose ghost ring is filled here by numpy reflection;
  * the radial dam break keeps the square's D4 symmetry;
  * ghost values reproduce linear fields across coarse-fine faces (fine to
    coarse averages and unlimited coarse to fine slopes are exact for them);
  * regrid conserves mass, refine-then-coarsen returns the data;
  * tag flags equal a numpy evaluation of the criterion;
  * sub-cycling on a single-level forest equals global stepping bit for bit;
  * smooth advection converges at second order.
"""
import numpy as np
import pytest

from oracle import fco
from oracle.fco import Oracle, OracleParams
from fc_inputs import dambreak_params, humps_params, random_forest_flags


def amr_dambreak(subcycle=0, refluxing=1, m=8, lmin=3, lmax=5, conn=fco.CONN_SQUARE, thr=0.05):
    o = Oracle(OracleParams(conn=conn, m=m, min_level=lmin, max_level=lmax, subcycle=subcycle,
                            refluxing=refluxing, tag_threshold=thr))
    o.init_refine(fco.INIT_DAMBREAK, dambreak_params())
    return o


def test_init_refine_makes_multilevel_balanced_forest():
    o = amr_dambreak()
    _, lv, _, _ = o.leaves()
    assert set(lv.tolist()) == {3, 4, 5}
    assert o.is_balanced()


@pytest.mark.parametrize("subcycle", [0, 1])
def test_lake_at_rest_bitwise(subcycle):
    o = amr_dambreak(subcycle=subcycle)
    q = o.fields()
    q[:, 0] = 1.375
    q[:, 1:] = 0.0
    o.set_fields(q)
    for _ in range(3):
        o.advance(2)
        o.regrid(random_forest_flags(o.n, 7))
    q2 = o.fields()
    assert np.all(q2[:, 0] == 1.375) and np.all(q2[:, 1:] == 0.0)


@pytest.mark.parametrize("subcycle", [0, 1])
def test_mass_conserved_amr(subcycle):
    o = amr_dambreak(subcycle=subcycle)
    s0 = o.sums()
    for _ in range(5):
        o.advance(4)
        o.regrid(o.tag())
    s1 = o.sums()
    assert abs(s1[0] - s0[0]) / s0[0] < 1e-13
    # reflecting walls: momentum stays ~0 by symmetry of the centred dam break
    assert abs(s1[1]) < 1e-12 and abs(s1[2]) < 1e-12


@pytest.mark.parametrize("subcycle", [0, 1])
def test_mass_not_conserved_without_correction(subcycle):
    o = amr_dambreak(subcycle=subcycle, refluxing=0)
    s0 = o.sums()
    o.advance(10)
    assert abs(o.sums()[0] - s0[0]) / s0[0] > 1e-9


@pytest.mark.parametrize("subcycle", [0, 1])
def test_momentum_conserved_periodic_amr(subcycle):
    o = Oracle(OracleParams(conn=fco.CONN_PERIODIC, m=8, min_level=2, max_level=4, subcycle=subcycle,
                            tag_threshold=0.01))
    o.init_refine(fco.INIT_HUMPS, humps_params(n_humps=6, seed=3, width=(0.05, 0.1)))
    q = o.fields()
    q[:, 1] = 0.1 * q[:, 0]          # uniform drift so that momentum is not ~0
    q[:, 2] = -0.05 * q[:, 0]
    o.set_fields(q)
    s0 = o.sums()
    o.advance(12)
    s1 = o.sums()
    np.testing.assert_allclose(s1, s0, rtol=1e-13)


def test_translation_at_courant_one_bitwise():
    m, lev = 8, 2
    o = Oracle(OracleParams(conn=fco.CONN_PERIODIC, equation=fco.EQ_ADV, m=m, min_level=lev,
                            max_level=lev, adv_u=1.0, adv_v=0.0, refluxing=0))
    rng = np.random.default_rng(5)
    n = 4 * m
    G0 = 1.0 + rng.random((n, n))            # values in [1, 2)
    tr, lv, xs, ys = o.leaves()
    q = np.zeros((o.n, 1, m, m))
    for k in range(o.n):
        q[k, 0] = G0[ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m]
    o.set_fields(q)
    dx = 1.0 / n
    steps = 11
    o.advance(steps, dx)
    q2 = o.fields()
    G1 = np.zeros_like(G0)
    for k in range(o.n):
        G1[ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m] = q2[k, 0]
    assert np.array_equal(G1, np.roll(G0, steps, axis=1))


def reflect_pad(Q, m):
    """Pad a (3, n, n) shallow-water array with 2 reflecting ghost layers
    (x walls then y walls), normal momentum negated."""
    F, n, _ = Q.shape
    P = np.zeros((F, n + 4, n + 4))
    P[:, 2:-2, 2:-2] = Q
    for k in range(2):
        P[:, 2:-2, 1 - k] = P[:, 2:-2, 2 + k]
        P[:, 2:-2, n + 2 + k] = P[:, 2:-2, n + 1 - k]
    P[1, 2:-2, :2] *= -1
    P[1, 2:-2, -2:] *= -1
    for k in range(2):
        P[:, 1 - k, :] = P[:, 2 + k, :]
        P[:, n + 2 + k, :] = P[:, n + 1 - k, :]
    P[2, :2, :] *= -1
    P[2, -2:, :] *= -1
    return P


def test_uniform_forest_equals_single_patch_bitwise():
    m, lev = 8, 2
    o = Oracle(OracleParams(m=m, min_level=lev, max_level=lev))
    o.init_fields(fco.INIT_DAMBREAK, dambreak_params())
    tr, lv, xs, ys = o.leaves()
    n = 4 * m
    q = o.fields()
    Q = np.zeros((3, n, n))
    for k in range(o.n):
        Q[:, ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m] = q[k]
    dx = 1.0 / n
    for step in range(5):
        dt = 0.3 * dx
        o.advance(1, dt)
        Q, _ = fco.patch_step(fco.EQ_SWE, reflect_pad(Q, n), dx, dx, dt)
    q2 = o.fields()
    for k in range(o.n):
        assert np.array_equal(q2[k], Q[:, ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m])


def assemble(o, lev_out):
    """Piecewise-constant sample of the forest's fields on the level-lev_out grid."""
    tr, lv, xs, ys = o.leaves()
    m = o.m
    n = (1 << lev_out) * m
    G = np.zeros((o.F, n, n))
    q = o.fields()
    for k in range(o.n):
        r = 1 << (lev_out - lv[k])
        blk = np.repeat(np.repeat(q[k], r, axis=1), r, axis=2)
        G[:, ys[k] * m * r:(ys[k] + 1) * m * r, xs[k] * m * r:(xs[k] + 1) * m * r] = blk
    return G


@pytest.mark.parametrize("subcycle", [0, 1])
def test_dambreak_d4_symmetry(subcycle):
    o = amr_dambreak(subcycle=subcycle)
    for _ in range(3):
        o.advance(4)
        o.regrid(o.tag())
    G = assemble(o, 4)
    h = G[0]
    for other in (h.T, h[::-1, :], h[:, ::-1], h[::-1, ::-1].T):
        np.testing.assert_allclose(h, other, rtol=0, atol=1e-13)
    np.testing.assert_allclose(G[1], G[2].T, rtol=0, atol=1e-13)


def test_ghost_fill_linear_and_constant_exact():
    o = Oracle(OracleParams(equation=fco.EQ_ADV, m=8, min_level=2, max_level=4))
    # refine a balanced patch in the middle, levels 2..4
    flags = np.zeros(o.n, np.int8)
    tr, lv, xs, ys = o.leaves()
    flags[(xs == 1) & (ys == 1)] = 1
    o.adapt_topology(flags)
    tr, lv, xs, ys = o.leaves()
    flags = np.zeros(o.n, np.int8)
    flags[(lv == 3) & (xs == 3) & (ys == 3)] = 1
    o.adapt_topology(flags)
    assert o.is_balanced()
    tr, lv, xs, ys = o.leaves()
    assert set(lv.tolist()) == {2, 3, 4}
    m = o.m
    a, b, c = 0.7, 0.3, -0.2
    q = np.zeros((o.n, 1, m, m))
    for k in range(o.n):
        dx = 1.0 / ((1 << lv[k]) * m)
        x = (xs[k] * m + np.arange(m) + 0.5) * dx
        y = (ys[k] * m + np.arange(m) + 0.5) * dx
        q[k, 0] = a + b * x[None, :] + c * y[:, None]
    o.set_fields(q)
    pad = o.fill_ghosts()
    checked = 0
    for k in range(o.n):
        dx = 1.0 / ((1 << lv[k]) * m)
        ii = np.arange(-2, m + 2)
        x = (xs[k] * m + ii + 0.5) * dx
        y = (ys[k] * m + ii + 0.5) * dx
        exact = a + b * x[None, :] + c * y[:, None]
        inside = (x[None, :] > 0.15) & (x[None, :] < 0.85) & (y[:, None] > 0.15) & (y[:, None] < 0.85)
        np.testing.assert_allclose(pad[k, 0][inside], exact[inside], rtol=0, atol=1e-14)
        checked += inside.sum()
    assert checked > 1000
    # constant field: bit-exact everywhere including walls
    q[:] = 0.8125
    o.set_fields(q)
    assert np.all(o.fill_ghosts() == 0.8125)


def test_regrid_conserves_and_refine_coarsen_roundtrip():
    o = amr_dambreak()
    o.advance(3)
    s0 = o.sums()
    o.regrid(random_forest_flags(o.n, 11))
    s1 = o.sums()
    assert abs(s1[0] - s0[0]) / s0[0] < 1e-14
    # refine everything at level 2 then coarsen those families back
    o2 = Oracle(OracleParams(m=8, min_level=2, max_level=3))
    o2.init_fields(fco.INIT_HUMPS, humps_params(n_humps=5, seed=2, width=(0.1, 0.2)))
    q0 = o2.fields()
    o2.regrid(np.ones(o2.n, np.int8))
    assert o2.n == 64
    o2.regrid(-np.ones(o2.n, np.int8))
    assert o2.n == 16
    np.testing.assert_allclose(o2.fields(), q0, rtol=0, atol=4e-16)


def numpy_flags(o, thr, crit):
    """criterion from the oracle's padded arrays, evaluated in numpy"""
    pad = o.fill_ghosts()
    m = o.m
    tr, lv, xs, ys = o.leaves()
    out = np.zeros(o.n, np.int8)
    for k in range(o.n):
        A = pad[k, 0]
        if crit == fco.TAG_GRAD:
            gx = (A[2:-2, 3:-1] - A[2:-2, 1:-3]) * 0.5
            gy = (A[3:-1, 2:-2] - A[1:-3, 2:-2]) * 0.5
            v = np.sqrt(gx * gx + gy * gy).max()
        else:
            I = A[2:-2, 2:-2]
            v = I.max() - I.min()
        out[k] = 1 if v > thr else 0
    q = o.fields()
    h = m // 2
    for k in range(o.n - 3):
        if lv[k] <= o.params.min_level or xs[k] % 2 or ys[k] % 2:
            continue
        fam = all(lv[k + c] == lv[k] and xs[k + c] == xs[k] + (c & 1) and ys[k + c] == ys[k] + (c >> 1)
                  for c in range(4))
        if not fam:
            continue
        par = np.zeros((m, m))
        for c in range(4):
            ch = q[k + c, 0]
            avg = 0.25 * ((ch[0::2, 0::2] + ch[0::2, 1::2]) + (ch[1::2, 0::2] + ch[1::2, 1::2]))
            par[(c >> 1) * h:(c >> 1) * h + h, (c & 1) * h:(c & 1) * h + h] = avg
        if crit == fco.TAG_GRAD:
            gx = (par[1:-1, 2:] - par[1:-1, :-2]) * 0.5
            gy = (par[2:, 1:-1] - par[:-2, 1:-1]) * 0.5
            v = np.sqrt(gx * gx + gy * gy).max()
        else:
            v = par.max() - par.min()
        if not v > thr:
            for c in range(4):
                if out[k + c] == 0:
                    out[k + c] = -1
    return out


@pytest.mark.parametrize("crit", [fco.TAG_GRAD, fco.TAG_MAXMIN])
def test_tag_matches_numpy(crit):
    o = Oracle(OracleParams(m=8, min_level=2, max_level=5, tag_crit=crit, tag_threshold=0.05))
    o.init_refine(fco.INIT_DAMBREAK, dambreak_params())
    o.advance(6)
    f = o.tag()
    assert np.array_equal(f, numpy_flags(o, 0.05, crit))
    assert (f == 1).any() and (f == -1).any()


def test_subcycle_equals_global_on_single_level():
    outs = []
    for sc in (0, 1):
        o = Oracle(OracleParams(m=8, min_level=3, max_level=3, subcycle=sc))
        o.init_fields(fco.INIT_DAMBREAK, dambreak_params())
        o.advance(7)
        outs.append(o.fields())
    assert np.array_equal(outs[0], outs[1])


def test_subcycle_takes_fewer_cell_updates():
    counts = []
    for sc in (0, 1):
        o = amr_dambreak(subcycle=sc)
        o.advance(4)
        counts.append((o.cell_updates, o.time))
    # sub-cycling: coarse levels take larger steps, so more simulated time per update
    assert counts[1][1] / counts[1][0] > counts[0][1] / counts[0][0]


def test_smooth_advection_second_order():
    errs = []
    for lev in (2, 3, 4):
        m = 8
        o = Oracle(OracleParams(conn=fco.CONN_PERIODIC, equation=fco.EQ_ADV, m=m, min_level=lev,
                                max_level=lev, adv_u=1.0, adv_v=0.5, refluxing=0))
        o.init_fields(fco.INIT_ADV_SINE, [1.0, 0.5, 1.0, 1.0])
        n = (1 << lev) * m
        dx = 1.0 / n
        T = 0.5
        steps = int(np.ceil(T / (0.5 * dx)))
        o.advance(steps, T / steps)
        tr, lv, xs, ys = o.leaves()
        q = o.fields()
        err = 0.0
        for k in range(o.n):
            x = (xs[k] * m + np.arange(m) + 0.5) * dx
            y = (ys[k] * m + np.arange(m) + 0.5) * dx
            ex = 1.0 + 0.5 * np.sin(2 * np.pi * ((x[None, :] - T) + (y[:, None] - 0.5 * T)))
            err += np.abs(q[k, 0] - ex).sum() * dx * dx
        errs.append(err)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 1.6, rates


def test_cfl_driven_dt():
    o = amr_dambreak()
    o.advance(1)
    for _ in range(5):
        dt_pred = o.next_dt
        t0 = o.time
        o.advance(1)
        # the predicted step is taken unless its Courant number exceeds 1, in
        # which case it is retaken with a smaller step
        assert o.time - t0 <= dt_pred * (1 + 1e-12)
        assert 0.5 < o.last_courant <= 1.0
