"""Oracle pins of the entropy fix and of the T2 transverse variant.

Harten-Hyman entropy fix (LeVeque, Finite Volume Methods, Sec. 15.3.5):
  * a stationary expansion shock (an entropy-violating jump on the 1-shock
    Hugoniot locus with speed 0) is an exact steady state of the Roe scheme
    without the fix, bit for bit, and never approaches the true solution;
    with the fix it opens into the transonic rarefaction of the exact
    Riemann solution at first order;
  * the fixed fluctuations still add up to the flux jump, and edges without
    a transonic wave keep their fluctuations bit for bit (so subsonic runs
    are unchanged).
T2 (the limited second-order corrections split transversely with the
fluctuations, LeVeque 1997):
  * on smooth diagonal advection it keeps second-order convergence with a
    much smaller error than T1 (a sign error in the split doubles T1's);
  * a planar problem still reproduces the 1D scheme bit for bit, a lake at
    rest stays at rest bit for bit, mass is conserved with the coarse-fine
    correction, and the radial dam break keeps its D4 symmetry.
"""
import numpy as np
import pytest

from fc_inputs import dambreak_params
from oracle import fco
from oracle.fco import Oracle, OracleParams

G = 1.0
# stationary 1-shock on the Hugoniot locus of (h, u) = (1, 0.5): equal mass
# flux h u and momentum flux h u^2 + h^2/2, with u - c < 0 on the left and
# u - c > 0 on the right (characteristics leave the jump: entropy-violating)
HL, UL = 1.0, 0.5
HR = (np.sqrt(3.0) - 1.0) / 2.0
UR = HL * UL / HR


def test_stationary_expansion_shock_data():
    assert HL * UL == pytest.approx(HR * UR, rel=1e-15)
    assert HL * UL ** 2 + 0.5 * G * HL ** 2 == pytest.approx(HR * UR ** 2 + 0.5 * G * HR ** 2, rel=1e-14)
    assert UL - np.sqrt(G * HL) < 0.0 < UR - np.sqrt(G * HR)


def _riemann_1d(n, efix, T=0.2):
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx - 0.5
    h = np.where(x < 0, HL, HR)
    hu = np.where(x < 0, HL * UL, HR * UR)
    dt = 0.4 * dx / 2.0
    steps = int(round(T / dt))
    h1, _ = fco.swe1d(h, hu, dx, T / steps, steps, G, efix=efix)
    he, _ = fco.swe_exact(HL, UL, HR, UR, x / T, G)
    return h, h1, np.abs(h1 - he).sum() * dx


def test_expansion_shock_steady_without_fix_opens_with_it():
    errs = {0: [], 1: []}
    for n in (100, 200, 400, 800):
        for efix in (0, 1):
            h0, h1, err = _riemann_1d(n, efix)
            errs[efix].append(err)
            if efix == 0:
                assert np.array_equal(h1, h0)          # the jump never moves
    e0, e1 = np.array(errs[0]), np.array(errs[1])
    assert np.all(np.abs(e0 / e0[0] - 1.0) < 1e-3)      # no convergence without the fix
    rates = np.log2(e1[:-1] / e1[1:])
    assert rates.min() > 0.9, rates                     # first order with it
    assert e1[-1] < 0.01 * e0[-1]


def test_fixed_fluctuations_add_to_flux_jump_and_leave_subsonic_edges_alone():
    def flux(q):
        h, hu = q[0], q[1]
        return np.array([hu, hu * hu / h + 0.5 * G * h * h, hu * q[2] / h])
    pairs = [([HL, HL * UL, 0.0], [HR, HR * UR, 0.0]),        # transonic 1-wave
             ([1.0, 0.0, 0.2], [0.05, 0.0, 0.0]),             # strong dam break edge
             ([0.05, 0.0, 0.0], [1.0, 0.0, 0.1])]             # its mirror: transonic 3-wave
    for qL, qR in pairs:
        am, ap = fco.roe_x_efix(qL, qR, G)
        np.testing.assert_allclose(am + ap, flux(np.array(qR)) - flux(np.array(qL)), rtol=1e-13, atol=1e-15)
    # subsonic jump: exactly the unfixed fluctuations
    qL, qR = [2.0, 0.1, 0.3], [1.0, -0.2, 0.1]
    _, _, am0, ap0 = fco.roe_x(qL, qR, G)
    am1, ap1 = fco.roe_x_efix(qL, qR, G)
    assert np.array_equal(am0, am1) and np.array_equal(ap0, ap1)


def _amr_dambreak(**kw):
    o = Oracle(OracleParams(m=8, min_level=2, max_level=4, **kw))
    o.init_refine(fco.INIT_DAMBREAK, dambreak_params())
    return o


@pytest.mark.parametrize("subcycle", [0, 1])
def test_entropy_fix_leaves_a_subsonic_run_unchanged(subcycle):
    a = _amr_dambreak(subcycle=subcycle)
    b = _amr_dambreak(subcycle=subcycle, entropy_fix=1)
    for _ in range(2):
        a.advance(3)
        b.advance(3)
        f = a.tag()
        a.regrid(f)
        b.regrid(f)
    assert np.array_equal(a.fields(), b.fields())


def _diag_advection_error(lev, transverse):
    m = 8
    o = Oracle(OracleParams(conn=fco.CONN_PERIODIC, equation=fco.EQ_ADV, m=m, min_level=lev, max_level=lev,
                            adv_u=1.0, adv_v=1.0, refluxing=0, transverse=transverse))
    o.init_fields(fco.INIT_ADV_SINE, [1.0, 0.5, 1.0, 1.0])
    n = (1 << lev) * m
    dx = 1.0 / n
    T = 0.5
    steps = int(np.ceil(T / (0.6 * dx)))
    o.advance(steps, T / steps)
    _, _, xs, ys = o.leaves()
    q = o.fields()
    err = 0.0
    for k in range(o.n):
        x = (xs[k] * m + np.arange(m) + 0.5) * dx
        y = (ys[k] * m + np.arange(m) + 0.5) * dx
        ex = 1.0 + 0.5 * np.sin(2 * np.pi * ((x[None, :] - T) + (y[:, None] - T)))
        err += np.abs(q[k, 0] - ex).sum() * dx * dx
    return err


def test_t2_second_order_with_smaller_error_on_diagonal_advection():
    e1 = np.array([_diag_advection_error(lev, 1) for lev in (2, 3, 4)])
    e2 = np.array([_diag_advection_error(lev, 2) for lev in (2, 3, 4)])
    assert np.log2(e2[:-1] / e2[1:]).min() > 1.9
    assert np.all(e2 < 0.3 * e1), (e1, e2)


@pytest.mark.parametrize("efix", [0, 1])
def test_t2_planar_equals_1d_bitwise(efix):
    m, lev = 8, 3
    o = Oracle(OracleParams(m=m, min_level=lev, max_level=lev, refluxing=0, transverse=2, entropy_fix=efix))
    _, _, xs, _ = o.leaves()
    n = 8 * m
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    if efix:      # the stationary expansion shock at x = 1/2
        h1 = np.where(xc < 0.5, HL, HR)
        hu1 = np.where(xc < 0.5, HL * UL, HR * UR)
    else:
        h1 = np.where(xc < 0.5, 2.0, 1.0)
        hu1 = np.zeros(n)
    q = np.zeros((o.n, 3, m, m))
    for k in range(o.n):
        q[k, 0] = h1[xs[k] * m:(xs[k] + 1) * m][None, :]
        q[k, 1] = hu1[xs[k] * m:(xs[k] + 1) * m][None, :]
    o.set_fields(q)
    dt = 0.2 * dx
    steps = 5
    o.advance(steps, dt)
    q2 = o.fields()
    hh, hu = fco.swe1d(h1, hu1, dx, dt, steps, G, efix=efix)
    # compare away from the ends (reflecting walls in 2D, transmissive ends in
    # 1D): 5 steps reach at most 10 cells in from them
    H = np.zeros((3, n, n))
    _, _, xs, ys = o.leaves()
    for k in range(o.n):
        H[:, ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m] = q2[k]
    mid = slice(12, n - 12)
    assert np.array_equal(H[0][:, mid], np.broadcast_to(hh[mid], (n, n - 24)))
    assert np.array_equal(H[1][:, mid], np.broadcast_to(hu[mid], (n, n - 24)))
    assert np.all(H[2] == 0.0)


@pytest.mark.parametrize("subcycle", [0, 1])
def test_t2_lake_at_rest_and_mass(subcycle):
    o = _amr_dambreak(subcycle=subcycle, transverse=2, entropy_fix=1)
    q = o.fields()
    lake = np.zeros_like(q)
    lake[:, 0] = 1.5
    o.set_fields(lake)
    o.advance(4)
    assert np.array_equal(o.fields(), lake)
    o.set_fields(q)
    s0 = o.sums()
    for _ in range(3):
        o.advance(3)
        o.regrid(o.tag())
    s1 = o.sums()
    assert abs(s1[0] - s0[0]) <= 1e-13 * abs(s0[0])


def test_t2_dambreak_d4_symmetry():
    o = _amr_dambreak(subcycle=1, transverse=2)
    for _ in range(2):
        o.advance(4)
        o.regrid(o.tag())
    _, lv, xs, ys = o.leaves()
    q = o.fields()
    m, L = 8, 4
    N = (1 << L) * m
    H = np.zeros((N, N))
    for k in range(o.n):
        r = 1 << (L - lv[k])
        blk = np.repeat(np.repeat(q[k, 0], r, axis=0), r, axis=1)
        H[ys[k] * m * r:(ys[k] + 1) * m * r, xs[k] * m * r:(xs[k] + 1) * m * r] = blk
    for other in (H.T, H[::-1, :], H[:, ::-1]):
        np.testing.assert_allclose(H, other, rtol=0, atol=1e-13)


def test_t2_not_on_the_sphere():
    with pytest.raises(RuntimeError):
        Oracle(OracleParams(conn=fco.CONN_SPHERE, equation=fco.EQ_ADV, m=8, min_level=1, max_level=1,
                            transverse=2))
