"""Pins of the oracle's edge solvers against mathematics that fixes them.

Each check is chosen so that a plausible slip in the oracle (dropped term,
wrong sign, swapped component) fails it:
  * Roe waves sum to the jump, and speed-weighted waves sum to the flux jump
    (the defining property of Roe's linearisation, cited in Sec. 3);
  * a jump obeying the Rankine-Hugoniot relations is a single wave moving at
    the shock speed; a pure shear jump is a single contact wave;
  * the transverse split sums to the Roe-averaged y-Jacobian applied to the
    fluctuation (matrix written out independently here);
  * the MC limiter matches its piecewise closed form;
  * the exact Riemann solver satisfies the jump relations and the Riemann
    invariant, and the 1D scheme converges to it;
  * a planar problem on the 2D grid reproduces the 1D scheme bit for bit.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import fco
from oracle.fco import Oracle, OracleParams

G = 1.0


def flux_x(q, g=G):
    h, hu, hv = q
    return np.array([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h])


def rand_states(rng, n):
    for _ in range(n):
        qL = np.array([0.5 + rng.random(), rng.normal() * 0.3, rng.normal() * 0.3])
        qR = np.array([0.5 + rng.random(), rng.normal() * 0.3, rng.normal() * 0.3])
        yield qL, qR


def test_roe_waves_sum_to_jump_and_flux_jump():
    rng = np.random.default_rng(0)
    for qL, qR in rand_states(rng, 200):
        W, s, am, ap = fco.roe_x(qL, qR, G)
        np.testing.assert_allclose(W.sum(axis=0), qR - qL, rtol=0, atol=1e-14)
        dF = flux_x(qR) - flux_x(qL)
        np.testing.assert_allclose((s[:, None] * W).sum(axis=0), dF, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(am + ap, dF, rtol=1e-13, atol=1e-13)
        # speeds are u_hat -/+ c_hat around u_hat
        assert s[0] < s[1] < s[2]


def test_roe_single_shock_and_shear():
    # right-going shock into still water hR=1 from hL=2: RH gives uL, speed
    hL, hR, uR = 2.0, 1.0, 0.0
    # mass and momentum RH: s (hL - hR) = hL uL - hR uR ; s(hL uL - hR uR) = (hL uL^2 + g hL^2/2) - (...)
    sp = np.sqrt(G * hL * (hL + hR) / (2 * hR))     # shock speed into still water
    uL = sp * (hL - hR) / hL
    qL = np.array([hL, hL * uL, 0.0])
    qR = np.array([hR, 0.0, 0.0])
    W, s, am, ap = fco.roe_x(qL, qR, G)
    nz = [p for p in range(3) if np.abs(W[p]).max() > 1e-12]
    assert nz == [2]
    assert s[2] == pytest.approx(sp, rel=1e-13)
    # pure shear: only the transverse momentum jumps
    qL = np.array([1.3, 0.2 * 1.3, 0.5])
    qR = np.array([1.3, 0.2 * 1.3, -0.1])
    W, s, am, ap = fco.roe_x(qL, qR, G)
    assert np.abs(W[0]).max() < 1e-15 and np.abs(W[2]).max() < 1e-15
    np.testing.assert_allclose(W[1], [0, 0, -0.6], atol=1e-15)
    assert s[1] == pytest.approx(0.2, rel=1e-15)


def test_transverse_split_is_roe_y_jacobian():
    rng = np.random.default_rng(1)
    for qL, qR in rand_states(rng, 100):
        d = rng.normal(size=3)
        bm, bp = fco.roe_transverse_x(qL, qR, d, G)
        sL, sR = np.sqrt(qL[0]), np.sqrt(qR[0])
        u = (sL * qL[1] / qL[0] + sR * qR[1] / qR[0]) / (sL + sR)
        v = (sL * qL[2] / qL[0] + sR * qR[2] / qR[0]) / (sL + sR)
        c2 = G * 0.5 * (qL[0] + qR[0])
        B = np.array([[0.0, 0.0, 1.0], [-u * v, v, u], [c2 - v * v, 0.0, 2 * v]])
        np.testing.assert_allclose(bm + bp, B @ d, rtol=1e-12, atol=1e-13)


def mc_closed(t):
    if t <= 0:
        return 0.0
    if t <= 1.0 / 3.0:
        return 2 * t
    if t <= 3.0:
        return 0.5 * (1 + t)
    return 2.0


@pytest.mark.parametrize("t", [-2.0, -0.1, 0.0, 0.1, 1.0 / 3.0, 0.5, 1.0, 2.0, 3.0, 7.5])
def test_mc_limiter_closed_form(t):
    assert fco.mc(t) == pytest.approx(mc_closed(t), rel=1e-15, abs=0)


def _exact_middle(hL, hR, g=G):
    """Middle depth of the still-water dam break from the closed-form relations."""
    f = lambda h: 2 * (np.sqrt(g * h) - np.sqrt(g * hL)) + (h - hR) * np.sqrt(g * (h + hR) / (2 * h * hR))
    return brentq(f, hR, hL, xtol=1e-15, rtol=1e-15)


def test_exact_solver_jump_relations_and_invariant():
    hL, hR = 2.0, 1.0
    hs = _exact_middle(hL, hR)
    xi = np.linspace(-2.0, 2.0, 4001)
    h, u = fco.swe_exact(hL, 0.0, hR, 0.0, xi, G)
    # middle state
    us = 2 * (np.sqrt(G * hL) - np.sqrt(G * hs))
    mid = (xi > us - 0.01) & (xi < us + 0.01)
    np.testing.assert_allclose(h[mid], hs, rtol=1e-12)
    np.testing.assert_allclose(u[mid], us, rtol=1e-12)
    # shock: mass and momentum Rankine-Hugoniot across the jump
    jump = np.nonzero(np.diff(h[xi > 0]) != 0)[0][-1]
    sh = xi[xi > 0][jump]
    s_mass = (hs * us) / (hs - hR)
    assert abs(sh - s_mass) < 2e-3
    mom_l = hs * us * us + 0.5 * G * hs * hs
    mom_r = 0.5 * G * hR * hR
    assert s_mass * (hs * us) == pytest.approx(mom_l - mom_r, rel=1e-10)
    # rarefaction: u + 2c constant through the fan
    fan = (xi > -np.sqrt(G * hL) + 0.05) & (xi < us - np.sqrt(G * hs) - 0.05)
    inv = u[fan] + 2 * np.sqrt(G * h[fan])
    np.testing.assert_allclose(inv, 2 * np.sqrt(G * hL), rtol=1e-12)


def test_1d_scheme_converges_to_exact():
    errs = []
    for n in (100, 200, 400, 800):
        dx = 1.0 / n
        x = (np.arange(n) + 0.5) * dx - 0.5
        h = np.where(x < 0, 2.0, 1.0)
        hu = np.zeros(n)
        T = 0.2
        dt = 0.4 * dx / np.sqrt(G * 2.0) * 1.0
        steps = int(round(T / dt))
        dt = T / steps
        h1, _ = fco.swe1d(h, hu, dx, dt, steps, G)
        he, _ = fco.swe_exact(2.0, 0.0, 1.0, 0.0, x / T, G)
        errs.append(np.abs(h1 - he).sum() * dx)
    errs = np.array(errs)
    assert np.all(np.diff(errs) < 0)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates.min() > 0.6, rates


def test_planar_2d_equals_1d_bitwise():
    m, lev = 8, 2
    o = Oracle(OracleParams(m=m, min_level=lev, max_level=lev, refluxing=0))
    tr, lv, xs, ys = o.leaves()
    n = 4 * m
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    h1 = np.where(xc < 0.5, 2.0, 1.0)
    q = np.zeros((o.n, 3, m, m))
    for k in range(o.n):
        q[k, 0] = h1[xs[k] * m:(xs[k] + 1) * m][None, :]
    o.set_fields(q)
    dt = 0.3 * dx
    steps = 6          # waves stay away from the walls
    o.advance(steps, dt)
    q2 = o.fields()
    hh, hu = fco.swe1d(h1, np.zeros(n), dx, dt, steps, G)
    for k in range(o.n):
        blk = q2[k, 0]
        ref = hh[xs[k] * m:(xs[k] + 1) * m]
        assert np.array_equal(blk, np.broadcast_to(ref, blk.shape))
        assert np.array_equal(q2[k, 1], np.broadcast_to(hu[xs[k] * m:(xs[k] + 1) * m], blk.shape))
        assert np.all(q2[k, 2] == 0.0)
