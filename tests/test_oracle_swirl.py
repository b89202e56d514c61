"""Oracle pins of the swirl velocity field (the paper's Example 1 flow is
prescribed but not given; reading: stream function
psi = sin^2(pi x) sin^2(pi y) / pi, u = dpsi/dy, v = -dpsi/dx, each edge's
normal velocity a stream-function difference over its length).

  * a smooth profile advected for t = 1/4 converges at second order to the
    exact solution traced back along the characteristics of the continuous
    field (scipy's adaptive integrator at 1e-10);
  * a constant state stays constant bit for bit (the discrete field is
    divergence-free cell by cell) through sub-cycled AMR steps;
  * the walls carry no flux, so mass is conserved to roundoff through steps
    and regrids of the paper's Example 1 data (0 on the left half, 1 on the
    right half) with max-min tagging.
"""
import numpy as np
import pytest

from oracle import fco
from oracle.fco import Oracle, OracleParams


def _swirl(**kw):
    base = dict(equation=fco.EQ_ADV, m=8, adv_u=1.0, velocity=fco.VEL_SWIRL, tag_crit=fco.TAG_MAXMIN,
                tag_threshold=0.05)
    base.update(kw)
    return Oracle(OracleParams(**base))


def test_swirl_converges_to_characteristics_solution():
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp

    def vel(t, z):
        n = z.size // 2
        x, y = z[:n], z[n:]
        return np.concatenate([np.sin(np.pi * x) ** 2 * np.sin(2 * np.pi * y),
                               -np.sin(2 * np.pi * x) * np.sin(np.pi * y) ** 2])
    T, errs = 0.25, []
    for lev in (2, 3, 4):
        m = 8
        o = _swirl(min_level=lev, max_level=lev, refluxing=0)
        o.init_fields(fco.INIT_ADV_SINE, [1.0, 0.5, 1.0, 1.0])
        n = (1 << lev) * m
        dx = 1.0 / n
        steps = int(np.ceil(T / (0.5 * dx)))
        o.advance(steps, T / steps)
        _, _, xs, ys = o.leaves()
        q = o.fields()
        H = np.zeros((n, n))
        for k in range(o.n):
            H[ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m] = q[k, 0]
        xc = (np.arange(n) + 0.5) * dx
        X, Y = np.meshgrid(xc, xc)
        sol = solve_ivp(vel, (T, 0.0), np.concatenate([X.ravel(), Y.ravel()]), rtol=1e-10, atol=1e-12)
        x0, y0 = sol.y[:n * n, -1], sol.y[n * n:, -1]
        ex = (1.0 + 0.5 * np.sin(2 * np.pi * (x0 + y0))).reshape(n, n)
        errs.append(np.abs(H - ex).sum() * dx * dx)
    errs = np.array(errs)
    assert np.log2(errs[:-1] / errs[1:]).min() > 1.8, errs


@pytest.mark.parametrize("subcycle", [0, 1])
def test_swirl_freestream_and_mass(subcycle):
    o = _swirl(min_level=2, max_level=4, subcycle=subcycle)
    o.init_refine(fco.INIT_ADV_BOX, [0.5, 1.0, 0.0, 1.0, 1.0, 0.0])
    q = o.fields()
    const = np.full_like(q, 0.7)
    o.set_fields(const)
    o.advance(4)
    assert np.array_equal(o.fields(), const)
    o.set_fields(q)
    s0 = o.sums()
    for _ in range(4):
        o.advance(3)
        o.regrid(o.tag())
    _, lv, _, _ = o.leaves()
    assert lv.max() > lv.min()          # the distorted interface is refined
    assert abs(o.sums()[0] - s0[0]) <= 1e-13 * s0[0]


def test_swirl_needs_advection():
    with pytest.raises(RuntimeError):
        Oracle(OracleParams(equation=fco.EQ_SWE, velocity=fco.VEL_SWIRL))
