"""GPU parity of the optional parts of the method: the Harten-Hyman entropy
fix (transonic rarefactions in the shallow-water fluctuations) and the T2
transverse variant (limited corrections split transversely with the
fluctuations).  FP64 kernels within 1e-12 relative L1 of the FP64 oracle,
FP32 within 2e-5, in the one-CTA-per-patch launch shapes that carry them."""
import numpy as np
import pytest

from fc_inputs import dambreak_params, humps_params
from gpu_helpers import FP32_TOL, FP64_TOL, assert_same_forest, fcmod, rel_l1
from oracle import fco

pytestmark = pytest.mark.gpu

# stationary entropy-violating expansion shock (an exact steady state of the
# Roe scheme without the fix)
HL, UL = 1.0, 0.5
HR = (np.sqrt(3.0) - 1.0) / 2.0
UR = HL * UL / HR


def _planar_shock(ora, m, axis):
    _, _, xs, ys = ora.leaves()
    q = np.zeros((ora.n, 3, m, m))
    n = int(round(np.sqrt(ora.n))) * m
    c = (np.arange(n) + 0.5) / n
    h = np.where(c < 0.5, HL, HR)
    hu = np.where(c < 0.5, HL * UL, HR * UR)
    for k in range(ora.n):
        if axis == 0:
            sl = slice(xs[k] * m, (xs[k] + 1) * m)
            q[k, 0] = h[sl][None, :]
            q[k, 1] = hu[sl][None, :]
        else:
            sl = slice(ys[k] * m, (ys[k] + 1) * m)
            q[k, 0] = h[sl][:, None]
            q[k, 2] = hu[sl][:, None]
    return q


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("transverse", [1, 2])
@pytest.mark.parametrize("efix", [0, 1])
def test_expansion_shock_fp64(axis, transverse, efix):
    """periodic square: the expansion shock at the middle and, across the
    periodic boundary, the reverse jump (an admissible stationary shock)"""
    fc = fcmod()
    m = 16
    kw = dict(conn=1, m=m, min_level=2, max_level=2, refluxing=0, transverse=transverse, entropy_fix=efix)
    ctx = fc.Context(device=0, **kw)
    ora = fco.Oracle(fco.OracleParams(**kw))
    q = _planar_shock(ora, m, axis)
    ora.set_fields(q)
    ctx.write_fields(q)
    dt = 0.1 / (4 * m)
    ctx.advance(8, dt)
    ora.advance(8, dt)
    qg, qo = ctx.read_fields(), ora.fields()
    assert rel_l1(qg, qo)[0] < FP64_TOL
    assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()
    moved = np.abs(qo - q).max()
    if efix:
        assert moved > 1e-3            # the fix opens the jump
    else:
        assert moved < 1e-12           # steady without it


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("transverse,efix", [(2, 0), (1, 1), (2, 1)])
def test_strong_dambreak_amr_fp64(subcycle, transverse, efix):
    """radial dam break with depth ratio 10 (transonic rarefaction) on levels
    2-4 through steps and regrids"""
    fc = fcmod()
    kw = dict(m=8, min_level=2, max_level=4, subcycle=subcycle, transverse=transverse, entropy_fix=efix)
    ctx = fc.Context(device=0, **kw)
    ora = fco.Oracle(fco.OracleParams(**kw))
    p = [0.5, 0.5, 0.04, 10.0, 1.0]
    ctx.init_refine(fc.FC_INIT_DAMBREAK, p)
    ora.init_refine(fco.INIT_DAMBREAK, p)
    assert_same_forest(ctx, ora)
    for _ in range(2):
        tg, _ = ctx.advance(3)
        to, _ = ora.advance(3)
        assert abs(tg - to) <= 1e-12 * to
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert np.all(rr < FP64_TOL), rr
        f = ora.tag()
        ctx.regrid(f)
        ora.regrid(f)
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12, atol=1e-12)


def test_t2_periodic_humps_and_advection_fp64():
    fc = fcmod()
    kw = dict(conn=1, m=16, min_level=2, max_level=3, subcycle=1, transverse=2)
    ctx = fc.Context(device=0, **kw)
    ora = fco.Oracle(fco.OracleParams(**kw))
    p = humps_params(12, 4)
    ctx.init_refine(fc.FC_INIT_HUMPS, p)
    ora.init_refine(fco.INIT_HUMPS, p)
    ctx.advance(5)
    ora.advance(5)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP64_TOL), rr
    kw = dict(conn=1, equation=1, m=8, min_level=3, max_level=3, adv_u=1.0, adv_v=1.0, refluxing=0, transverse=2)
    ctx = fc.Context(device=0, **kw)
    ora = fco.Oracle(fco.OracleParams(**kw))
    ctx.set_initial(fc.FC_INIT_ADV_SINE, [1.0, 0.5, 1.0, 1.0])
    ora.init_fields(fco.INIT_ADV_SINE, [1.0, 0.5, 1.0, 1.0])
    dt = 0.6 / 64
    ctx.advance(20, dt)
    ora.advance(20, dt)
    assert rel_l1(ctx.read_fields(), ora.fields())[0] < FP64_TOL


def test_t2_efix_fp32():
    fc = fcmod()
    kw = dict(m=16, min_level=2, max_level=4, subcycle=1, transverse=2, entropy_fix=1)
    ctx = fc.Context(device=0, precision=fc.FC_FP32, **kw)
    ora = fco.Oracle(fco.OracleParams(**kw))
    ora.init_refine(fco.INIT_DAMBREAK, [0.5, 0.5, 0.04, 10.0, 1.0])
    tr, lv, x, y = ora.leaves()
    ctx.forest_set_leaves(tr, lv, x, y)
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    dt = 0.25 * ora.next_dt
    ctx.advance(12, dt)
    ora.advance(12, dt)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP32_TOL), rr


def test_launch_shapes_with_t2_or_efix():
    fc = fcmod()
    for kw in (dict(transverse=2), dict(entropy_fix=1)):
        ctx = fc.Context(m=8, min_level=2, max_level=3, subcycle=1, device=0, **kw)
        ctx.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
        v, ms = ctx.autotune()
        assert v in (0, 1) and np.all(ms[2:] == -1.0)
        for bad in (2, 4, 5):
            with pytest.raises(fc.FCError):
                ctx.set_variant(bad)
        ctx.set_variant(1)
        ctx.advance(2)
    with pytest.raises(fc.FCError):
        fc.Context(conn=fc.FC_CONN_SPHERE, equation=fc.FC_EQ_ADV, m=8, min_level=1, max_level=1, device=0,
                   transverse=2)
    with pytest.raises(fc.FCError):
        fc.Context(m=8, min_level=1, max_level=1, device=0, transverse=3)
