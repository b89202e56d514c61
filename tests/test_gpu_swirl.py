"""GPU parity of advection in the swirl field on the square (the paper's
Example 1 setting: 0 on the left half, 1 on the right half, max-min
tagging): FP64 within 1e-12 relative L1 of the oracle through sub-cycled and
global-dt AMR steps and regrids, FP32 within 2e-5."""
import numpy as np
import pytest

from gpu_helpers import FP32_TOL, FP64_TOL, assert_same_forest, fcmod, rel_l1
from oracle import fco

pytestmark = pytest.mark.gpu

BOX = [0.5, 1.0, 0.0, 1.0, 1.0, 0.0]


def _pair(fc, **kw):
    base = dict(equation=1, m=8, min_level=2, max_level=4, adv_u=1.0, velocity=1, tag_crit=1, tag_threshold=0.05)
    base.update(kw)
    prec = base.pop("precision", 0)
    ctx = fc.Context(device=0, precision=prec, **base)
    ora = fco.Oracle(fco.OracleParams(**base))
    return ctx, ora


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("m", [8, 16])
def test_swirl_amr_fp64(subcycle, m):
    fc = fcmod()
    ctx, ora = _pair(fc, m=m, subcycle=subcycle)
    ctx.init_refine(fc.FC_INIT_ADV_BOX, BOX)
    ora.init_refine(fco.INIT_ADV_BOX, BOX)
    for _ in range(3):
        tg, _ = ctx.advance(4)
        to, _ = ora.advance(4)
        assert abs(tg - to) <= 1e-12 * to
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert rr[0] < FP64_TOL, rr
        fg, fo = ctx.tag(), ora.tag()
        assert np.array_equal(fg, fo)
        ctx.regrid(fo)
        ora.regrid(fo)
        assert_same_forest(ctx, ora)
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12)


def test_swirl_fp32_and_launch_shapes():
    fc = fcmod()
    ctx, ora = _pair(fc, precision=1, subcycle=1)
    ora.init_refine(fco.INIT_ADV_BOX, BOX)
    tr, lv, x, y = ora.leaves()
    ctx.forest_set_leaves(tr, lv, x, y)
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    dt = 0.5 * ora.next_dt
    ctx.advance(12, dt)
    ora.advance(12, dt)
    assert rel_l1(ctx.read_fields(), ora.fields())[0] < FP32_TOL
    v, ms = ctx.autotune()
    assert v in (0, 1) and np.all(ms[2:] == -1.0)
    with pytest.raises(fc.FCError):
        ctx.set_variant(2)
    with pytest.raises(fc.FCError):
        fc.Context(device=0, equation=0, velocity=1)
