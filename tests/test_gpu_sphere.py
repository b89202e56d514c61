"""Cubed sphere on the GPU vs the oracle (Fig. 1 right, Sec. 4 transformations
across trees, Sec. 5 Eq. (1) in capacity form with solid-body rotation):
forest tables including orientation codes bit-exact, FP64 fields within 1e-12
relative L1, FP32 within 2e-5, mass conserved, regrid transfers matching."""
import math

import numpy as np
import pytest

from fc_inputs import random_forest_flags
from gpu_helpers import FP32_TOL, FP64_TOL, assert_same_forest, fcmod, make_pair, rel_l1
from oracle import fco

pytestmark = pytest.mark.gpu

OMEGA, TILT = 2 * math.pi, math.pi / 4
HILL = [0.3, 0.2, 0.35]


def _pair(fc, **kw):
    args = dict(conn=fc.FC_CONN_SPHERE, equation=fc.FC_EQ_ADV, omega=OMEGA, omega_axis_tilt=TILT,
                tag_threshold=0.02)
    args.update(kw)
    return make_pair(fc, **args)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_sphere_forest_uniform_bitexact(level):
    fc = fcmod()
    ctx, ora = _pair(fc, min_level=level, max_level=level)
    ctx.forest_uniform(level)
    ora.uniform(level)
    assert_same_forest(ctx, ora)
    nb = ctx.forest_get_neighbors()
    if level > 0:
        assert np.any(nb[:, :, 3] != 0)      # cross-tree entries carry an orientation


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sphere_forest_adapted_bitexact(seed):
    fc = fcmod()
    ctx, ora = _pair(fc, min_level=1, max_level=4)
    ctx.forest_uniform(2)
    ora.uniform(2)
    for r in range(3):
        f = random_forest_flags(ora.n, seed * 10 + r)
        ctx.regrid(f)
        ora.regrid(f)
        assert_same_forest(ctx, ora)


def _run(ctx, ora, rounds, steps, regrid=True):
    for r in range(rounds):
        tg, _ = ctx.advance(steps)
        to, _ = ora.advance(steps)
        assert abs(tg - to) <= 1e-12 * to
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert rr[0] < FP64_TOL, (r, rr)
        if regrid:
            fg, fo = ctx.tag(), ora.tag()
            assert np.array_equal(fg, fo)
            ctx.regrid(fo)
            ora.regrid(fo)
            assert_same_forest(ctx, ora)
            rr = rel_l1(ctx.read_fields(), ora.fields())
            assert rr[0] < FP64_TOL, (r, "regrid", rr)


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("m,lmin,lmax", [(8, 1, 3), (16, 1, 2)])
def test_sphere_amr_fp64(subcycle, m, lmin, lmax):
    fc = fcmod()
    ctx, ora = _pair(fc, m=m, min_level=lmin, max_level=lmax, subcycle=subcycle)
    ctx.init_refine(fc.FC_INIT_HILL, HILL)
    ora.init_refine(fco.INIT_HILL, HILL)
    assert_same_forest(ctx, ora)
    assert len(set(ora.leaves()[1].tolist())) >= 2
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert rr[0] < 1e-14, rr
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-13)
    s0 = ctx.conservation_sums()
    _run(ctx, ora, 3, 3)
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12)
    assert abs(ctx.conservation_sums()[0] - s0[0]) <= 1e-13 * abs(s0[0])


def test_sphere_uniform_m32_fp64():
    fc = fcmod()
    ctx, ora = _pair(fc, m=32, min_level=1, max_level=1)
    ctx.set_initial(fc.FC_INIT_HILL, HILL)
    ora.uniform(1)
    ora.init_fields(fco.INIT_HILL, HILL)
    _run(ctx, ora, 2, 4, regrid=False)


@pytest.mark.parametrize("subcycle", [0, 1])
def test_sphere_amr_fp32(subcycle):
    fc = fcmod()
    ctx, ora = _pair(fc, m=16, min_level=1, max_level=3, subcycle=subcycle, precision=1)
    ora.init_refine(fco.INIT_HILL, HILL)
    tr, lv, x, y = ora.leaves()
    ctx.forest_set_leaves(tr, lv, x, y)
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    dt = 0.5 * ora.next_dt
    ctx.advance(12, dt)
    ora.advance(12, dt)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert rr[0] < FP32_TOL, rr
    s = ctx.conservation_sums()
    ctx.advance(12, dt)
    assert abs(ctx.conservation_sums()[0] - s[0]) <= 1e-5 * abs(s[0])


def test_sphere_random_regrid_conserves_fp64():
    fc = fcmod()
    ctx, ora = _pair(fc, min_level=1, max_level=3)
    ctx.forest_uniform(2)
    ora.uniform(2)
    ctx.set_initial(fc.FC_INIT_HILL, [1.0, -0.4, 0.5])
    ora.init_fields(fco.INIT_HILL, [1.0, -0.4, 0.5])
    s0 = ctx.conservation_sums()[0]
    for r in range(3):
        f = random_forest_flags(ora.n, 40 + r)
        ctx.regrid(f)
        ora.regrid(f)
        assert_same_forest(ctx, ora)
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert rr[0] < FP64_TOL, rr
        assert abs(ctx.conservation_sums()[0] - s0) <= 1e-13 * abs(s0)


def test_sphere_rejects_shallow_water():
    fc = fcmod()
    with pytest.raises(fc.FCError):
        fc.Context(conn=fc.FC_CONN_SPHERE, equation=fc.FC_EQ_SWE, device=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_sphere_freestream(precision):
    """a constant stays exactly constant without the coarse-fine correction
    and to roundoff with it (edge speeds of a coarse edge and of its two fine
    halves agree only to rounding)"""
    fc = fcmod()
    for reflux, tol in ((0, 0.0), (1, 1e-13 if precision == 0 else 1e-6)):
        ctx, ora = _pair(fc, min_level=1, max_level=3, subcycle=1, refluxing=reflux, precision=precision)
        ora.init_refine(fco.INIT_HILL, HILL)
        ctx.forest_set_leaves(*ora.leaves())
        dt = np.float64 if precision == 0 else np.float32
        ctx.write_fields(np.full((ctx.n, 1, 8, 8), 1.25, dt))
        ctx.advance(6)
        q = ctx.read_fields().astype(np.float64)
        assert np.max(np.abs(q - 1.25)) <= tol
