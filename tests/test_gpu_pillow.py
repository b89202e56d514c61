"""Two-tree sphere on the GPU vs the oracle (Sec. 5, Example 2: two quadtrees
on [-1,1]^2, one per hemisphere, solid-body rotation of a field that is 1 on
one half of the sphere and 0 on the other): forest tables including the
orientation codes bit-exact, FP64 fields within 1e-12 relative L1 through
steps, tags and regrids (both time-stepping modes), FP32 within 2e-5, every
singular tree corner coarse-fine, freestream and mass."""
import math

import numpy as np
import pytest

from fc_inputs import random_forest_flags
from gpu_helpers import FP32_TOL, FP64_TOL, assert_same_forest, fcmod, make_pair, rel_l1
from oracle import fco

pytestmark = pytest.mark.gpu

OMEGA, TILT = 2 * math.pi, math.pi / 4
HALF = [0.4, 0.5]          # the half facing (lon, lat) holds 1


def _pair(fc, **kw):
    args = dict(conn=fc.FC_CONN_PILLOW, equation=fc.FC_EQ_ADV, omega=OMEGA, omega_axis_tilt=TILT,
                tag_threshold=0.05, tag_crit=fc.FC_TAG_MAXMIN)
    args.update(kw)
    return make_pair(fc, **args)


def _morton(x, y):
    return sum((((x >> b) & 1) << (2 * b)) | (((y >> b) & 1) << (2 * b + 1)) for b in range(16))


def _two_levels(l0, l1):
    """tree 0 uniform at level l0, tree 1 at level l1: every border between
    the trees, the four singular corners included, is coarse-fine"""
    tr, lv, xs, ys = [], [], [], []
    for t, lev in ((0, l0), (1, l1)):
        w = 1 << lev
        for x, y in sorted(((x, y) for y in range(w) for x in range(w)), key=lambda c: _morton(*c)):
            tr.append(t); lv.append(lev); xs.append(x); ys.append(y)
    return [np.asarray(a, np.int32) for a in (tr, lv, xs, ys)]


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_pillow_forest_uniform_bitexact(level):
    fc = fcmod()
    ctx, ora = _pair(fc, min_level=level, max_level=level)
    ctx.forest_uniform(level)
    ora.uniform(level)
    assert_same_forest(ctx, ora)
    assert np.any(ctx.forest_get_neighbors()[:, :, 3] != 0)   # the half turn across the y borders


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pillow_forest_adapted_bitexact(seed):
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
def test_pillow_singular_corners_coarse_fine_fp64(subcycle):
    fc = fcmod()
    ctx, ora = _pair(fc, min_level=1, max_level=2, subcycle=subcycle)
    leaves = _two_levels(1, 2)
    ctx.forest_set_leaves(*leaves)
    ora.set_leaves(*leaves)
    assert_same_forest(ctx, ora)
    ctx.set_initial(fc.FC_INIT_HALF, [0.3, 0.4])
    ora.init_fields(fco.INIT_HALF, [0.3, 0.4])
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert rr[0] == 0.0, rr
    s0 = ora.sums()[0]
    _run(ctx, ora, 2, 3, regrid=False)
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12)
    assert abs(ctx.conservation_sums()[0] - s0) <= 1e-13 * abs(s0)


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("m,lmin,lmax", [(8, 1, 3), (16, 1, 2)])
def test_pillow_example2_amr_fp64(subcycle, m, lmin, lmax):
    fc = fcmod()
    ctx, ora = _pair(fc, m=m, min_level=lmin, max_level=lmax, subcycle=subcycle)
    ctx.init_refine(fc.FC_INIT_HALF, HALF)
    ora.init_refine(fco.INIT_HALF, HALF)
    assert_same_forest(ctx, ora)
    assert len(set(ora.leaves()[1].tolist())) >= 2
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert rr[0] == 0.0, rr
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-13)
    s0 = ctx.conservation_sums()
    _run(ctx, ora, 3, 2)
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12)
    assert abs(ctx.conservation_sums()[0] - s0[0]) <= 1e-13 * abs(s0[0])


def test_pillow_hill_uniform_m32_fp64():
    fc = fcmod()
    ctx, ora = _pair(fc, m=32, min_level=1, max_level=1)
    ctx.set_initial(fc.FC_INIT_HILL, [0.5, 0.3, 0.35])
    ora.uniform(1)
    ora.init_fields(fco.INIT_HILL, [0.5, 0.3, 0.35])
    _run(ctx, ora, 2, 4, regrid=False)


@pytest.mark.parametrize("subcycle", [0, 1])
def test_pillow_amr_fp32(subcycle):
    fc = fcmod()
    ctx, ora = _pair(fc, m=16, min_level=1, max_level=3, subcycle=subcycle, precision=1)
    ora.init_refine(fco.INIT_HALF, HALF)
    ctx.forest_set_leaves(*ora.leaves())
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


@pytest.mark.parametrize("precision", [0, 1])
def test_pillow_freestream(precision):
    """a constant stays exactly constant without the coarse-fine correction
    and to roundoff with it"""
    fc = fcmod()
    for reflux, tol in ((0, 0.0), (1, 1e-13 if precision == 0 else 1e-6)):
        ctx, ora = _pair(fc, min_level=1, max_level=2, subcycle=1, refluxing=reflux, precision=precision)
        ctx.forest_set_leaves(*_two_levels(1, 2))
        dt = np.float64 if precision == 0 else np.float32
        ctx.write_fields(np.full((ctx.n, 1, 8, 8), 0.75, dt))
        ctx.advance(6)
        q = ctx.read_fields().astype(np.float64)
        assert np.max(np.abs(q - 0.75)) <= tol


def test_pillow_random_regrid_conserves_fp64():
    fc = fcmod()
    ctx, ora = _pair(fc, min_level=1, max_level=3)
    ctx.forest_uniform(2)
    ora.uniform(2)
    ctx.set_initial(fc.FC_INIT_HALF, HALF)
    ora.init_fields(fco.INIT_HALF, HALF)
    s0 = ctx.conservation_sums()[0]
    for r in range(3):
        f = random_forest_flags(ora.n, 70 + r)
        ctx.regrid(f)
        ora.regrid(f)
        assert_same_forest(ctx, ora)
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert rr[0] < FP64_TOL, rr
        assert abs(ctx.conservation_sums()[0] - s0) <= 1e-13 * abs(s0)
