"""GPU parity of the three-dimensional path (octree of m^3 patches,
scalar advection with a constant velocity, periodic cube) against the 3D
oracle through the C ABI: FP64 within 1e-12 relative L1 (and max abs),
FP32 within 2e-5; forests and tag flags bit-exact."""
import numpy as np
import pytest

from gpu_helpers import FP32_TOL, FP64_TOL, fcmod
from oracle.fco3 import INIT_GAUSS, Oracle3, Oracle3Params

pytestmark = pytest.mark.gpu


def _fc3():
    fcmod()
    from paper_1308_1472_gb300 import fc3
    return fc3


def _pair(m=8, lmin=1, lmax=1, precision=0, **kw):
    fc3 = _fc3()
    ctx = fc3.Context3(m=m, min_level=lmin, max_level=lmax, precision=precision, device=0, **kw)
    ora = Oracle3(Oracle3Params(m=m, min_level=lmin, max_level=lmax, **kw))
    return ctx, ora


def _copy_state(ctx, ora, precision):
    lv, x, y, z = ora.leaves()
    ctx.forest_set_leaves(lv, x, y, z)
    if precision:
        q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
        ctx.write_fields(q32)
        ora.set_fields(q32.astype(np.float64))
    else:
        ctx.write_fields(ora.fields())


def _rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def _same_forest(ctx, ora):
    for a, b in zip(ctx.forest_get_leaves(), ora.leaves()):
        assert np.array_equal(a.astype(np.int64), b.astype(np.int64))


@pytest.mark.parametrize("m", [4, 8])
@pytest.mark.parametrize("vel", [(0.6, -0.35, 0.5), (-0.9, 0.2, -0.45)])
@pytest.mark.parametrize("limiter,transverse", [(1, 2), (0, 2), (1, 1), (1, 0)])
def test_uniform_fp64(m, vel, limiter, transverse):
    ctx, ora = _pair(m=m, lmin=2, lmax=2, u=vel[0], v=vel[1], w=vel[2], limiter=limiter, transverse=transverse)
    rng = np.random.default_rng(7)
    ora.set_fields(1.0 + rng.random((ora.n, m, m, m)))
    _copy_state(ctx, ora, 0)
    dt = 0.8 / (m << 2)
    ctx.advance(4, dt)
    ora.advance(4, dt)
    qg, qo = ctx.read_fields(), ora.fields()
    assert _rel(qg, qo) < FP64_TOL
    assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()


def _amr_oracle(m, **kw):
    ora = Oracle3(Oracle3Params(m=m, min_level=2, max_level=4, tag_threshold=0.02, **kw))
    ora.init_refine(INIT_GAUSS, [0.1, 1.0, 0.3, 0.3, 0.3, 0.08])
    return ora


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("m", [4, 8])
def test_amr_steps_tags_and_regrids_fp64(m, subcycle):
    kw = dict(u=0.7, v=0.4, w=-0.55, tag_threshold=0.02)
    ora = _amr_oracle(m, u=kw["u"], v=kw["v"], w=kw["w"], subcycle=subcycle)
    assert len(set(ora.leaves()[0])) == 3
    fc3 = _fc3()
    ctx = fc3.Context3(m=m, min_level=2, max_level=4, device=0, subcycle=subcycle, **kw)
    _copy_state(ctx, ora, 0)
    s0 = ora.sum()
    for r in range(2):
        tg, dg = ctx.advance(3)
        to, do = ora.advance(3)
        assert dg == do and abs(tg - to) <= 1e-15
        qg, qo = ctx.read_fields(), ora.fields()
        assert _rel(qg, qo) < FP64_TOL, r
        assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()
        fg, fo = ctx.tag(), ora.tag()
        assert np.array_equal(fg, fo)
        ctx.regrid(fo)
        ora.regrid(fo)
        _same_forest(ctx, ora)
        assert _rel(ctx.read_fields(), ora.fields()) < FP64_TOL
    assert abs(ctx.conservation_sum() - s0) <= 1e-13 * abs(s0)
    assert abs(ctx.conservation_sum() - ora.sum()) <= 1e-13 * abs(s0)


@pytest.mark.parametrize("m", [4, 8])
@pytest.mark.parametrize("subcycle", [0, 1])
def test_amr_fp32_within_tolerance(subcycle, m):
    ora = _amr_oracle(m, u=-0.5, v=0.65, w=0.3, subcycle=subcycle)
    fc3 = _fc3()
    ctx = fc3.Context3(m=m, min_level=2, max_level=4, precision=1, device=0, u=-0.5, v=0.65, w=0.3,
                       tag_threshold=0.02, subcycle=subcycle)
    _copy_state(ctx, ora, 1)
    dt = 0.5 * ora.next_dt
    ctx.advance(10, dt)
    ora.advance(10, dt)
    assert _rel(ctx.read_fields().astype(np.float64), ora.fields()) < FP32_TOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_courant_one_translates_bitexact(precision, axis):
    vel = [0.0, 0.0, 0.0]
    vel[axis] = 1.0
    ctx, ora = _pair(m=8, lmin=1, lmax=1, precision=precision, u=vel[0], v=vel[1], w=vel[2])
    rng = np.random.default_rng(3)
    q = 1.0 + rng.random((ctx.n, 8, 8, 8))
    q = q.astype(np.float32 if precision else np.float64)
    ctx.write_fields(q)
    ora.set_fields(q.astype(np.float64))
    ctx.advance(1, 1.0 / 16)
    ora.advance(1, 1.0 / 16)
    assert np.array_equal(ctx.read_fields().astype(np.float64), ora.fields())


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_constant_state_on_amr_bitexact(precision, subcycle):
    ora = _amr_oracle(8, u=0.6, v=-0.5, w=0.4)
    fc3 = _fc3()
    ctx = fc3.Context3(m=8, min_level=2, max_level=4, precision=precision, device=0, u=0.6, v=-0.5, w=0.4,
                       subcycle=subcycle)
    lv, x, y, z = ora.leaves()
    ctx.forest_set_leaves(lv, x, y, z)
    ctx.write_fields(np.full((ctx.n, 8, 8, 8), 1.25, np.float32 if precision else np.float64))
    ctx.advance(3)
    assert np.all(ctx.read_fields() == 1.25)


def test_errors_reported():
    fc3 = _fc3()
    from paper_1308_1472_gb300 import fc
    ctx = fc3.Context3(m=4, min_level=1, max_level=3, device=0)
    # one leaf at level 3 beside level-1 leaves: unbalanced
    lv = [1] * 7 + [3] * 64
    leaves = [(1, x, y, z) for z in range(2) for y in range(2) for x in range(2)][1:]
    fine = [(3, x, y, z) for z in range(4) for y in range(4) for x in range(4)]
    lv, X, Y, Z = zip(*sorted(fine + leaves, key=lambda t: _key(*t)))
    with pytest.raises(fc.FCError) as ei:
        ctx.forest_set_leaves(lv, X, Y, Z)
    assert ei.value.rc == fc.FC_ERR_UNBALANCED
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(1, 1.5 / 8)
    assert ei.value.rc == fc.FC_ERR_CFL_VIOLATION
    with pytest.raises(fc.FCError) as ei:
        ctx.write_fields(np.zeros(3))
    assert ei.value.rc == fc.FC_ERR_CAPACITY
    ctx.advance(0)
    ctx.close()


def _key(l, x, y, z, L=20):
    s = L - l
    k = 0
    for b in range(L):
        k |= (((x << s) >> b) & 1) << (3 * b) | (((y << s) >> b) & 1) << (3 * b + 1) | (((z << s) >> b) & 1) << (3 * b + 2)
    return k


def test_init_refine_matches_oracle_forest():
    fc3 = _fc3()
    ctx = fc3.Context3(m=8, min_level=2, max_level=4, device=0, tag_threshold=0.02)
    ora = Oracle3(Oracle3Params(m=8, min_level=2, max_level=4, tag_threshold=0.02))
    p = [0.1, 1.0, 0.3, 0.3, 0.3, 0.08]
    ctx.init_refine(INIT_GAUSS, p)
    ora.init_refine(INIT_GAUSS, p)
    _same_forest(ctx, ora)
    np.testing.assert_allclose(ctx.read_fields(), ora.fields(), rtol=0, atol=1e-14)


def test_subcycled_step_size_and_cell_updates():
    """sub-cycling: the coarse step is set by the coarsest level, a step
    updates each leaf 2^(l - lmin) times, a Courant number above 1 at the
    coarsest level is refused"""
    fc3 = _fc3()
    from paper_1308_1472_gb300 import fc
    ora = _amr_oracle(8, u=1.0, subcycle=1)
    ctx = fc3.Context3(m=8, min_level=2, max_level=4, device=0, u=1.0, subcycle=1)
    lv, x, y, z = ora.leaves()
    ctx.forest_set_leaves(lv, x, y, z)
    st = ctx.stats()
    assert st["next_dt"] == pytest.approx(ora.next_dt, rel=1e-15)
    assert st["next_dt"] == pytest.approx(0.9 / (8 << int(lv.min())), rel=1e-15)
    ctx.advance(2)
    per = sum(1 << (int(l) - int(lv.min())) for l in lv) * 512
    assert ctx.stats()["cell_updates"] == 2 * per
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(1, 1.01 / (8 << int(lv.min())))
    assert ei.value.rc == fc.FC_ERR_CFL_VIOLATION


@pytest.mark.parametrize("seed", [11, 12, 13])
@pytest.mark.parametrize("subcycle", [0, 1])
def test_random_regrid_sequences_fp64(seed, subcycle):
    """random refine / coarsen flags on both sides, steps in between: forests
    bit for bit, fields within 1e-12 (balance, tables, transfer, sub-cycling
    on forest shapes the fixed cases do not reach)"""
    fc3 = _fc3()
    rng = np.random.default_rng(seed)
    kw = dict(m=4, min_level=1, max_level=4, u=0.55, v=-0.35, w=0.6, subcycle=subcycle)
    ctx = fc3.Context3(device=0, **kw)
    ora = Oracle3(Oracle3Params(**kw))
    ora.init(INIT_GAUSS, [0.2, 1.0, 0.3, 0.6, 0.45, 0.2])
    ctx.write_fields(ora.fields())
    for r in range(4):
        lv = ora.leaves()[0]
        flags = rng.choice(np.array([-1, 0, 1], np.int8), size=ora.n, p=[0.35, 0.4, 0.25])
        ora.regrid(flags)
        ctx.regrid(flags)
        _same_forest(ctx, ora)
        assert _rel(ctx.read_fields(), ora.fields()) < FP64_TOL, r
        ctx.advance(2)
        ora.advance(2)
        qg, qo = ctx.read_fields(), ora.fields()
        assert _rel(qg, qo) < FP64_TOL, r
        assert np.abs(qg - qo).max() <= 1e-12 * np.abs(qo).max()
    assert abs(ctx.conservation_sum() - ora.sum()) <= 1e-13 * abs(ora.sum())


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("limiter,transverse", [(0, 2), (1, 1), (0, 0)])
def test_amr_scheme_options_fp64(limiter, transverse, subcycle):
    """the scheme's options (limiter off, transverse without corner terms,
    neither) on a three-level forest, both time-stepping modes"""
    kw = dict(u=0.45, v=-0.6, w=0.35, limiter=limiter, transverse=transverse, subcycle=subcycle)
    ora = _amr_oracle(4, **kw)
    fc3 = _fc3()
    ctx = fc3.Context3(m=4, min_level=2, max_level=4, device=0, tag_threshold=0.02, **kw)
    _copy_state(ctx, ora, 0)
    ctx.advance(3)
    ora.advance(3)
    qg, qo = ctx.read_fields(), ora.fields()
    assert _rel(qg, qo) < FP64_TOL
    assert abs(ctx.conservation_sum() - ora.sum()) <= 1e-13 * abs(ora.sum())


@pytest.mark.parametrize("m", [4, 8])
def test_single_patch_and_zero_steps(m):
    """one patch at level 0: every neighbour is the patch itself through the
    periodic wrap; zero steps change nothing"""
    fc3 = _fc3()
    kw = dict(m=m, min_level=0, max_level=0, u=0.7, v=-0.45, w=0.3)
    ctx = fc3.Context3(device=0, **kw)
    ora = Oracle3(Oracle3Params(**kw))
    assert ctx.n == 1 and ora.n == 1
    ora.init(INIT_GAUSS, [0.1, 1.0, 0.4, 0.5, 0.6, 0.2])
    ctx.write_fields(ora.fields())
    t0, _ = ctx.advance(0)
    assert t0 == 0.0 and np.array_equal(ctx.read_fields(), ora.fields())
    ctx.advance(5)
    ora.advance(5)
    assert _rel(ctx.read_fields(), ora.fields()) < FP64_TOL
    assert abs(ctx.conservation_sum() - ora.sum()) <= 1e-14 * abs(ora.sum())
