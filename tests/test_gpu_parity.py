"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Bars: forest and neighbour data and tag flags bit-exact; FP64 fields within
1e-12 relative L1 per field; FP32 fields within 2e-5 relative L1 per field;
invariants (translation at Courant 1, lake at rest) bit-exact on the GPU too.
"""
import numpy as np
import pytest

from fc_inputs import dambreak_params, humps_params, random_forest_flags, random_unbalanced_leaves
from gpu_helpers import FP32_TOL, FP64_TOL, assert_same_forest, fcmod, make_pair, rel_l1
from oracle import fco

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("conn", [0, 1])
@pytest.mark.parametrize("level", [0, 1, 3, 5])
def test_forest_uniform_bitexact(conn, level):
    fc = fcmod()
    ctx, ora = make_pair(fc, conn=conn, min_level=0, max_level=8)
    ctx.forest_uniform(level)
    ora.uniform(level)
    assert_same_forest(ctx, ora)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("conn", [0, 1])
def test_forest_random_balance_bitexact(seed, conn):
    fc = fcmod()
    ctx, ora = make_pair(fc, conn=conn, min_level=0, max_level=9)
    lv = np.array(random_unbalanced_leaves(300 + seed, max_level=6), dtype=np.int32)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(lv))             # import order must not matter
    ctx.forest_set_leaves(*[lv[perm, k] for k in range(4)])
    ora.set_leaves(*[lv[:, k] for k in range(4)])
    ctx.forest_balance()
    ora.balance()
    assert_same_forest(ctx, ora)


@pytest.mark.parametrize("seed", range(4))
def test_regrid_topology_bitexact(seed):
    fc = fcmod()
    ctx, ora = make_pair(fc, m=8, min_level=1, max_level=6)
    ctx.forest_uniform(3)
    ora.uniform(3)
    for r in range(3):
        f = random_forest_flags(ora.n, 40 + 7 * seed + r)
        ctx.regrid(f)
        ora.regrid(f)
        assert_same_forest(ctx, ora)


def test_config1_dambreak_fp64():
    """16 patches of m = 8 at level 2 (32 x 32 cells), dam break, 50 CFL steps."""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=8, min_level=2, max_level=2)
    p = dambreak_params()
    ctx.set_initial(fc.FC_INIT_DAMBREAK, p)
    ora.init_fields(fco.INIT_DAMBREAK, p)
    tg, _ = ctx.advance(50)
    to, _ = ora.advance(50)
    assert abs(tg - to) <= 1e-12 * to
    r = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(r < FP64_TOL), r
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("m,lmin,lmax", [(8, 3, 5), (16, 2, 4)])
def test_amr_dambreak_fp64(subcycle, m, lmin, lmax):
    """adaptive dam break, tag + regrid every 4 steps: forest and flags
    bit-exact, fields within 1e-12 relative L1"""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=m, min_level=lmin, max_level=lmax, subcycle=subcycle)
    p = dambreak_params()
    ctx.init_refine(fc.FC_INIT_DAMBREAK, p)
    ora.init_refine(fco.INIT_DAMBREAK, p)
    assert_same_forest(ctx, ora)
    for r in range(4):
        tg, _ = ctx.advance(4)
        to, _ = ora.advance(4)
        assert abs(tg - to) <= 1e-12 * to
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert np.all(rr < FP64_TOL), (r, rr)
        fg, fo = ctx.tag(), ora.tag()
        assert np.array_equal(fg, fo)
        ctx.regrid(fo)
        ora.regrid(fo)
        assert_same_forest(ctx, ora)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP64_TOL), rr
    s0 = ora.sums()
    np.testing.assert_allclose(ctx.conservation_sums(), s0, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("variant", [0, 4, 5, 6])
@pytest.mark.parametrize("subcycle", [0, 1])
def test_amr_fp32_within_tolerance(subcycle, variant):
    """FP32 kernels (every launch shape, the packed two-column sweep
    included) against the FP64 oracle from the same FP32-rounded start"""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=16, min_level=2, max_level=4, subcycle=subcycle, precision=1)
    ctx.set_variant(variant)
    ora.init_refine(fco.INIT_DAMBREAK, dambreak_params())
    tr, lv, x, y = ora.leaves()
    ctx.forest_set_leaves(tr, lv, x, y)
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    dt = 0.25 * ora.next_dt
    ctx.advance(20, dt)
    ora.advance(20, dt)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP32_TOL), rr


@pytest.mark.parametrize("variant", [0, 5])
@pytest.mark.parametrize("subcycle", [0, 1])
@pytest.mark.parametrize("problem", ["dambreak", "humps"])
def test_fp32_at_cfl_09(problem, subcycle, variant):
    """the configured runs' Courant number: each side takes its own CFL 0.9
    step from its own wave speeds (FP32 speeds on the GPU, FP64 in the
    oracle) for 24 steps on a three-level forest, coarse-fine correction on;
    every field within the FP32 bar"""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=16, min_level=2, max_level=4, subcycle=subcycle, precision=1)
    ctx.set_variant(variant)
    if problem == "dambreak":
        ora.init_refine(fco.INIT_DAMBREAK, dambreak_params())
    else:
        ora.init_refine(fco.INIT_HUMPS, humps_params(16, 4))
    ctx.forest_set_leaves(*ora.leaves())
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    for _ in range(3):
        tg, _ = ctx.advance(8)
        to, _ = ora.advance(8)
        assert abs(tg - to) <= 1e-5 * to
    assert ctx.stats()["last_courant"] > 0.8
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP32_TOL), rr


@pytest.mark.parametrize("variant", [0, 5, 6])
def test_sweep_fp32_transonic_dambreak(variant):
    """depth ratio 10: the flow behind the front turns supercritical, so the
    packed sweep's warps take the general forms of the fluctuations and
    transverse splits there (the cell margin u^2 + v^2 < 0.45 g h fails) and
    the subsonic forms elsewhere; against the FP64 oracle"""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=16, min_level=2, max_level=4, subcycle=1, precision=1)
    ctx.set_variant(variant)
    ora.init_refine(fco.INIT_DAMBREAK, [0.5, 0.5, 0.04, 10.0, 1.0])
    tr, lv, x, y = ora.leaves()
    ctx.forest_set_leaves(tr, lv, x, y)
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    dt = 0.25 * ora.next_dt
    for _ in range(3):
        ctx.advance(8, dt)
        ora.advance(8, dt)
    q = ora.fields()
    h = q[:, 0]
    froude2 = (q[:, 1] ** 2 + q[:, 2] ** 2) / (h ** 3)
    assert froude2.max() > 0.45, froude2.max()          # the margin fails somewhere
    rr = rel_l1(ctx.read_fields(), q)
    assert np.all(rr < FP32_TOL), rr


@pytest.mark.parametrize("precision", [0, 1])
def test_translation_courant_one_bitexact(precision):
    fc = fcmod()
    m, lev = 8, 3
    ctx, ora = make_pair(fc, conn=1, equation=1, m=m, min_level=lev, max_level=lev, refluxing=0,
                         adv_u=1.0, adv_v=0.0, precision=precision)
    n = (1 << lev) * m
    rng = np.random.default_rng(9)
    G0 = 1.0 + rng.random((n, n))
    if precision:
        G0 = G0.astype(np.float32).astype(np.float64)
    tr, lv, xs, ys = ora.leaves()
    q = np.zeros((ora.n, 1, m, m))
    for k in range(ora.n):
        q[k, 0] = G0[ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m]
    ctx.write_fields(q)
    steps = 13
    ctx.advance(steps, 1.0 / n)
    q2 = ctx.read_fields().astype(np.float64)
    G1 = np.zeros_like(G0)
    for k in range(ora.n):
        G1[ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m] = q2[k, 0]
    assert np.array_equal(G1, np.roll(G0, steps, axis=1))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("subcycle", [0, 1])
def test_lake_at_rest_bitexact(precision, subcycle):
    fc = fcmod()
    ctx, ora = make_pair(fc, m=8, min_level=3, max_level=5, precision=precision, subcycle=subcycle)
    ctx.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
    q = ctx.read_fields()
    q[:, 0] = 1.375
    q[:, 1:] = 0.0
    ctx.write_fields(q)
    for r in range(3):
        ctx.advance(3)
        ctx.regrid(random_forest_flags(ctx.n, 70 + r))
    q2 = ctx.read_fields()
    assert np.all(q2[:, 0] == 1.375) and np.all(q2[:, 1:] == 0.0)


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
@pytest.mark.parametrize("subcycle", [0, 1])
def test_mass_conservation_gpu(precision, tol, subcycle):
    fc = fcmod()
    ctx, _ = make_pair(fc, m=16, min_level=2, max_level=4, precision=precision, subcycle=subcycle)
    ctx.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
    s0 = ctx.conservation_sums()
    for r in range(4):
        ctx.advance(4)
        ctx.regrid(ctx.tag())
    s1 = ctx.conservation_sums()
    assert abs(s1[0] - s0[0]) / s0[0] < tol


def test_humps_periodic_momentum_fp64():
    fc = fcmod()
    ctx, ora = make_pair(fc, conn=1, m=8, min_level=2, max_level=4, subcycle=1, tag_threshold=0.01)
    p = humps_params(n_humps=6, seed=3, width=(0.05, 0.1))
    ctx.init_refine(fc.FC_INIT_HUMPS, p)
    ora.init_refine(fco.INIT_HUMPS, p)
    assert_same_forest(ctx, ora)
    q = ora.fields()
    q[:, 1] = 0.1 * q[:, 0]
    q[:, 2] = -0.05 * q[:, 0]
    ora.set_fields(q)
    ctx.write_fields(q)
    ctx.advance(10)
    ora.advance(10)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP64_TOL), rr
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-13)


def test_autotune_before_first_step_changes_nothing():
    """the launch-shape trials may run before any step (the coarse-source
    tiles are filled first) and leave the state and the step sequence as they
    were, up to the rounding of a different launch shape (the compiler may
    fuse multiply-adds differently in each)"""
    fc = fcmod()
    runs = []
    for tune in (False, True):
        ctx = fc.Context(m=8, min_level=2, max_level=4, subcycle=1, device=0)
        ctx.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
        if tune:
            ctx.autotune()
        ctx.advance(6)
        runs.append((ctx.read_fields(), ctx.stats()["time"]))
    assert np.all(rel_l1(runs[1][0], runs[0][0]) < 1e-13)
    assert abs(runs[1][1] - runs[0][1]) <= 1e-13 * runs[0][1]


@pytest.mark.parametrize("variant", list(range(7)))
@pytest.mark.parametrize("conn,m", [(0, 8), (1, 16)])
def test_update_variants_match_oracle(variant, conn, m):
    """every launch shape of the fused update (threads per CTA; one CTA per
    patch or persistent CTAs with asynchronous copies of the next patch; the
    row sweep with 1, 2 or 4 columns per lane) against the oracle through
    sub-cycled AMR steps and a regrid"""
    fc = fcmod()
    ctx, ora = make_pair(fc, conn=conn, m=m, min_level=2, max_level=4, subcycle=1)
    p = dambreak_params() if conn == 0 else humps_params(16, 3)
    kind = fc.FC_INIT_DAMBREAK if conn == 0 else fc.FC_INIT_HUMPS
    ctx.init_refine(kind, p)
    ora.init_refine(fco.INIT_DAMBREAK if conn == 0 else fco.INIT_HUMPS, p)
    ctx.set_variant(variant)
    for r in range(2):
        tg, _ = ctx.advance(3)
        to, _ = ora.advance(3)
        assert abs(tg - to) <= 1e-12 * to
        rr = rel_l1(ctx.read_fields(), ora.fields())
        assert np.all(rr < FP64_TOL), (r, rr)
        f = ora.tag()
        ctx.regrid(f)
        ora.regrid(f)
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("variant", [4, 5, 6])
@pytest.mark.parametrize("m", [8, 16])
def test_sweep_global_dt_mixed_levels(variant, m):
    """row sweep under one global dt: a launch covers every level, so the
    patches sharing a warp sit on different levels (own dt/dx, output buffer
    and CFL maximum each), with coarse-fine registers on every side kind"""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=m, min_level=1, max_level=4, subcycle=0)
    p = humps_params(24, 11)
    ctx.init_refine(fc.FC_INIT_HUMPS, p)
    ora.init_refine(fco.INIT_HUMPS, p)
    assert_same_forest(ctx, ora)
    ctx.set_variant(variant)
    tg, _ = ctx.advance(5)
    to, _ = ora.advance(5)
    assert abs(tg - to) <= 1e-12 * to
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP64_TOL), rr
    np.testing.assert_allclose(ctx.conservation_sums(), ora.sums(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("variant", [0, 4, 5, 6])
def test_update_variants_m32_fp32(variant):
    """m = 32 (FP32 only for shallow water): every launch shape against the
    FP64 oracle from the same FP32-rounded start"""
    fc = fcmod()
    ctx, ora = make_pair(fc, m=32, min_level=1, max_level=3, subcycle=1, precision=1)
    ora.init_refine(fco.INIT_HUMPS, humps_params(16, 4))
    tr, lv, x, y = ora.leaves()
    ctx.forest_set_leaves(tr, lv, x, y)
    q32 = ora.fields().astype(np.float32)   # FP32-rounded start, rounded on the host
    ctx.write_fields(q32)
    ora.set_fields(q32.astype(np.float64))
    ctx.set_variant(variant)
    dt = 0.5 * ora.next_dt
    ctx.advance(10, dt)
    ora.advance(10, dt)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP32_TOL), rr


def test_update_variants_fp32_agree():
    fc = fcmod()
    out = []
    for variant in range(7):
        ctx = fc.Context(m=16, min_level=3, max_level=5, precision=fc.FC_FP32, subcycle=1, device=0,
                         tag_threshold=0.01)
        ctx.init_refine(fc.FC_INIT_HUMPS, humps_params(32, 5))
        ctx.set_variant(variant)
        ctx.advance(6)
        out.append(ctx.read_fields().astype(np.float64))
    # FP32 roundings differ between launch shapes (the row sweep sums the
    # transverse parts of a y-edge before subtracting them); the momenta,
    # small in most cells, show it first.  Both bounds sit below the 2e-5
    # relative L1 that the FP32 path keeps against the FP64 oracle.
    for q in out[1:]:
        assert np.all(rel_l1(q, out[0]) < np.array([1e-6, 1e-5, 1e-5]))


def test_set_variant_rejects_unknown():
    fc = fcmod()
    ctx = fc.Context(m=8, min_level=2, max_level=2, device=0)
    with pytest.raises(fc.FCError):
        ctx.set_variant(7)
    adv = fc.Context(equation=fc.FC_EQ_ADV, m=8, min_level=2, max_level=2, device=0)
    with pytest.raises(fc.FCError):
        adv.set_variant(4)
    sph = fc.Context(conn=fc.FC_CONN_SPHERE, equation=fc.FC_EQ_ADV, m=8, min_level=1, max_level=1, device=0)
    with pytest.raises(fc.FCError):
        sph.set_variant(2)


def test_checkpoint_resume_bitexact(tmp_path):
    fc = fcmod()
    a, _ = make_pair(fc, m=8, min_level=3, max_level=5, subcycle=1)
    a.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
    a.advance(3)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.advance(5)
    b, _ = make_pair(fc, m=8, min_level=3, max_level=5, subcycle=1)
    b.load(path)
    b.advance(5)
    assert np.array_equal(a.read_fields(), b.read_fields())
    assert a.stats()["time"] == b.stats()["time"]


def test_degenerate_single_patch_and_zero_steps():
    fc = fcmod()
    ctx, ora = make_pair(fc, m=16, min_level=0, max_level=0)
    p = dambreak_params()
    ctx.set_initial(fc.FC_INIT_DAMBREAK, p)
    ora.init_fields(fco.INIT_DAMBREAK, p)
    before = ctx.read_fields()
    ctx.advance(0)
    assert np.array_equal(before, ctx.read_fields())
    ctx.advance(7)
    ora.advance(7)
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP64_TOL), rr


def test_dry_state_reported_not_faulted():
    fc = fcmod()
    ctx, _ = make_pair(fc, m=8, min_level=1, max_level=1)
    q = np.zeros((ctx.n, 3, 8, 8))
    q[:, 0] = 1.0
    q[0, 0, 3, 3] = -0.5
    ctx.write_fields(q)
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(1, 1e-3)
    assert ei.value.rc == fc.FC_ERR_DRY_STATE


@pytest.mark.parametrize("precision,variant", [(0, 0), (0, 5), (1, 0), (1, 5), (1, 6)])
def test_nonfinite_state_reported_and_recoverable(precision, variant):
    """a NaN momentum is reported as FC_ERR_NONFINITE without a device fault
    (one CTA per patch, the row sweep, the packed and persistent packed
    sweeps); writing a valid state clears the error and stepping resumes"""
    fc = fcmod()
    ctx = fc.Context(m=8, min_level=2, max_level=2, device=0, precision=precision)
    ctx.set_variant(variant)
    ctx.set_initial(fc.FC_INIT_DAMBREAK, dambreak_params())
    good = ctx.read_fields()
    bad = good.copy()
    bad[5, 1, 3, 4] = np.nan
    ctx.write_fields(bad)
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(2, 1e-3)
    assert ei.value.rc == fc.FC_ERR_NONFINITE
    ctx.write_fields(good)
    ctx.advance(2, 1e-3)
    assert np.all(np.isfinite(ctx.read_fields()))


def test_fixed_step_above_courant_one_reported():
    fc = fcmod()
    ctx = fc.Context(m=8, min_level=2, max_level=2, device=0)
    ctx.set_initial(fc.FC_INIT_DAMBREAK, dambreak_params())
    ctx.advance(1)
    dt = ctx.stats()["next_dt"]
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(1, 3.0 * dt)
    assert ei.value.rc == fc.FC_ERR_CFL_VIOLATION
    ctx.set_initial(fc.FC_INIT_DAMBREAK, dambreak_params())
    ctx.advance(2)                                  # cleared by the new state


def test_unbalanced_forest_refused_until_balanced():
    fc = fcmod()
    ctx = fc.Context(m=8, min_level=0, max_level=6, device=0)
    lv = np.array(random_unbalanced_leaves(11, max_level=6), dtype=np.int32)
    ctx.forest_set_leaves(lv[:, 0], lv[:, 1], lv[:, 2], lv[:, 3])
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(1, 1e-4)
    assert ei.value.rc == fc.FC_ERR_UNBALANCED
    ctx.forest_balance()
    ctx.set_initial(fc.FC_INIT_DAMBREAK, dambreak_params())
    ctx.advance(1)


def test_invalid_leaves_and_capacity_errors():
    fc = fcmod()
    ctx = fc.Context(m=8, min_level=1, max_level=3, device=0)
    with pytest.raises(fc.FCError) as ei:        # leaves that overlap
        ctx.forest_set_leaves([0, 0, 0, 0, 0], [1, 1, 1, 1, 2], [0, 1, 0, 1, 0], [0, 0, 1, 1, 0])
    assert ei.value.rc == fc.FC_ERR_INVALID_ARG
    with pytest.raises(fc.FCError) as ei:        # leaves that leave a hole
        ctx.forest_set_leaves([0, 0, 0], [1, 1, 1], [0, 1, 0], [0, 0, 1])
    assert ei.value.rc == fc.FC_ERR_INVALID_ARG
    buf = np.zeros(10, np.float64)
    rc = ctx.L.fc_read_fields(ctx.h, -1, buf.ctypes.data, buf.nbytes, 0)
    assert rc == fc.FC_ERR_CAPACITY
    ctx.forest_uniform(1)                         # still usable
    assert ctx.n == 4


@pytest.mark.parametrize("precision", [0, 1])
def test_field_transfer_pinned_and_pageable(precision):
    """page-locked host buffers are read and written by the layout kernels
    directly, pageable ones through a staging copy: both give the same bytes"""
    torch = pytest.importorskip("torch")
    fc = fcmod()
    ctx = fc.Context(m=16, min_level=2, max_level=3, precision=precision, subcycle=1, device=0)
    ctx.init_refine(fc.FC_INIT_HUMPS, humps_params(8, 2))
    ctx.advance(2)
    ref = ctx.read_fields()                      # pageable numpy
    dt = torch.float64 if precision == 0 else torch.float32
    pinned = torch.empty(ref.shape, dtype=dt).pin_memory()
    fc.check(ctx.L.fc_read_fields(ctx.h, -1, pinned.data_ptr(), pinned.numel() * pinned.element_size(), 0),
             "fc_read_fields")
    assert np.array_equal(pinned.numpy(), ref)
    one = torch.empty(ref.shape[0:1] + ref.shape[2:], dtype=dt).pin_memory()
    fc.check(ctx.L.fc_read_fields(ctx.h, 1, one.data_ptr(), one.numel() * one.element_size(), 0), "fc_read_fields")
    assert np.array_equal(one.numpy(), ref[:, 1])
    # write a modified state from pinned memory, read it back through the pageable path
    mod = torch.from_numpy(ref * 1.5 + 0.25).to(dt).pin_memory()
    fc.check(ctx.L.fc_write_fields(ctx.h, mod.data_ptr(), mod.numel() * mod.element_size(), 0), "fc_write_fields")
    assert np.array_equal(ctx.read_fields(), mod.numpy())
    ctx.write_fields(ref)                        # pageable write
    fc.check(ctx.L.fc_read_fields(ctx.h, -1, pinned.data_ptr(), pinned.numel() * pinned.element_size(), 0),
             "fc_read_fields")
    assert np.array_equal(pinned.numpy(), ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_async_field_transfers_and_two_contexts(precision):
    """the asynchronous transfers give the synchronous ones' bytes; pageable
    host buffers are refused; two contexts on two streams, alternating
    write / step / read as a double-buffered pipeline, each end where the
    same steps taken one context at a time end"""
    torch = pytest.importorskip("torch")
    fc = fcmod()
    dt = torch.float64 if precision == 0 else torch.float32

    def make():
        s = torch.cuda.Stream()
        c = fc.Context(m=16, min_level=2, max_level=3, precision=precision, subcycle=1, device=0,
                       stream=s.cuda_stream)
        c.init_refine(fc.FC_INIT_HUMPS, humps_params(8, 2))
        return c

    a, b = make(), make()
    ref = a.read_fields()
    nb = ref.nbytes
    buf = torch.empty(ref.shape, dtype=dt).pin_memory()
    a.read_fields_async(buf.data_ptr(), nb)
    a.sync()
    assert np.array_equal(buf.numpy(), ref)
    with pytest.raises(fc.FCError) as ei:
        a.read_fields_async(np.zeros_like(ref).ctypes.data, nb)
    assert ei.value.rc == fc.FC_ERR_INVALID_ARG
    # pipeline: both contexts start from the same modified state
    start = torch.from_numpy(ref * 1.01).to(dt).pin_memory()
    outs = [torch.empty_like(start).pin_memory() for _ in range(2)]
    for k in range(6):
        c = (a, b)[k % 2]
        c.write_fields_async(start.data_ptr(), nb)
        c.advance_async(1)
        c.read_fields_async(outs[k % 2].data_ptr(), nb)
    a.sync()
    b.sync()
    solo = make()
    solo.write_fields(start.numpy())
    solo.advance(1)
    want = solo.read_fields()
    for o in outs:
        assert np.array_equal(o.numpy(), want)
