"""The benchmark's workload at its full size (one quadtree, levels 6-8,
m = 16, 64 humps, seed 1, gradient tagging threshold 0.0003: 39,262
leaves, 10.1 M cells), FP32, in the launch shapes the benchmark times.  The
forest and the initial state are the oracle's (its FP64 initial refinement
gives the same 39,262 leaves), rounded to FP32 on the host and written into
the library, so that both sides start from identical data:

  * the benchmark's own step in full: one sub-cycled coarse step (level 8
    takes four substeps) with the coarse-fine correction on and the launch
    shape of every level from the autotuner, every cell of every field
    against the oracle's sub-cycled step (FP32 tolerance, 2e-5 relative L1
    per field);
  * sampled patches: one step of one global dt with the packed row sweep (a
    global-dt launch covers all three levels), each sampled patch against
    the oracle's update of the same patch from the oracle's own ghost fill
    of the same forest and state (2e-5 relative L1 per field over the
    sampled patches, and per patch for the depth);
  * properties that hold at any size, in the benchmark's own configuration:
    mass conserved to FP32 round-off over four coarse steps, and a lake at
    rest that stays at rest bit for bit.
"""
import numpy as np
import pytest

from fc_inputs import humps_params
from gpu_helpers import FP32_TOL, fcmod, rel_l1
from oracle import fco
from oracle.fco import Oracle, OracleParams

pytestmark = pytest.mark.gpu

W = dict(m=16, min_level=6, max_level=8, tag_threshold=0.0003)
HUMPS = (64, 1)


@pytest.fixture(scope="module")
def oracle_start():
    """the oracle's initial refinement of the workload: leaves and the
    FP32-rounded initial state"""
    ora = Oracle(OracleParams(**W))
    ora.init_refine(fco.INIT_HUMPS, humps_params(*HUMPS))
    assert ora.n == 39262
    return ora.leaves(), ora.fields().astype(np.float32)


def _context(fc, **kw):
    ctx = fc.Context(precision=fc.FC_FP32, device=0, **W, **kw)
    ctx.init_refine(fc.FC_INIT_HUMPS, humps_params(*HUMPS))
    return ctx


def test_full_size_benchmark_step_against_oracle(oracle_start):
    fc = fcmod()
    leaves, q32 = oracle_start
    ora = Oracle(OracleParams(subcycle=1, refluxing=1, **W))
    ora.set_leaves(*leaves)
    ora.set_fields(q32.astype(np.float64))
    dt = ora.next_dt                            # CFL 0.9 from the cell speeds of the start state
    assert dt > 0.0
    ctx = fc.Context(precision=fc.FC_FP32, device=0, subcycle=1, refluxing=1, **W)
    ctx.forest_set_leaves(*leaves)
    ctx.write_fields(q32)
    ctx.autotune()
    assert np.array_equal(ctx.read_fields(), q32)   # the trials leave the state as it was
    _, dt1 = ctx.advance(1, dt)
    assert dt1 == dt
    ora.advance(1, dt)
    assert ctx.stats()["cell_updates"] == ora.cell_updates == 38033664
    rr = rel_l1(ctx.read_fields(), ora.fields())
    assert np.all(rr < FP32_TOL), rr


def test_full_size_sampled_patches_against_oracle(oracle_start):
    fc = fcmod()
    (tr, lv, x, y), q32 = oracle_start
    n = len(tr)
    ctx = fc.Context(precision=fc.FC_FP32, device=0, subcycle=0, refluxing=0, **W)
    ctx.forest_set_leaves(tr, lv, x, y)
    ctx.write_fields(q32)
    ctx.set_variant(5)                         # packed row sweep
    ora = Oracle(OracleParams(refluxing=0, **W))
    ora.set_leaves(tr, lv, x, y)
    ora.set_fields(q32.astype(np.float64))
    pads = ora.fill_ghosts()
    dt = ora.next_dt                           # CFL 0.9 from the cell speeds of the same state
    assert dt > 0.0
    t1, dt1 = ctx.advance(1, dt)
    assert dt1 == dt
    q1 = ctx.read_fields().astype(np.float64)
    rng = np.random.default_rng(5)
    # random patches of every level, plus patches on the walls and next to each level change
    sample = set(rng.choice(n, 160, replace=False).tolist())
    for l in (6, 7, 8):
        sample |= set(rng.choice(np.nonzero(lv == l)[0], 16, replace=False).tolist())
    walls = np.nonzero((x == 0) | (y == 0) | (x == (1 << lv.astype(np.int64)) - 1) | (y == (1 << lv.astype(np.int64)) - 1))[0]
    sample |= set(rng.choice(walls, 16, replace=False).tolist())
    ks = sorted(sample)
    ref = np.stack([fco.patch_step(fco.EQ_SWE, pads[k], 1.0 / (16 << int(lv[k])), 1.0 / (16 << int(lv[k])), dt)[0]
                    for k in ks])
    # relative L1 per field over the sampled patches (the bar of the whole
    # run); the depth also patch by patch
    rr = rel_l1(q1[ks], ref)
    assert np.all(rr < FP32_TOL), rr
    per_patch_h = np.abs(q1[ks, 0] - ref[:, 0]).sum(axis=(1, 2)) / np.abs(ref[:, 0]).sum(axis=(1, 2))
    assert per_patch_h.max() < FP32_TOL, per_patch_h.max()


def test_full_size_benchmark_configuration_properties():
    fc = fcmod()
    ctx = _context(fc, subcycle=1)
    assert ctx.stats()["num_leaves"] == 39262
    ctx.autotune()
    s0 = ctx.conservation_sums()
    ctx.advance(4)
    s1 = ctx.conservation_sums()
    assert abs(s1[0] - s0[0]) <= 1e-6 * abs(s0[0])
    # a lake at rest on the same forest stays at rest, bit for bit
    q = ctx.read_fields()
    lake = np.zeros_like(q)
    lake[:, 0] = 1.5
    ctx.write_fields(lake)
    ctx.advance(2)
    assert np.array_equal(ctx.read_fields(), lake)


def test_maximum_size_every_leaf_at_level_8():
    """the configuration's largest forest, every leaf at level 8 (65,536
    patches of m = 16, 16.8 M cells, FP32): the oracle's humps on it, one
    CFL 0.9 step of the packed sweep; sampled patches (every wall, corner
    and a random sample) against the oracle's update from its own ghost
    fill, per field over the sample; mass conserved by the step to FP32
    round-off"""
    fc = fcmod()
    ora = Oracle(OracleParams(refluxing=0, **W))
    ora.uniform(8)
    ora.init_fields(fco.INIT_HUMPS, humps_params(*HUMPS))
    q32 = ora.fields().astype(np.float32)
    ora.set_fields(q32.astype(np.float64))
    tr, lv, x, y = ora.leaves()
    n = len(tr)
    assert n == 65536
    ctx = fc.Context(precision=fc.FC_FP32, device=0, subcycle=0, refluxing=0, **W)
    ctx.forest_set_leaves(tr, lv, x, y)
    ctx.write_fields(q32)
    ctx.set_variant(5)
    s0 = ctx.conservation_sums()
    pads = ora.fill_ghosts()
    dt = ora.next_dt
    ctx.advance(1, dt)
    q1 = ctx.read_fields().astype(np.float64)
    rng = np.random.default_rng(8)
    last = 255
    ks = set(rng.choice(n, 200, replace=False).tolist())
    ks |= set(np.nonzero((x == 0) | (y == 0) | (x == last) | (y == last))[0][::16].tolist())
    ks |= set(np.nonzero(((x == 0) | (x == last)) & ((y == 0) | (y == last)))[0].tolist())
    ks = sorted(ks)
    dx = 1.0 / (16 << 8)
    ref = np.stack([fco.patch_step(fco.EQ_SWE, pads[k], dx, dx, dt)[0] for k in ks])
    rr = rel_l1(q1[ks], ref)
    assert np.all(rr < FP32_TOL), rr
    s1 = ctx.conservation_sums()
    assert abs(s1[0] - s0[0]) <= 1e-6 * abs(s0[0])
