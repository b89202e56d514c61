"""The step graph's launches spread over several streams by their data
dependences (the sub-cycling recursion of Sec. 4 orders a coarse level's
substep only before the finer substeps that read it, and the finest level's
patches without a coarser neighbour read no coarse data at all): the results
must be the same bits as the launches one after another in plan order, both
as a one-stream graph and eagerly (fc_profile_steps), over several steps and
across regrids."""
import numpy as np
import pytest

from fc_inputs import dambreak_params, humps_params
from gpu_helpers import fcmod

pytestmark = pytest.mark.gpu


def _bench_workload(fc, streams, variant):
    ctx = fc.Context(precision=fc.FC_FP32, device=0, m=16, min_level=6, max_level=8, tag_threshold=0.0003,
                     subcycle=1, refluxing=1)
    ctx.init_refine(fc.FC_INIT_HUMPS, humps_params(64, 1))
    ctx.set_variant(variant)
    ctx.set_step_streams(streams)
    return ctx


@pytest.mark.parametrize("variant", [5, 0])
def test_concurrent_step_equals_serial_on_the_benchmark_forest(variant):
    fc = fcmod()
    a = _bench_workload(fc, 3, variant)
    b = _bench_workload(fc, 1, variant)
    c = _bench_workload(fc, 2, variant)
    assert a.stats()["num_leaves"] == 39262
    # levels 6-8: 7 substeps, 8 tile fills, 3 corrections and the step control;
    # on several streams each level-8 substep is two launches (the patches next
    # to level 7, and the others, which need neither fills nor corrections);
    # the longest chain of launches runs through the border launches, the
    # fills that feed them and the corrections of level 7
    assert a.step_schedule() == (23, 3, 13)
    assert b.step_schedule() == (19, 1, 19)
    assert c.step_schedule() == (23, 2, 13)
    q0 = a.read_fields()
    assert np.array_equal(b.read_fields(), q0)
    a.advance(6)
    b.advance(6)
    c.advance(3)
    c.profile_steps(3)
    qa = a.read_fields()
    assert not np.array_equal(qa, q0)
    assert np.array_equal(qa, b.read_fields())
    assert np.array_equal(qa, c.read_fields())
    assert a.stats()["time"] == b.stats()["time"] == c.stats()["time"]


def test_concurrent_step_equals_serial_across_regrids_fp64():
    """four levels of a dam break in FP64, one CTA per patch, tag and regrid
    every two steps (the step graph is updated in place or captured anew)"""
    fc = fcmod()
    ctxs = []
    for streams in (4, 1):
        ctx = fc.Context(precision=fc.FC_FP64, device=0, m=8, min_level=3, max_level=6, tag_threshold=0.02,
                         subcycle=1, refluxing=1)
        ctx.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
        ctx.set_variant(0)
        ctx.set_step_streams(streams)
        ctxs.append(ctx)
    a, b = ctxs
    la, sa, ca = a.step_schedule()
    lb, sb, cb = b.step_schedule()
    assert sb == 1 and cb == lb
    # 4 levels: every finest substep (8 of them) as a border and an interior launch
    assert la == lb + 8
    assert 2 <= sa <= 4 and ca < lb
    for _ in range(4):
        a.advance(2)
        b.advance(2)
        fa, fb = a.tag(), b.tag()
        assert np.array_equal(fa, fb)
        a.regrid(fa)
        b.regrid(fb)
        assert np.array_equal(a.read_fields(), b.read_fields())
    assert a.stats()["regrids"] == 4
    assert np.array_equal(a.conservation_sums(), b.conservation_sums())


def test_step_streams_argument_range():
    fc = fcmod()
    ctx = fc.Context(precision=fc.FC_FP32, device=0, m=8, min_level=2, max_level=2)
    assert ctx.step_schedule() == (2, 1, 2)       # one level: one update and the step control
    for bad in (0, fc.FC_MAX_STEP_STREAMS + 1, -1):
        with pytest.raises(fc.FCError):
            ctx.set_step_streams(bad)
    ctx.set_step_streams(fc.FC_MAX_STEP_STREAMS)
    assert ctx.step_schedule() == (2, 1, 2)
    ctx.set_initial(fc.FC_INIT_DAMBREAK, dambreak_params())
    ctx.advance(2)
