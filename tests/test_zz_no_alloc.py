"""fc_conservation_sums_noalloc: the allocation-free variant of the
conservation sums, for callers that must not allocate device memory (a
process with a fixed, pre-reserved device-memory budget, or code where an
allocation could stall or fail).  Its scratch is a fixed array inside the
library, shared by every call, so this test makes two calls in a row on
different forests (a larger one, then a smaller one) and checks that each
matches fc_conservation_sums, i.e. that nothing left over from the first
call leaks into the second.  It lives in its own file, collected last."""
import ctypes

import numpy as np
import pytest

from fc_inputs import dambreak_params, humps_params

pytestmark = pytest.mark.gpu

REL_TOL = 1e-13     # the tolerance of the other conservation-sum comparisons


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_1472_gb300 import fc
    return torch, fc


def _noalloc_sums(torch, fc, ctx, precision):
    n, m, F = ctx.n, ctx.m, ctx.F
    dt = torch.float64 if precision == fc.FC_FP64 else torch.float32
    q = torch.empty((n, F, m, m), dtype=dt, device="cuda")
    ctx.read_fields_device(q.data_ptr(), q.numel() * q.element_size())
    _, lv, _, _ = ctx.forest_get_leaves()
    level = torch.from_numpy(lv.astype(np.int32)).cuda()
    out = torch.full((F,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = ctx.L.fc_conservation_sums_noalloc(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(level.data_ptr()),
                                            n, m, F, precision, ctypes.c_void_p(out.data_ptr()), None)
    fc.check(rc, "fc_conservation_sums_noalloc")
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_sums_match_two_calls_in_a_row(precision):
    torch, fc = _setup()
    big = fc.Context(m=16, min_level=3, max_level=5, precision=precision, device=0)
    big.init_refine(fc.FC_INIT_HUMPS, humps_params(n_humps=8, seed=5, width=(0.03, 0.08)))
    big.advance(2)
    small = fc.Context(m=8, min_level=2, max_level=3, precision=precision, device=0)
    small.init_refine(fc.FC_INIT_DAMBREAK, dambreak_params())
    assert small.n < big.n
    for ctx in (big, small):                      # two calls in a row
        got = _noalloc_sums(torch, fc, ctx, precision)
        ref = ctx.conservation_sums()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref, rtol=REL_TOL, atol=1e-15)
    big.close()
    small.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, fc = _setup()
    L = fc.lib()
    rc = L.fc_conservation_sums_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 131073, 16, 3, 0,
                                        ctypes.c_void_p(16), None)
    assert rc == fc.FC_ERR_CAPACITY
    assert b"static scratch" in L.fc_last_error()
