"""Shared helpers of the GPU parity tests (CUDA library vs oracle)."""
import numpy as np
import pytest

from oracle import fco
from oracle.fco import Oracle, OracleParams

FP64_TOL = 1e-12     # relative L1 per field, FP64 kernels vs FP64 oracle
FP32_TOL = 2e-5      # relative L1 per field, FP32 kernels vs FP64 oracle


def fcmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_1472_gb300 import fc
    return fc


def make_pair(fc, conn=0, m=8, min_level=2, max_level=2, equation=0, precision=0, subcycle=0,
              tag_crit=0, refluxing=1, g=1.0, cfl=0.9, tag_threshold=0.05, adv_u=1.0, adv_v=0.0,
              omega=0.0, omega_axis_tilt=0.0):
    ctx = fc.Context(conn=conn, m=m, min_level=min_level, max_level=max_level, equation=equation,
                     precision=precision, subcycle=subcycle, tag_crit=tag_crit, refluxing=refluxing, device=0,
                     g=g, cfl=cfl, tag_threshold=tag_threshold, adv_u=adv_u, adv_v=adv_v, omega=omega,
                     omega_axis_tilt=omega_axis_tilt)
    ora = Oracle(OracleParams(conn=conn, m=m, min_level=min_level, max_level=max_level, equation=equation,
                              subcycle=subcycle, tag_crit=tag_crit, refluxing=refluxing, g=g, cfl=cfl,
                              tag_threshold=tag_threshold, adv_u=adv_u, adv_v=adv_v, omega=omega,
                              omega_axis_tilt=omega_axis_tilt))
    return ctx, ora


def rel_l1(a, b):
    """relative L1 difference per field of [n][F][m][m] arrays"""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    num = np.abs(a - b).sum(axis=(0, 2, 3))
    den = np.abs(b).sum(axis=(0, 2, 3))
    return num / np.maximum(den, 1e-300)


def assert_same_forest(ctx, ora):
    g = ctx.forest_get_leaves()
    o = ora.leaves()
    for a, b in zip(g, o):
        assert np.array_equal(a, b)
    assert np.array_equal(ctx.forest_get_neighbors(), ora.neighbors())
