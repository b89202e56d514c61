"""The row sweep takes the subsonic forms of the shallow-water fluctuations
and transverse splits (u_hat - c_hat < 0 < u_hat + c_hat for both normal
directions) for a warp's row when every cell of rows r-2..r satisfies
u^2 + v^2 < 0.45 g h.  The claim behind it: the Roe averages of two such
cells satisfy |u_hat|, |v_hat| < sqrt(0.9) c_hat, whatever their depth
ratio (|u_hat| <= max_k |u_k| / c_k * sqrt(2) * c_hat).  Checked here on
random pairs, depth ratios up to 1e12, in FP64 and in the kernel's FP32
arithmetic, and on the worst case (one depth tending to zero)."""
import numpy as np

G = 1.0
MARGIN = 0.45


def _pairs(rng, n, dtype):
    lh = rng.uniform(-6.0, 6.0, size=(2, n))
    h = (10.0 ** lh).astype(dtype)
    # speeds up to the margin, in random directions
    r = np.sqrt(MARGIN * G * h.astype(np.float64)) * rng.uniform(0.0, 1.0, size=(2, n)) * (1 - 1e-6)
    th = rng.uniform(0.0, 2 * np.pi, size=(2, n))
    u = (r * np.cos(th)).astype(dtype)
    v = (r * np.sin(th)).astype(dtype)
    return h, u, v


def _roe(h, u, v, dtype):
    sq = np.sqrt(h).astype(dtype)
    inv = (dtype(1) / (sq[0] + sq[1])).astype(dtype)
    uh = ((sq[0] * u[0] + sq[1] * u[1]) * inv).astype(dtype)
    vh = ((sq[0] * v[0] + sq[1] * v[1]) * inv).astype(dtype)
    ch = np.sqrt(dtype(0.5 * G) * (h[0] + h[1])).astype(dtype)
    return uh, vh, ch


def test_margin_cells_give_subsonic_roe_edges_fp64():
    rng = np.random.default_rng(1)
    h, u, v = _pairs(rng, 200000, np.float64)
    assert np.all(u * u + v * v < MARGIN * G * h)
    uh, vh, ch = _roe(h, u, v, np.float64)
    assert np.all(np.abs(uh) < np.sqrt(0.9) * ch)
    assert np.all(np.abs(vh) < np.sqrt(0.9) * ch)


def test_margin_cells_give_subsonic_roe_edges_fp32():
    rng = np.random.default_rng(2)
    h, u, v = _pairs(rng, 200000, np.float32)
    ok = u * u + v * v < np.float32(MARGIN * G) * h       # the kernel's cell test, FP32
    uh, vh, ch = _roe(h[:, np.all(ok, axis=0)], u[:, np.all(ok, axis=0)], v[:, np.all(ok, axis=0)], np.float32)
    for s in (uh, vh):
        assert np.all(s - ch < 0) and np.all(s + ch > 0)


def test_bound_is_tight_at_a_vanishing_depth():
    """h_R -> 0 with |u_L| at the margin: |u_hat| / c_hat -> sqrt(2 * 0.45)"""
    hL, hR = 1.0, 1e-14
    uL = np.sqrt(MARGIN * G * hL)
    uh, _, ch = _roe(np.array([[hL], [hR]]), np.array([[uL], [0.0]]), np.zeros((2, 1)), np.float64)
    assert abs(abs(uh[0]) / ch[0] - np.sqrt(2 * MARGIN)) < 1e-6
