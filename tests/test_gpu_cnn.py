"""Learned-tagger kernels vs the FP64 oracle (gradients checked by central
differences in tests/test_oracle_cnn.py).  Bars: with FP32 weights the
logits and every gradient tensor agree to 1e-5 relative L2.  With BF16
weights and activations the bar is 4u, u = 2^-8 the BF16 unit roundoff: every
product on a gradient path takes a rounded weight and up to three rounded
operands (input, first and second hidden activation), each within u."""
import ctypes

import numpy as np
import pytest

from oracle import fco

pytestmark = pytest.mark.gpu

TENSORS = [("w1", 0, 432), ("b1", 432, 448), ("w2", 448, 2752), ("b2", 2752, 2768), ("w3", 2768, 3056),
           ("b3", 3056, 3058)]


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_1472_gb300 import fc
    return torch, fc


def _bf16(a):
    """round float32 values to the nearest BF16 (ties to even), kept as float32"""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _data(seed, n=37, S=20, feature=False):
    rng = np.random.default_rng(seed)
    # He-style scale so that activations stay O(1) through the three layers
    w = np.concatenate([rng.normal(size=432) * np.sqrt(2 / 27), np.zeros(16) + 0.01,
                        rng.normal(size=2304) * np.sqrt(2 / 144), np.zeros(16) + 0.01,
                        rng.normal(size=288) * np.sqrt(2 / 144), np.zeros(2)]).astype(np.float32)
    x = rng.normal(size=(n, 3, S, S)).astype(np.float32)
    if feature:
        # a localized feature per sample (like a front in a patch), so the
        # pooled maximum is not a near-tie that rounding could move
        x *= 0.2
        ii, jj = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
        for k in range(n):
            ci, cj = rng.integers(min(4, S // 2), max(S - 4, S // 2 + 1), size=2)
            x[k, 0] += 3.0 * np.exp(-((ii - ci) ** 2 + (jj - cj) ** 2) / 3.0)
    t = (rng.random((n, 2)) < 0.4).astype(np.float32)
    return w, x, t


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


BF16_TOL = 4 * 2.0 ** -8


@pytest.mark.parametrize("bf16,tol", [(0, 1e-5), (1, BF16_TOL)])
def test_forward_and_gradients_match_oracle(bf16, tol):
    torch, fc = _setup()
    L = fc.lib()
    w, x, t = _data(11, feature=bool(bf16))
    if bf16:
        # the oracle sees the same BF16-representable input and weights, so the
        # comparison measures the kernels' rounding of activations and sums
        x = _bf16(x)
        w = np.concatenate([_bf16(w[:432]), w[432:448], _bf16(w[448:2752]), w[2752:2768],
                            _bf16(w[2768:3056]), w[3056:]]).astype(np.float32)
    n, S = x.shape[0], x.shape[-1]
    dw, dx, dt = (torch.from_numpy(a).cuda() for a in (w, x, t))
    logits = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    grad = torch.zeros(3058, dtype=torch.float32, device="cuda")
    loss = ctypes.c_float()
    fc.check(L.fc_cnn_forward(n, S, dw.data_ptr(), dx.data_ptr(), logits.data_ptr(), bf16, None), "forward")
    fc.check(L.fc_cnn_loss_grad(n, S, dw.data_ptr(), dx.data_ptr(), dt.data_ptr(), grad.data_ptr(),
                                ctypes.byref(loss), bf16, None), "loss_grad")
    ref_logits = fco.cnn_forward(w.astype(np.float64), x.astype(np.float64))
    ref_loss, ref_grad = fco.cnn_loss_grad(w.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert _rel(logits.cpu().numpy(), ref_logits) < tol
    assert abs(loss.value - ref_loss) <= tol * abs(ref_loss)
    g = grad.cpu().numpy()
    errs = {name: _rel(g[a:b], ref_grad[a:b]) for name, a, b in TENSORS}
    assert max(errs.values()) < tol, errs


def test_adam_step_closed_form():
    torch, fc = _setup()
    L = fc.lib()
    rng = np.random.default_rng(3)
    w = rng.normal(size=3058).astype(np.float32)
    g = rng.normal(size=3058).astype(np.float32)
    m1 = rng.normal(size=3058).astype(np.float32) * 0.1
    m2 = np.abs(rng.normal(size=3058)).astype(np.float32) * 0.01
    dw, dg, dm1, dm2 = (torch.from_numpy(a.copy()).cuda() for a in (w, g, m1, m2))
    step, lr = 7, 1e-3
    fc.check(L.fc_cnn_adam(dw.data_ptr(), dg.data_ptr(), dm1.data_ptr(), dm2.data_ptr(), step, ctypes.c_float(lr),
                           None), "adam")
    torch.cuda.synchronize()
    a = 0.9 * m1.astype(np.float64) + 0.1 * g
    v = 0.999 * m2.astype(np.float64) + 0.001 * g.astype(np.float64) ** 2
    ref = w - lr * (a / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    np.testing.assert_allclose(dw.cpu().numpy(), ref, rtol=2e-5, atol=2e-6)


def test_training_reduces_loss():
    torch, fc = _setup()
    L = fc.lib()
    w, x, _ = _data(5, n=256)
    # a learnable target: refine iff the first channel's range is large
    rng_t = (x[:, 0].max(axis=(1, 2)) - x[:, 0].min(axis=(1, 2)))
    t = np.stack([rng_t > np.median(rng_t), rng_t < np.quantile(rng_t, 0.25)], axis=1).astype(np.float32)
    n, S = x.shape[0], x.shape[-1]
    dw, dx, dt = (torch.from_numpy(a).cuda() for a in (w, x, t))
    m1 = torch.zeros_like(dw)
    m2 = torch.zeros_like(dw)
    g = torch.zeros_like(dw)
    loss = ctypes.c_float()
    losses = []
    for step in range(1, 61):
        fc.check(L.fc_cnn_loss_grad(n, S, dw.data_ptr(), dx.data_ptr(), dt.data_ptr(), g.data_ptr(),
                                    ctypes.byref(loss), 1, None), "loss_grad")
        fc.check(L.fc_cnn_adam(dw.data_ptr(), g.data_ptr(), m1.data_ptr(), m2.data_ptr(), step,
                               ctypes.c_float(3e-3), None), "adam")
        losses.append(loss.value)
    assert losses[-1] < 0.7 * losses[0], losses[::10]


def _bf16_params(w):
    return np.concatenate([_bf16(w[:432]), w[432:448], _bf16(w[448:2752]), w[2752:2768], _bf16(w[2768:3056]),
                           w[3056:]]).astype(np.float32)


@pytest.mark.parametrize("S,n", [(7, 40), (20, 1500), (36, 400)])
def test_tensor_core_forward_matches_oracle(S, n):
    """BF16 inference on the tensor cores (one MMA per 3x3 tap and 128 output
    positions, accumulators in tensor memory) against the FP64 oracle, at the
    BF16 bar; n large enough that every CTA takes several samples (the
    accumulators and the completion barrier are reused), S from the smallest
    input to the m = 32 patch plus ghosts"""
    torch, fc = _setup()
    L = fc.lib()
    w, x, _ = _data(17 + S, n=n, S=S, feature=True)
    x = _bf16(x)
    w = _bf16_params(w)
    dw, dx = (torch.from_numpy(a).cuda() for a in (w, x))
    logits = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    fc.check(L.fc_cnn_forward(n, S, dw.data_ptr(), dx.data_ptr(), logits.data_ptr(), 1, None), "forward")
    ref = fco.cnn_forward(w.astype(np.float64), x.astype(np.float64))
    got = logits.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert _rel(got, ref) < BF16_TOL
    # sample by sample as well: every logit within the bar of its sample's scale
    scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-3)
    assert np.max(np.abs(got - ref) / scale) < 4 * BF16_TOL


def test_tensor_core_forward_timeout_is_reported():
    """a wait limit of zero polls makes every tile's completion wait give up:
    the call reports FC_ERR_TIMEOUT (the kernel still lets its MMAs finish
    before freeing their tensor memory), and with the limit restored the
    device computes the same logits as before"""
    torch, fc = _setup()
    L = fc.lib()
    w, x, _ = _data(23, n=64, feature=True)
    x = _bf16(x)
    w = _bf16_params(w)
    dw, dx = (torch.from_numpy(a).cuda() for a in (w, x))
    a = torch.zeros((64, 2), dtype=torch.float32, device="cuda")
    b = torch.zeros((64, 2), dtype=torch.float32, device="cuda")
    fc.check(L.fc_cnn_forward(64, 20, dw.data_ptr(), dx.data_ptr(), a.data_ptr(), 1, None), "forward")
    try:
        fc.check(L.fc_cnn_set_wait_limit(0), "set_wait_limit")
        rc = L.fc_cnn_forward(64, 20, dw.data_ptr(), dx.data_ptr(), b.data_ptr(), 1, None)
        assert rc == fc.FC_ERR_TIMEOUT
    finally:
        fc.check(L.fc_cnn_set_wait_limit(1 << 24), "set_wait_limit")
    assert L.fc_cnn_set_wait_limit(-1) == fc.FC_ERR_INVALID_ARG
    fc.check(L.fc_cnn_forward(64, 20, dw.data_ptr(), dx.data_ptr(), b.data_ptr(), 1, None), "forward")
    assert torch.equal(a, b)
