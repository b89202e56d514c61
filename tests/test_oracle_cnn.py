"""Pins of the oracle's learned-tagger network (FP64).

* forward equals an independent numpy evaluation (sliding-window products);
* backward equals central finite differences of the loss (rel. 1e-7);
* the loss equals binary cross-entropy written from its definition.
"""
import numpy as np

from oracle import fco

S = 12


def unpack(w):
    o = 0
    out = []
    for shape in [(16, 3, 3, 3), (16,), (16, 16, 3, 3), (16,), (2, 16, 3, 3), (2,)]:
        n = int(np.prod(shape))
        out.append(w[o:o + n].reshape(shape))
        o += n
    assert o == fco.CNN_NPARAM
    return out


def conv_np(x, w, b):
    Ci, H, _ = x.shape
    win = np.lib.stride_tricks.sliding_window_view(x, (3, 3), axis=(1, 2))  # Ci, H-2, W-2, 3, 3
    return np.einsum("ihwab,oiab->ohw", win, w) + b[:, None, None]


def forward_np(w, x):
    w1, b1, w2, b2, w3, b3 = unpack(w)
    out = []
    for s in range(x.shape[0]):
        a1 = np.maximum(conv_np(x[s], w1, b1), 0)
        a2 = np.maximum(conv_np(a1, w2, b2), 0)
        z = conv_np(a2, w3, b3)
        out.append(z.reshape(2, -1).max(axis=1))
    return np.array(out)


def rand_net(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=fco.CNN_NPARAM) * 0.3
    x = rng.normal(size=(3, 3, S, S))
    t = (rng.random((3, 2)) < 0.5).astype(np.float64)
    return w, x, t


def test_forward_matches_numpy():
    w, x, _ = rand_net(0)
    np.testing.assert_allclose(fco.cnn_forward(w, x), forward_np(w, x), rtol=1e-13, atol=1e-13)


def test_loss_is_bce_of_logits():
    w, x, t = rand_net(1)
    z = forward_np(w, x)
    # -log sigmoid(z) = log(1 + e^-z), -log(1 - sigmoid(z)) = log(1 + e^z)
    ref = (t * np.logaddexp(0.0, -z) + (1 - t) * np.logaddexp(0.0, z)).sum(axis=1).mean()
    loss, _ = fco.cnn_loss_grad(w, x, t)
    assert abs(loss - ref) < 1e-12 * max(1.0, abs(ref))


def test_gradient_matches_finite_differences():
    w, x, t = rand_net(2)
    loss, g = fco.cnn_loss_grad(w, x, t)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(432, 20, replace=False), 432 + np.arange(16),
                          448 + rng.choice(2304, 30, replace=False), 2752 + np.arange(16),
                          2768 + rng.choice(288, 20, replace=False), 3056 + np.arange(2)])
    eps = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += eps
        wm = w.copy(); wm[i] -= eps
        fd = (fco.cnn_loss_grad(wp, x, t)[0] - fco.cnn_loss_grad(wm, x, t)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
