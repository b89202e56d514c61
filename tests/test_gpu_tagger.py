"""What the learned tagger gains over the plain criterion.

The network is trained on the GPU by the library's own kernels on patches
from hump runs with seeds 1-4 (tiles at time t, plain flags at t + 8 on the
same forest; input statistics and normalisation by the library too), then
both taggers drive adaptive runs of an unseen seed, regridding every 8
coarse steps, at several tag thresholds.  Against the same problem on the
uniform finest level, each threshold gives a point (cell-updates, L1 error
in h); the plain criterion's points trace its cost-error curve.  The learned
tagger (combined with the plain flags) must lie below that curve: at equal
cell-updates a clearly smaller error at every threshold inside the curve's
range, and at equal error fewer cell-updates than the plain criterion."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def test_input_statistics_and_normalisation_match_their_definition():
    torch = _torch()
    from paper_1308_1472_gb300 import tagger
    rng = np.random.default_rng(4)
    xh = rng.normal(size=(37, 3, 20, 20)) * np.array([0.1, 0.3, 0.2])[None, :, None, None]
    xh[:, 0] += 1.25
    xh = xh.astype(np.float32)
    x = torch.from_numpy(xh).cuda()
    xf = tagger.input_transform(x)
    v = xh.astype(np.float64)
    mean = v.mean(axis=(0, 2, 3))
    sd = np.sqrt(((v - mean[None, :, None, None]) ** 2).mean(axis=(0, 2, 3)))
    np.testing.assert_allclose(xf, [mean[0], 1 / sd[0], 1 / sd[1], 1 / sd[2]], rtol=1e-12)
    tagger.apply_transform(x, xf)
    ref = np.empty_like(v)
    ref[:, 0] = (v[:, 0] - xf[0]) * xf[1]
    ref[:, 1] = v[:, 1] * xf[2]
    ref[:, 2] = v[:, 2] * xf[3]
    assert np.array_equal(x.cpu().numpy(), ref.astype(np.float32))


def test_learned_tagger_below_the_plain_cost_error_curve():
    _torch()
    from paper_1308_1472_gb300 import tagger

    x, t = tagger.collect(seeds=range(1, 5), snapshots=5)
    xf = tagger.input_transform(x)
    w, losses = tagger.train(tagger.apply_transform(x, xf), t, epochs=10)
    assert losses[-1] < losses[0]
    pa = tagger.pareto(w, xf, thresholds=(0.003, 0.002, 0.0015, 0.001), every=8, seed=999, steps=32)
    print(pa)
    inside = [c for c in pa["comparison"] if c["plain_error_at_same_cell_updates"] is not None]
    assert len(inside) >= 2, pa
    for c in inside:                  # equal cost: smaller error
        assert c["l1_error"] < 0.9 * c["plain_error_at_same_cell_updates"], c
    fewer = [c for c in pa["comparison"] if c["plain_cell_updates_at_same_error"] is not None
             and c["cell_updates"] < c["plain_cell_updates_at_same_error"]]
    assert fewer, pa                  # equal error: fewer cell-updates
    assert all(p["regrids"] == q["regrids"] for p, q in zip(pa["plain"], pa["learned"]))
