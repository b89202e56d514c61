"""What the learned tagger gains over the plain criterion.

The network is trained on the GPU by the library's own kernels on patches
from hump runs with seeds 1-4 (tiles at time t, plain flags at t + 8 on the
same forest), then both taggers drive an adaptive run of an unseen seed with
regridding every 8 coarse steps.  Against the same problem on the uniform
finest level, the learned tagger (combined with the plain flags) must give a
clearly smaller L1 error in h; the cell-updates of both runs are reported."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_tagger_lowers_error_at_equal_regrid_frequency():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1308_1472_gb300 import tagger

    x, t = tagger.collect(seeds=range(1, 5), snapshots=5)
    xf = tagger.input_transform(x)
    w, losses = tagger.train(tagger.apply_transform(x, xf), t, epochs=10)
    assert losses[-1] < losses[0]
    ev = tagger.evaluate(w, xf, seed=999, steps=32)
    plain, learned = ev["plain_every8"], ev["learned_every8"]
    print(ev)
    assert learned["l1_error"] < 0.8 * plain["l1_error"], ev
    assert learned["regrids"] == plain["regrids"]
