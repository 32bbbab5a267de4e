"""The learned warm start end to end on a small scale: samples generated by the method,
a network trained by the library's kernels, and its gain over the plain iteration on
channels it has not seen -- with the iteration's tolerance still met everywhere."""
import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def test_trained_network_saves_passes_on_unseen_channels():
    from paper_2003_12186_gb300 import learned as LL

    # the workload's own data set: 64 channels, 64 recorded steps (about 2e5 samples);
    # a few thousand samples do not generalise to unseen channels
    X, T, S = LL.generate(count=64, seed=1, spin_up=400, records=64, every=100)
    assert X.shape[1] == 30 and len(X) == len(T) > 150000
    assert np.isfinite(X).all() and np.isfinite(T).all()
    m, norm, rep = LL.train(X, T, epochs=30)
    assert rep["last_loss"] < 0.2 * rep["first_loss"]
    assert rep["val_mse"] < 0.05  # held-out error of the normalised outputs
    ev = LL.evaluate(m, count=16, seed=2, spin_up=400, count_steps=8, timed_steps=32)
    for mode in ("plain", "previous", "mlp"):
        assert ev[mode]["worst_residual"] < LL.TOL and ev[mode]["capped"] == 0
    assert ev["mlp"]["passes_per_step"] < 0.85 * ev["plain"]["passes_per_step"]
