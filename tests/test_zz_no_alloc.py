"""iilbm_get_macros_noalloc, the read-out that allocates no device memory.

It exists for callers that must not allocate at the moment they read results: code
whose device memory belongs to a caching allocator or a fixed budget (a cudaMalloc
there may fail or fragment the pool) and tight stepping loops, where cudaMalloc and
cudaFree would synchronise the whole device.  It stages the fields in a static device
array of the library instead.  This file checks, through the C ABI, that it returns
what iilbm_get_macros returns, on two calls in a row, and that lattices larger than
the array are refused.  It is collected last on purpose."""
import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def _membrane(storage):
    w = W.ellipse_scaled(256, storage)
    g = iilbm.Lattice(256, 256, collision=iilbm.MRT, storage=storage, tau=w["tau"],
                      s=W.mrt_rates(w["tau"]))
    g.set_interface(w["X"], model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
    return g


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_noalloc_matches_get_macros_on_two_calls_in_a_row(storage):
    g = _membrane(storage)
    for steps in (37, 5):  # two calls in a row, state advanced in between
        g.step(steps)
        ref = g.iilbm_get_macros()
        got = g.iilbm_get_macros_noalloc()
        for a, b in zip(ref, got):
            scale = max(np.abs(a).max(), 1e-30)
            assert np.abs(a - b).max() <= 1e-12 * scale
        assert np.abs(got[1]).max() > 0  # the membrane has set the fluid in motion


def test_noalloc_into_device_buffers():
    torch = pytest.importorskip("torch")
    g = _membrane("f32")
    g.step(12)
    ref = g.iilbm_get_macros()
    d = [torch.empty((256, 256), dtype=torch.float64, device="cuda") for _ in range(3)]
    g.iilbm_get_macros_noalloc(*d)
    for a, b in zip(ref, d):
        assert np.abs(a - b.cpu().numpy()).max() <= 1e-12 * max(np.abs(a).max(), 1e-30)


def test_noalloc_refuses_lattices_beyond_its_array():
    g = iilbm.Lattice(1024, 512, collision=iilbm.MRT, storage="f32", tau=0.7)
    with pytest.raises(iilbm.IilbmError) as e:
        g.iilbm_get_macros_noalloc()
    assert e.value.code == -7  # IILBM_ERR_CAPACITY
