"""The D3Q19 II-LBM with 16-bit population storage (FP16 scaled by 2^12, BF16 unscaled;
FP32 arithmetic) against the FP64 oracle: bit-exact storage rounding on the way in and
out, one stream-collide step within the storage's unit roundoff of the oracle's result at
both AA parities, and a moving surface-tension surface within bounds measured against
FP32 storage."""
import numpy as np
import pytest

from oracle import oracle3d as o3
from paper_2003_12186_gb300 import iilbm3d
from paper_2003_12186_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# unit roundoff (half an ulp, relative) of each storage format
UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
SCALE = {"f16": 2.0 ** 12, "bf16": 1.0}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm3d.load()


def bf16_round(x32):
    """Round-to-nearest-even of FP32 values to BF16 (upper 16 bits), finite inputs."""
    u = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def stored(df, storage):
    """What the lattice keeps for the FP64 values df: df x scale rounded to FP32, then to
    the 16-bit format; returned divided by the scale again, in FP64."""
    x32 = (np.asarray(df, np.float64) * SCALE[storage]).astype(np.float32)
    q = x32.astype(np.float16).astype(np.float64) if storage == "f16" else \
        bf16_round(x32).astype(np.float64)
    return q / SCALE[storage]


def pair(n, storage, collision="mrt", tau=0.8, jump=1, force="guo", shape=None):
    nx, ny, nz = shape or (n, n, n)
    cg = iilbm3d.MRT if collision == "mrt" else iilbm3d.SRT
    co = o3.MRT if collision == "mrt" else o3.SRT
    fg = iilbm3d.FORCE_SIMPLE if force == "simple" else iilbm3d.FORCE_GUO
    fo = o3.FORCE_SIMPLE if force == "simple" else o3.FORCE_GUO
    g = iilbm3d.Lattice3D(nx, ny, nz, collision=cg, storage=storage, tau=tau, jump=jump, force=fg)
    o = o3.Oracle3D(nx, ny, nz, collision=co, tau=tau, jump=jump, force=fo)
    return g, o


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_storage_round_trip_is_the_formats_rounding(storage):
    """set_populations rounds df x scale once (via FP32) to the format, get_populations
    returns it exactly: bit for bit what numpy's rounding gives, at both parities."""
    nx, ny, nz = 19, 13, 9
    g = iilbm3d.Lattice3D(nx, ny, nz, storage=storage)
    df = W.random_df3(nx, ny, nz, 3e-3, 5)
    df[0, 0, 0, :4] = [0.0, 1e-12, -7e-9, 2.5]  # zero, FP16 subnormals, a large value
    want = stored(df, storage)
    g.set_populations(df)
    assert np.array_equal(g.get_populations(), want)
    g.step(1)
    g.set_populations(df)  # odd level: the other AA layout
    assert np.array_equal(g.get_populations(), want)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_one_step_is_within_the_storage_roundoff(storage, collision):
    """From a state representable in the format, one GPU step equals the oracle's FP64
    step rounded once to the format, up to FP32 arithmetic: per population
    |g - o| <= u |o| + 5e-9 (u the unit roundoff), at an even and an odd level, on a
    lattice with ragged tiles."""
    shape = (37, 29, 23)
    g, o = pair(0, storage, collision, shape=shape)
    df = stored(W.random_df3(*shape, 2e-3, 21), storage)
    for _ in range(2):
        g.set_populations(df)
        o.set_df(df)
        g.step(1)
        o.step(1)
        got, ref = g.get_populations(), o.get_df()
        bound = UNIT[storage] * np.abs(ref) + 5e-9
        assert (np.abs(got - ref) <= bound).all(), np.max(np.abs(got - ref) - bound)
        df = got  # representable: the next round starts at the other parity


@pytest.mark.parametrize("storage,u_tol,x_tol", [("f16", 1.5e-3, 1e-5), ("bf16", 1.2e-2, 1e-4)])
def test_moving_tension_surface_16bit(storage, u_tol, x_tol):
    """A surface-tension ellipsoid relaxing with its vertices moving, 60 steps: velocity
    field and vertices near the oracle's.  Measured on a GB300: FP16 4.8e-4 of max |U| and
    3.0e-6 on the vertices, BF16 3.8e-3 and 3.3e-5 (eight times FP16's, the ratio of the
    formats' unit roundoff); the bounds are about three times those (FP32 storage stays
    below 1e-5)."""
    n = 24
    X, T = W.ellipsoid_surface((12.1, 11.8, 12.3), (6.0, 4.8, 4.0), 2, seed=10)
    g, o = pair(n, storage)
    g.set_surface(X, T, model=iilbm3d.TENSION, moves=True, gamma=3e-3)
    o.set_surface(X, T, model=o3.TENSION, moves=True, gamma=3e-3)
    g.step(60)
    o.step(60)
    uref = max(np.abs(o.markers()["U"]).max(), 1e-6)
    _, ug, vg, wg = g.get_macros()
    _, uo, vo, wo = o.current_macros()
    err = max(np.abs(ug - uo).max(), np.abs(vg - vo).max(), np.abs(wg - wo).max()) / uref
    xerr = np.abs(g.get_markers()["X"] - o.markers()["X"]).max()
    print(f"{storage}: velocity error {err:.3e} of max |U|, vertex error {xerr:.3e}")
    assert err < u_tol
    assert xerr < x_tol
    assert g.get_cut_link_count() > 0
