"""Execution variants of the CUDA path give the same results: the vectorised and the
one-node-per-thread stream-collide (bitwise), CUDA-graph replay and eager launches,
the overlapped and the serial interface phase; kernel timing works in both modes."""
import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

from _pair import make_pair, set_membrane, vel_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def _lat(nx, ny, storage, collision, bc, **kw):
    return iilbm.Lattice(nx, ny, collision=iilbm.SRT if collision == "srt" else iilbm.MRT,
                         storage=storage, tau=0.7, s=W.mrt_rates(0.7),
                         bc=iilbm.BC_PERIODIC if bc == "periodic" else iilbm.BC_WALLS_Y,
                         body=(1e-5, -3e-6), **kw)


ULP = {"f32": 2.0 ** -23, "f64": 2.0 ** -52, "f16": 2.0 ** -10, "bf16": 2.0 ** -7}


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("bc", ["periodic", "walls"])
@pytest.mark.parametrize("shape", [(256, 24), (100, 13), (36, 9), (128, 40)])
def test_vector_kernel_matches_scalar(storage, bc, shape):
    """Same populations from both kernels, seven steps of random data, up to 64 ulps of
    the storage type relative to the field's scale (the compiler contracts multiply-
    adds differently in the two kernels and the differences compound); a wrong
    neighbour from a shuffle or an edge lane would differ by O(1)."""
    nx, ny = shape
    df = W.random_df(nx, ny, 2e-3, nx + ny)
    out = []
    for vec in (0, 1):
        g = _lat(nx, ny, storage, "mrt", bc)
        g.set_option(iilbm.OPT_VECTOR_KERNEL, vec)
        g.set_populations(df)
        res = []
        for n in (1, 1, 2, 3):  # both parities, several times
            g.step(n)
            res.append(g.get_populations())
        out.append(res)
    for a, b in zip(*out):
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= 64 * ULP[storage] * scale


@pytest.mark.parametrize("collision", ["srt", "mrt"])
@pytest.mark.parametrize("bc", ["periodic", "walls", "channel"])
@pytest.mark.parametrize("body", [False, True])
@pytest.mark.parametrize("shape", [(264, 17), (520, 40), (392, 33), (1024, 72)])
def test_tma_kernel_matches_vector(collision, bc, body, shape):
    """FP32: the TMA stream-collide of the interior tiles (with the register path on the
    rest; every step, and odd steps only) against the register path everywhere, seven
    steps of random data at both parities, in the periodic box, between walls and in the
    channel (inflow, outflow, ghost columns), on lattices with one interior tile,
    several, and a ragged last tile column: equal up to the compiler's multiply-add
    contraction (64 ulps of the field's scale); a wrong box offset, shift or edge store
    would differ by O(1)."""
    nx, ny = shape
    df = W.random_df(nx, ny, 2e-3, 3 * nx + ny)
    out = []
    bcs = {"periodic": iilbm.BC_PERIODIC, "walls": iilbm.BC_WALLS_Y, "channel": iilbm.BC_CHANNEL}
    for tma in (0, 1, 2):
        g = iilbm.Lattice(nx, ny, collision=iilbm.SRT if collision == "srt" else iilbm.MRT,
                          storage="f32", tau=0.7, s=W.mrt_rates(0.7), bc=bcs[bc],
                          u_max=0.03 if bc == "channel" else 0.0,
                          body=(1e-5, -3e-6) if body else (0.0, 0.0))
        g.set_option(iilbm.OPT_TMA_KERNEL, tma)
        g.set_populations(df)
        res = []
        for n in (1, 1, 2, 3):
            g.step(n)
            res.append(g.get_populations())
        g.synchronize()
        out.append(res)
    for run in out[1:]:  # every step, odd steps only
        for a, b in zip(out[0], run):
            assert np.abs(a - b).max() <= 64 * ULP["f32"] * np.abs(a).max()


def test_tma_kernel_with_a_membrane_matches_the_oracle(orc):
    """A moving FP32 membrane on a 512 x 320 lattice (its flagged tiles inside the TMA
    kernel's interior rectangle, left to the forced kernel): 40 steps with and without
    the TMA kernel, both within 1e-5 of the oracle's velocity, and the launch count per
    step one higher with it (interior and edge tiles)."""
    w = W.ellipse_scaled(320, "f32")
    X = w["X"] + np.array([96.0, 0.0])
    for tma in (1, 0):
        g, o = make_pair(orc, 512, 320, collision="mrt", storage="f32", tau=w["tau"])
        g.set_option(iilbm.OPT_TMA_KERNEL, tma)
        set_membrane(orc, g, o, X, "spring", w["kappa"], w["dX"])
        g.step(2)
        g.iilbm_set_timing(True)
        g.step(38)
        ms, n, k = g.iilbm_get_timing()
        assert n == 38 and k == 38 * (4 if tma else 3) and ms > 0
        o.step(40)
        umax = np.abs(o.markers()["U"]).max()
        assert vel_error(g, o, max(umax, 1e-6)) < 1e-5
        assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-7


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_graph_and_overlap_match_eager(orc, storage):
    """70 steps (two 32-step graph replays plus eager steps) of a moving membrane, in
    every combination of graph / overlap, agree with each other and with the oracle."""
    w = W.ellipse_scaled(256, storage)
    ref = None
    for graph, overlap in ((0, 0), (1, 0), (0, 1), (1, 1)):
        g, o = make_pair(orc, 256, 256, collision="mrt", storage=storage, tau=w["tau"])
        g.set_option(iilbm.OPT_CUDA_GRAPH, graph)
        g.set_option(iilbm.OPT_OVERLAP, overlap)
        set_membrane(orc, g, o, w["X"], "spring", w["kappa"], w["dX"])
        g.step(3)
        g.step(67)
        d = g.get_populations()
        X = g.get_markers()["X"]
        if ref is None:
            o.step(70)
            umax = np.abs(o.markers()["U"]).max()
            tol = 1e-12 if storage == "f64" else 1e-5
            assert vel_error(g, o, max(umax, 1e-6)) < tol
            assert np.abs(X - o.markers()["X"]).max() < (1e-12 if storage == "f64" else 1e-7)
            ref = (d, X)
        else:
            scale = np.abs(ref[0]).max()
            tol = 1e-13 if storage == "f64" else 1e-5
            assert np.abs(d - ref[0]).max() < tol * scale
            assert np.abs(X - ref[1]).max() < (1e-13 if storage == "f64" else 1e-7)


def test_timing_counts_launches_in_graph_and_eager_modes():
    w = W.ellipse_scaled(256, "f32")
    g = iilbm.Lattice(256, 256, collision=iilbm.MRT, storage="f32", tau=w["tau"])
    g.set_interface(w["X"], model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
    g.step(2)
    g.iilbm_set_timing(True)
    g.step(64 + 5)
    ms, n, k = g.iilbm_get_timing()
    # per step: lean and forced stream-collide, interpolation fused with the next
    # level's interface phase
    assert n == 69 and k == 69 * 3 and 0 < ms < 69 * 10.0
    g.iilbm_set_option(iilbm.OPT_CUDA_GRAPH, 0)
    g.iilbm_set_timing(True)
    g.step(7)
    ms, n, k = g.iilbm_get_timing()
    assert n == 7 and ms > 0


def test_forced_blocks_option_leaves_results_unchanged():
    """The forced stream-collide's grid only changes which block takes which flagged
    tile: populations agree with the default grid's to FP32 rounding (the interface
    phase accumulates with atomics, so two runs agree to rounding, not bitwise)."""
    w = W.ellipse_scaled(256, "f32")
    gs = []
    for blocks in (0, 3):
        g = iilbm.Lattice(256, 256, collision=iilbm.MRT, storage="f32", tau=w["tau"],
                          s=W.mrt_rates(w["tau"]))
        g.set_option(iilbm.OPT_FORCED_BLOCKS, blocks)
        g.set_interface(w["X"], model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
        g.step(40)
        gs.append(g)
    a, b = gs[0].get_populations(), gs[1].get_populations()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max() and np.abs(a).max() > 0
    with pytest.raises(iilbm.IilbmError):
        gs[0].set_option(iilbm.OPT_FORCED_BLOCKS, -1)


@pytest.mark.parametrize("n", [3, 5, 10, 11, 17])
def test_fused_interface_phase_on_short_polygons(orc, n):
    """The pipelined step interpolates a halo of markers around each block of 8 segments
    (indices wrapping around the polygon); with 3 to 17 markers the halo wraps onto the
    block's own markers.  Overlapped (fused) and serial steps agree, and both follow the
    FP64 oracle."""
    X = W.circle_markers(20.3, 19.6, 2.0 + 0.4 * n, n)
    dX = W.polygon_perimeter(X) / n
    out = []
    for overlap in (1, 0):
        g, o = make_pair(orc, 40, 40, collision="mrt", storage="f64", tau=0.8)
        g.set_option(iilbm.OPT_OVERLAP, overlap)
        # a stretched polygon relaxing: the markers move every step
        set_membrane(orc, g, o, X * 1.1 - 2.0, "spring", 0.02, dX)
        g.step(45)
        o.step(45)
        umax = max(np.abs(o.markers()["U"]).max(), 1e-6)
        assert np.abs(o.markers()["U"]).max() > 1e-6
        assert vel_error(g, o, umax) < 1e-12
        assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-12
        out.append(g.get_markers())
    for k in ("X", "U", "G"):
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-13 * max(np.abs(out[1][k]).max(), 1e-9)


@pytest.mark.parametrize("bc", ["walls", "channel"])
def test_pipelined_membrane_near_walls(orc, bc):
    """The fused interpolation / interface kernel is compiled per boundary kind: a moving
    membrane about 4 nodes from a wall (and, in a channel, from the inflow end),
    overlapped and serial, against the FP64 oracle step by step."""
    nx, ny, tau = 48, 40, 0.8
    s = W.mrt_rates(tau)
    n = 26
    X = W.circle_markers(12.0, 11.0, 7.0, n) * np.array([1.08, 1.0]) - np.array([1.0, 0.0])
    assert X[:, 1].min() > 3.0 and X[:, 0].min() > 3.0
    dX = W.polygon_perimeter(X) / n * 0.9  # stretched: the membrane moves every step
    kw = dict(collision=iilbm.MRT, storage="f64", tau=tau, s=s)
    if bc == "walls":
        kw_g, kw_o = dict(bc=iilbm.BC_WALLS_Y), dict(bc=orc.BC_WALLS_Y)
    else:
        kw_g, kw_o = dict(bc=iilbm.BC_CHANNEL, u_max=0.02), dict(bc=orc.BC_CHANNEL, u_max=0.02)
    outs = []
    for overlap in (1, 0):
        g = iilbm.Lattice(nx, ny, **kw, **kw_g)
        o = orc.Oracle(nx, ny, collision=orc.MRT, tau=tau, s=s, **kw_o)
        g.set_option(iilbm.OPT_OVERLAP, overlap)
        set_membrane(orc, g, o, X, "spring", 0.03, dX)
        for _ in range(3):
            g.step(13)
            o.step(13)
            assert np.abs(g.get_populations() - o.get_df()).max() < 1e-14
            assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-12
            assert g.iilbm_get_cut_link_count() == o.cut_link_count()
        assert np.abs(o.markers()["U"]).max() > 1e-5
        outs.append(g.get_markers()["X"])
    assert np.abs(outs[0] - outs[1]).max() < 1e-13


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_graph_replay_for_any_length_and_parity(storage):
    """Calls of every length and starting parity replay graphs (32/16/8/4/2/1 steps from
    an even level, one step from an odd one) and give the state eager launches give:
    FP64 to 1e-13 and FP32 to 1e-6 of the field's scale (the spreading's atomics add in
    run-dependent order), markers likewise."""
    w = W.ellipse_scaled(256, storage)
    seq = (1, 2, 3, 5, 20, 33, 7, 64, 1)
    res = []
    for graph in (0, 1):
        g = iilbm.Lattice(256, 256, collision=iilbm.MRT, storage=storage, tau=w["tau"],
                          s=W.mrt_rates(w["tau"]))
        g.set_option(iilbm.OPT_CUDA_GRAPH, graph)
        g.set_interface(w["X"], model=iilbm.SPRING, stiffness=w["kappa"], dX=w["dX"])
        out = []
        for n in seq:
            g.step(n)
            out.append((g.get_populations(), g.get_markers()["X"]))
        res.append(out)
    # FP64: the atomics' rounding differences grow over the 136 steps to the conditioning
    # floor of a long membrane run (~1e-12 of the field)
    tol = 1e-12 if storage == "f64" else 1e-6
    for (a, Xa), (b, Xb) in zip(*res):
        d = np.abs(a - b).max() / np.abs(a).max()
        assert d <= tol and np.abs(a).max() > 0, f"graph vs eager: {d:.3e}"
        assert np.abs(Xa - Xb).max() <= (1e-12 if storage == "f64" else 1e-6)


def test_graph_replay_of_direct_forcing(orc):
    """A directly forced cylinder in a channel replays from graphs too (every captured
    step begins with its force iteration and interface phase), including after a
    read-out that ran that phase early (the next step then runs eagerly): graph and
    eager runs agree with each other and with the FP64 oracle."""
    nx, ny, n = 160, 64, 50
    s = W.mrt_rates(0.7)
    X = W.circle_markers(48.0, 32.5, 8.0, n)
    dX = W.polygon_perimeter(X) / n
    y = np.arange(ny) + 0.5
    u0 = np.repeat((4 * 0.05 * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.7, s=s, bc=orc.BC_CHANNEL, u_max=0.05)
    o.init_equilibrium(None, u0, None)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                    UD=np.zeros((n, 2)))
    seq = (3, 1, "read", 20, 2, 5)
    outs = []
    for graph in (1, 0):
        g = iilbm.Lattice(nx, ny, collision=iilbm.MRT, storage="f64", tau=0.7, s=s,
                          bc=iilbm.BC_CHANNEL, u_max=0.05)
        g.set_option(iilbm.OPT_CUDA_GRAPH, graph)
        g.init_equilibrium(None, u0, None)
        g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                        aux=np.zeros((n, 2)))
        for a in seq:
            if a == "read":
                g.get_macros()
            else:
                g.step(a)
        outs.append((g.get_populations(), g.get_markers()["G"]))
    o.step(sum(a for a in seq if a != "read"))
    assert np.abs(outs[0][0] - outs[1][0]).max() < 1e-14
    assert np.abs(outs[0][1] - outs[1][1]).max() < 1e-13
    assert np.abs(outs[0][0] - o.get_df()).max() < 1e-14
    assert np.abs(outs[0][1] - o.markers()["G"]).max() < 1e-12


def test_same_size_interface_replacement(orc):
    """A new polygon with the same marker count and parameters reuses the marker buffers
    and the captured graphs: the run still follows the FP64 oracle given the same
    replacement."""
    g, o = make_pair(orc, 96, 96, collision="mrt", storage="f64", tau=0.7)
    X = W.circle_markers(47.6, 48.3, 15.0, 96)
    dX = W.polygon_perimeter(X) / 96 * 0.9
    set_membrane(orc, g, o, X, "spring", 0.02, dX)
    g.step(10)
    o.step(10)
    X2 = X * np.array([1.05, 0.96]) + np.array([-2.13, 1.71])
    set_membrane(orc, g, o, X2, "spring", 0.02, dX)
    g.step(15)
    o.step(15)
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-14
    assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-12


@pytest.mark.parametrize("graph", [1, 0])
def test_nonfinite_population_is_reported(graph):
    """A NaN planted from the host in one population (iilbm_set_populations) is caught by
    the stream-collide's finiteness check and latched: the next synchronising call
    returns IILBM_ERR_NONFINITE.  No interface, so no index depends on the NaN."""
    g = iilbm.Lattice(64, 32, collision=iilbm.MRT, storage="f32", tau=0.8,
                      s=W.mrt_rates(0.8))
    g.set_option(iilbm.OPT_CUDA_GRAPH, graph)
    df = W.random_df(64, 32, 1e-4, 1)
    g.set_populations(df)
    g.step(3)
    g.synchronize()  # a finite state passes
    df[4, 10, 17] = np.nan
    g.set_populations(df)
    g.step(3)
    with pytest.raises(iilbm.IilbmError) as e:
        g.synchronize()
    assert e.value.code == iilbm.ERR_NONFINITE
