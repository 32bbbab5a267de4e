"""Rigid bodies carrying a directly forced interface (section 2.3, Eqs. 25-29): the CUDA
path against the FP64 oracle -- section 4.4's prescribed harmonic translation and a free
body with springs and dampers (section 4.5's oscillator), in both the IB and the II
forms.  The force iteration of a moving body rebuilds its band of nodes and its cut
links in every step; these cases move the body across many nodes so the rebuilt band is
exercised, and compare the body's state, the markers and every population."""

import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

from _pair import make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def body_pair(orc, mode, storage="f64", jump=1, dof=3, u0=0.01, D=10.0, n=32, rho_s=10.0,
              nx=64, ny=48, A=3.0, umax=0.02, spring=(0, 0, 0), damping=(0, 0, 0),
              iters=5, tol=0.0, centre=(23.7, 24.2)):
    """The same body on the CUDA library and on the oracle, a periodic box with a uniform
    stream u0 (MRT, tau 0.8)."""
    g, o = make_pair(orc, nx, ny, storage=storage, jump=jump)
    ux = np.full((ny, nx), u0)
    g.init_equilibrium(None, ux, None)
    o.init_equilibrium(None, ux, None)
    X = W.circle_markers(centre[0], centre[1], D / 2, n)
    dX = W.polygon_perimeter(X) / n
    UD = np.zeros((n, 2))
    g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=iters,
                    mdf_tol=tol, aux=UD)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=iters,
                    mdf_tol=tol, UD=UD)
    Vs = np.pi * D * D / 4
    m = rho_s * Vs
    g.iilbm_set_rigid_body(mode, dof=dof, amplitude=A, u_max=umax, mass=m,
                           inertia=m * D * D / 8, volume=Vs, spring=spring, damping=damping)
    o.set_body(mode, dof=dof, A=A, umax=umax, mass=m, inertia=m * D * D / 8, volume=Vs,
               spring=spring, damping=damping)
    return g, o, X


def state_of(g):
    b = g.iilbm_get_rigid_body()
    return np.array([b[k] for k in ("Xc", "Yc", "theta", "Ux", "Uy", "W", "Fx", "Fy", "T")])


def assert_same(g, o, tol_state, tol_df, tol_x=None):
    sg, so = state_of(g), np.asarray(o.body())
    scale = np.maximum(np.abs(so), 1e-6)
    err = np.abs(sg - so) / scale
    assert err.max() < tol_state, (sg, so)
    Xg, Xo = g.get_markers()["X"], o.markers()["X"]
    assert np.abs(Xg - Xo).max() < (tol_x if tol_x is not None else tol_state)
    dfg, dfo = g.get_populations(), o.get_df()
    assert np.abs(dfg - dfo).max() < tol_df * max(np.abs(dfo).max(), 1e-6)


@pytest.mark.parametrize("jump", [1, 0])
def test_prescribed_translation_fp64(orc, jump):
    """Section 4.4's harmonic translation in fluid at rest, A = 3, U_max = 0.02: centre,
    velocity, the reduced force (Eq. 25) and the flow it drives agree with the oracle
    step by step."""
    g, o, X = body_pair(orc, iilbm.BODY_PRESCRIBED_X, jump=jump, u0=0.0)
    for n in (1, 1, 5, 13, 40, 60):
        g.step(n)
        o.step(n)
        assert_same(g, o, 1e-9, 1e-10, tol_x=1e-11)
    s = state_of(g)
    assert abs(s[0] - (X.mean(0)[0] - 3.0 * np.sin(0.02 * 120 / 3.0))) < 1e-12
    assert abs(s[6]) > 1e-6  # the moving body pushes the fluid


@pytest.mark.parametrize("jump", [1, 0])
def test_free_body_fp64(orc, jump):
    """A free body (all three degrees of freedom) dragged by a uniform stream, density
    ratio 10: its trajectory under Eqs. 27-29 and the fluid around it follow the
    oracle's."""
    g, o, _ = body_pair(orc, iilbm.BODY_FREE, jump=jump, dof=7)
    for n in (1, 4, 25, 70):
        g.step(n)
        o.step(n)
        assert_same(g, o, 1e-8, 1e-10, tol_x=1e-11)
    assert state_of(g)[3] > 1e-5


def test_spring_mounted_body_in_a_channel_fp64(orc):
    """Section 4.5's oscillator: a cylinder free in y on a spring and damper in a channel
    with a parabolic inflow (II-LBM, density ratio 8 / pi, the paper's), 300 steps; the
    force iteration runs to a tolerance."""
    nx, ny, D, n = 160, 64, 16.0, 50
    s = W.mrt_rates(0.7)
    g = iilbm.Lattice(nx, ny, collision=iilbm.MRT, storage="f64", tau=0.7, s=s,
                      bc=iilbm.BC_CHANNEL, u_max=0.05, jump=1)
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.7, s=s, bc=orc.BC_CHANNEL, u_max=0.05,
                   jump=1)
    y = np.arange(ny) + 0.5
    u0 = np.repeat((4 * 0.05 * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)
    g.init_equilibrium(None, u0, None)
    o.init_equilibrium(None, u0, None)
    X = W.circle_markers(48.0, 33.1, D / 2, n)
    dX = W.polygon_perimeter(X) / n
    UD = np.zeros((n, 2))
    g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=60,
                    mdf_tol=1e-9, aux=UD)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=60,
                    mdf_tol=1e-9, UD=UD)
    Vs = np.pi * D * D / 4
    m = 8 / np.pi * Vs
    k = m * (2 * np.pi / 400.0) ** 2  # natural period 400 steps
    c = 2 * 0.05 * np.sqrt(k * m)
    g.iilbm_set_rigid_body(iilbm.BODY_FREE, dof=2, mass=m, inertia=m * D * D / 8, volume=Vs,
                           spring=(0, k, 0), damping=(0, c, 0))
    o.set_body(orc.BODY_FREE, dof=2, mass=m, inertia=m * D * D / 8, volume=Vs,
               spring=(0, k, 0), damping=(0, c, 0))
    for n in (1, 29, 70, 200):
        g.step(n)
        o.step(n)
        assert_same(g, o, 1e-7, 1e-9, tol_x=1e-10)
        assert g.iilbm_get_mdf_stats()[0] == o.mdf_stats()[0]
    sg = state_of(g)
    assert abs(sg[0] - X.mean(0)[0]) < 1e-12 and sg[2] == 0.0 and sg[3] == 0.0  # x, rotation held
    assert abs(sg[1] - X.mean(0)[1]) > 1e-6  # off-centre: the lift moves it in y


def test_long_travel_rebuilds_the_band_fp64(orc):
    """A prescribed translation of amplitude 12 nodes over 500 steps (the body crosses a
    dozen columns of the lattice and back), D = 20: the band rebuilt every step and the
    cut links found in the kernel agree with the oracle's set-up from the polygon."""
    g, o, _ = body_pair(orc, iilbm.BODY_PRESCRIBED_X, jump=1, u0=0.0, D=20.0, n=63, nx=96,
                        ny=64, A=12.0, umax=0.05, centre=(47.3, 31.9))
    for n in (100, 200, 200):
        g.step(n)
        o.step(n)
        assert_same(g, o, 1e-8, 1e-9, tol_x=1e-11)
    g.iilbm_synchronize()


def test_free_body_fp32(orc):
    """FP32 populations, FP64 markers and body: the trajectory within FP32 rounding of the
    FP64 oracle's."""
    g, o, _ = body_pair(orc, iilbm.BODY_FREE, storage="f32", jump=1, dof=7)
    g.step(100)
    o.step(100)
    sg, so = state_of(g), np.asarray(o.body())
    assert np.abs(sg[:2] - so[:2]).max() < 1e-5
    assert abs(sg[3] - so[3]) < 1e-4 * abs(so[3])


def test_graph_replay_equals_eager(orc):
    """The body's update is captured with the step: any step count replayed from graphs
    gives the eager result."""
    ga, _, _ = body_pair(orc, iilbm.BODY_FREE, jump=1, dof=7)
    gb, _, _ = body_pair(orc, iilbm.BODY_FREE, jump=1, dof=7)
    gb.set_option(iilbm.OPT_CUDA_GRAPH, 0)
    for n in (37, 1, 64, 3):
        ga.step(n)
        for _ in range(n):
            gb.step(1)
        assert np.abs(state_of(ga) - state_of(gb)).max() < 1e-12
        assert np.abs(ga.get_populations() - gb.get_populations()).max() < 1e-12


def test_rigid_body_argument_errors(orc):
    g, _ = make_pair(orc, 48, 48)
    with pytest.raises(iilbm.IilbmError) as e:  # no interface
        g.iilbm_set_rigid_body(iilbm.BODY_FREE, dof=7, mass=1.0, inertia=1.0)
    assert e.value.code == iilbm.ERR_INVALID_ARG
    X = W.circle_markers(23.7, 24.2, 5.0, 32)
    g.set_interface(X, model=iilbm.SPRING, moves=True, stiffness=0.05, dX=1.0)
    with pytest.raises(iilbm.IilbmError):  # not a directly forced interface
        g.iilbm_set_rigid_body(iilbm.BODY_FREE, dof=7, mass=1.0, inertia=1.0)
    g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=1.0, eta=2.0, mdf_iters=3,
                    aux=np.zeros((32, 2)))
    for kw in (dict(mode=0), dict(mode=iilbm.BODY_FREE, mass=0.0, inertia=1.0, dof=1),
               dict(mode=iilbm.BODY_FREE, mass=1.0, inertia=1.0, dof=8),
               dict(mode=iilbm.BODY_PRESCRIBED_X, amplitude=0.0, u_max=0.01)):
        with pytest.raises(iilbm.IilbmError):
            g.iilbm_set_rigid_body(**kw)
    with pytest.raises(iilbm.IilbmError):  # no body yet
        g.iilbm_get_rigid_body()
    g.iilbm_set_rigid_body(iilbm.BODY_FREE, dof=7, mass=800.0, inertia=5000.0, volume=78.5)
    g.step(3)
    assert np.all(np.isfinite(state_of(g)))
    g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=1.0, eta=2.0, mdf_iters=3,
                    aux=np.zeros((32, 2)))
    with pytest.raises(iilbm.IilbmError):  # a new interface drops the body
        g.iilbm_get_rigid_body()
