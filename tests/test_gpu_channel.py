"""Channel boundaries (parabolic inflow by non-equilibrium extrapolation, zero-gradient
outflow, halfway bounce-back walls) and direct forcing of a fixed cylinder with repeated
correction (Eq. 18), CUDA path against the FP64 oracle."""

import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

from _pair import assert_jump_fields_agree, oracle_jump_field, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def channel_pair(orc, nx, ny, storage="f64", tau=0.8, u_max=0.05, jump=1):
    s = W.mrt_rates(tau)
    g = iilbm.Lattice(nx, ny, collision=iilbm.MRT, storage=storage, tau=tau, s=s,
                      bc=iilbm.BC_CHANNEL, u_max=u_max, jump=jump)
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=tau, s=s, bc=orc.BC_CHANNEL, u_max=u_max,
                   jump=jump)
    return g, o


@pytest.mark.parametrize("vec", [1, 0])
@pytest.mark.parametrize("shape", [(96, 32), (70, 21)])
def test_empty_channel_fp64(orc, vec, shape):
    nx, ny = shape
    g, o = channel_pair(orc, nx, ny)
    g.set_option(iilbm.OPT_VECTOR_KERNEL, vec)
    df = W.random_df(nx, ny, 1e-4, 3)
    g.set_populations(df)
    o.set_df(df)
    for n in (1, 1, 7, 40):
        g.step(n)
        o.step(n)
        assert np.abs(g.get_populations() - o.get_df()).max() < 1e-15
    _, ug, vg = g.get_macros()
    _, uo, vo = o.current_macros()
    assert max(rel_err(ug, uo, 0.05), rel_err(vg, vo, 0.05)) < 1e-12


def parabola(nx, ny, u_max=0.05):
    y = np.arange(ny) + 0.5
    return np.repeat((4 * u_max * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)


def cylinder_case(orc, storage, iters, tol, nx=160, ny=64, D=16.0, n=50, steps=60):
    """Channel started from the parabolic inflow profile everywhere, so the cylinder sits
    in a developed stream from the first step."""
    g, o = channel_pair(orc, nx, ny, storage=storage, tau=0.7)
    u0 = parabola(nx, ny)
    g.init_equilibrium(None, u0, None)
    o.init_equilibrium(None, u0, None)
    X = W.circle_markers(48.0, 32.5, D / 2, n)
    dX = W.polygon_perimeter(X) / n
    UD = np.zeros((n, 2))
    g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=iters,
                    mdf_tol=tol, aux=UD)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=iters,
                    mdf_tol=tol, UD=UD)
    g.step(steps)
    o.step(steps)
    return g, o


def test_cylinder_direct_forcing_fp64(orc):
    """Five force updates per step (the channel cylinder setting), 60 steps: populations,
    Lagrangian force and interpolated velocity match the oracle."""
    g, o = cylinder_case(orc, "f64", 5, 0.0)
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-14
    mg = g.get_markers()  # both: the force of the last step's state
    mo = o.markers()
    assert np.abs(mg["G"] - mo["G"]).max() < 1e-13
    it_g, res_g = g.iilbm_get_mdf_stats()
    it_o, res_o = o.mdf_stats()
    assert it_g == it_o == 5 and abs(res_g - res_o) < 1e-14
    F = g.iilbm_get_body_force()
    Fo = -mo["G"].sum(0) * W.polygon_perimeter(mo["X"]) / 50
    assert abs(F[0] - Fo[0]) < 1e-12 and F[0] > 0  # drag along the stream


def test_cylinder_iteration_to_tolerance_fp64(orc):
    """Stopping on the residual: same pass count and residual as the oracle.  Markers
    about 1.5 lattice units apart: at a spacing near 1 the spread-interpolate operator
    has near-zero eigenvalues and the plain iteration stalls above the tolerance."""
    g, o = cylinder_case(orc, "f64", 200, 2e-4, steps=20, n=34)
    it_g, res_g = g.iilbm_get_mdf_stats()
    it_o, res_o = o.mdf_stats()
    assert it_g == it_o and res_g < 2e-4 and abs(res_g - res_o) < 1e-14
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-14


def test_cylinder_direct_forcing_fp32(orc):
    g, o = cylinder_case(orc, "f32", 5, 0.0, steps=100)
    _, ug, vg = g.get_macros()
    _, uo, vo = o.current_macros()
    assert max(rel_err(ug, uo, 0.05), rel_err(vg, vo, 0.05)) < 1e-5


def test_warm_start_changes_iterations_not_answer(orc):
    """A warm start near the converged force needs fewer passes to the same tolerance."""
    g, o = cylinder_case(orc, "f64", 300, 1e-5, steps=30, n=34)
    it0, res0 = g.iilbm_get_mdf_stats()
    assert it0 > 3 and res0 < 1e-5
    G = g.get_markers()["G"]
    g.iilbm_set_warm_start(G)
    g.step(1)
    it1, res1 = g.iilbm_get_mdf_stats()
    assert res1 < 1e-5 and it1 < it0


def test_channel_cylinder_full_size_fp32(orc):
    """The 1024 x 256 channel with the D = 40 cylinder (126 markers), Re = 100 (tau 0.56
    from Re with u_max = 0.05), five force updates per step with the normal part
    through the jump, started from the parabolic profile everywhere (so the body
    carries a force from the first step): 500 steps against the oracle (its OpenMP
    build), the velocity within 1e-5 and the cut links exactly."""
    w = W.cylinder_channel(100.0)
    s = W.mrt_rates(w["tau"])
    try:
        orc.lib(parallel=True)
        par, steps = True, 500
    except RuntimeError:  # no OpenMP runtime: a shorter run on one core
        par, steps = False, 60
    g = iilbm.Lattice(w["nx"], w["ny"], collision=iilbm.MRT, storage="f32", tau=w["tau"], s=s,
                      bc=iilbm.BC_CHANNEL, u_max=w["u_max"])
    o = orc.Oracle(w["nx"], w["ny"], parallel=par, collision=orc.MRT, tau=w["tau"], s=s,
                   bc=orc.BC_CHANNEL, u_max=w["u_max"])
    u0 = parabola(w["nx"], w["ny"])
    g.init_equilibrium(None, u0, None)
    o.init_equilibrium(None, u0, None)
    n = len(w["X"])
    g.set_interface(w["X"], model=iilbm.DIRECT, moves=False, dX=w["dX"], eta=2.0,
                    mdf_iters=5, aux=np.zeros((n, 2)))
    o.set_interface(w["X"], model=orc.DIRECT, moves=False, dX=w["dX"], eta=2.0, mdf_iters=5,
                    UD=np.zeros((n, 2)))
    for done in range(0, steps, 100):
        k = min(100, steps - done)
        g.step(k)
        o.step(k)
        _, ug, vg = g.get_macros()
        _, uo, vo = o.current_macros()
        err = max(rel_err(ug, uo, 0.05), rel_err(vg, vo, 0.05))
        assert err < 1e-5, f"step {done + k}: rel vel err {err:.3e}"
    assert g.iilbm_get_cut_link_count() == o.cut_link_count() > 0
    # the cut links of the fixed body exactly; the jump values follow the FP32 force
    Jo, _ = oracle_jump_field(orc, o)
    assert_jump_fields_agree(g.iilbm_get_jump(), Jo, 1e-4)
    Fg, Fo = g.iilbm_get_body_force(), -o.markers()["G"].sum(0) * w["dX"]
    assert abs(Fg[0] - Fo[0]) < 1e-4 * abs(Fo[0]) and Fo[0] > 0
    print(f"channel Re 100 f32 {steps} steps: rel vel err {err:.3e}, C_D "
          f"{2 * Fo[0] / (w['u_max'] ** 2 * 40.0):.4f}")


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_cylinder_of_the_papers_size(orc, storage):
    """A D = 80 cylinder (the finest of section 4.3's meshes, 251 markers one lattice
    unit apart) in a 480 x 200 channel: the force iteration's band of nodes (not the
    body's 85 x 85 bounding box) fits one CTA's shared memory.  30 steps against the
    oracle: FP64 to 1e-12, FP32 to 1e-5."""
    nx, ny, D, n = 480, 200, 80.0, 251
    tau = 0.5 + 3.0 * 0.05 * D / 100.0
    s = W.mrt_rates(tau)
    X = W.circle_markers(160.0, 100.5, D / 2, n)
    dX = W.polygon_perimeter(X) / n
    g = iilbm.Lattice(nx, ny, collision=iilbm.MRT, storage=storage, tau=tau, s=s,
                      bc=iilbm.BC_CHANNEL, u_max=0.05)
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=tau, s=s, bc=orc.BC_CHANNEL, u_max=0.05)
    u0 = parabola(nx, ny)
    g.init_equilibrium(None, u0, None)
    o.init_equilibrium(None, u0, None)
    g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                    aux=np.zeros((n, 2)))
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                    UD=np.zeros((n, 2)))
    g.step(30)
    o.step(30)
    _, ug, vg = g.get_macros()
    _, uo, vo = o.current_macros()
    tol = 1e-12 if storage == "f64" else 1e-5
    assert max(rel_err(ug, uo, 0.05), rel_err(vg, vo, 0.05)) < tol
    assert np.abs(o.markers()["G"]).max() > 1e-4  # the body carries a force
    Jo, _ = oracle_jump_field(orc, o)
    assert_jump_fields_agree(g.iilbm_get_jump(), Jo, 1e-10 if storage == "f64" else 1e-4)


def test_unforced_velocity_and_previous_force_start_fp64(orc):
    """U* (interpolation of u* before the first update) and the iteration started from
    the previous step's force: pass counts, force and populations match the oracle
    step by step, and once the impulsive start's transient has passed (60 steps; during
    the first dozen steps the force changes too fast for the previous one to help) the
    previous-force start needs fewer passes in total than the plain iteration run beside
    it on the same channel."""
    g, o = cylinder_case(orc, "f64", 300, 1e-5, steps=60, n=34)
    p, _ = cylinder_case(orc, "f64", 300, 1e-5, steps=60, n=34)  # plain, beside it
    g.iilbm_set_warm_start_mode(iilbm.WS_PREVIOUS)
    o.set_ws_previous(True)
    passes_prev, passes_plain = 0, 0
    for _ in range(8):
        g.step(1)
        o.step(1)
        p.step(1)
        it_g, res_g = g.iilbm_get_mdf_stats()
        it_o, res_o = o.mdf_stats()
        assert it_g == it_o and abs(res_g - res_o) < 1e-14 and res_g < 1e-5
        assert np.abs(g.iilbm_get_unforced_velocity() - o.unforced_velocity()).max() < 1e-14
        assert np.abs(g.get_markers()["G"] - o.markers()["G"]).max() < 1e-12
        passes_prev += it_g
        passes_plain += p.iilbm_get_mdf_stats()[0]
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-14
    assert passes_prev < passes_plain


def test_unforced_velocity_fp32(orc):
    g, o = cylinder_case(orc, "f32", 5, 0.0, steps=20)
    U = g.iilbm_get_unforced_velocity()
    Uo = o.unforced_velocity()
    assert np.abs(U - Uo).max() <= 1e-5 * max(np.abs(Uo).max(), 0.05)
