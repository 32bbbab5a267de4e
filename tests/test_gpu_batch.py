"""Batched executor: many independent lattices of uneven size advanced together, one
launch per phase per step, replayed from CUDA graphs.  Each batched lattice must follow
the same trajectory as the same lattice stepped on its own, and the FP64 oracle."""
import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

from _pair import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


# eight membranes of the batched sweep (sizes 64..512, several not a multiple of the
# 128-wide tile), plus one lattice without an interface
SIMS = W.batched_membranes(count=8, seed=3)


def membrane(sim, storage="f32"):
    g = iilbm.Lattice(sim["nx"], sim["ny"], collision=iilbm.MRT, storage=storage,
                      tau=sim["tau"], s=W.mrt_rates(sim["tau"]))
    g.set_interface(sim["X"], model=iilbm.SPRING, stiffness=sim["kappa"], dX=sim["dX"])
    return g


def lattices(storage="f32", empty=True):
    gs = [membrane(s, storage) for s in SIMS]
    if empty:
        g = iilbm.Lattice(96, 64, collision=iilbm.MRT, storage=storage, tau=0.7,
                          s=W.mrt_rates(0.7))
        g.set_populations(W.random_df(96, 64, 1e-4, 11))
        gs.append(g)
    return gs


def max_vel_diff(a, b):
    """Largest velocity difference of two lattices relative to the larger speed."""
    _, ua, va = a.get_macros()
    _, ub, vb = b.get_macros()
    ref = max(np.abs(ub).max(), np.abs(vb).max(), 1e-6)
    return max(np.abs(ua - ub).max(), np.abs(va - vb).max()) / ref


def markers_diff(a, b):
    return np.abs(a.get_markers()["X"] - b.get_markers()["X"]).max()


def test_batch_kinds_are_distinct():
    assert len({s["nx"] for s in SIMS}) >= 4
    assert any(s["nx"] % 128 for s in SIMS)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 1e-3)])
def test_batch_matches_solo(storage, tol):
    """70 steps (two 32-step graph replays and 6 eager steps) of the batch against each
    lattice stepped alone."""
    solo = lattices(storage)
    batched = lattices(storage)
    for g in solo:
        g.step(70)
    with iilbm.Batch(batched) as B:
        B.step(70)
        B.synchronize()
        for a, b in zip(batched, solo):
            assert max_vel_diff(a, b) < tol
        for a, b in zip(batched[:-1], solo[:-1]):
            # positions integrate 70 interpolated velocities, each within the FP32 bound
            umax = max(np.abs(b.get_markers()["U"]).max(), 1e-6)
            assert markers_diff(a, b) <= 70 * tol * umax


@pytest.mark.parametrize("variant", range(len(iilbm.BATCH_VARIANTS)))
def test_every_variant_matches_solo(variant):
    solo = lattices()
    batched = lattices()
    for g in solo:
        g.step(40)
    with iilbm.Batch(batched) as B:
        B.iilbm_batch_set_variant(variant)
        B.step(40)
        for a, b in zip(batched, solo):
            assert max_vel_diff(a, b) < 1e-5


def test_batch_against_oracle(orc):
    """A 96 x 96 and a 128 x 128 membrane batched together, 40 steps, against the FP64
    oracle at the FP32 tolerance."""
    sims = [s for s in W.batched_membranes(count=64, seed=5) if s["nx"] in (96, 128)][:2]
    assert len(sims) == 2
    gs = [membrane(s) for s in sims]
    os_ = []
    for s in sims:
        o = orc.Oracle(s["nx"], s["ny"], collision=orc.MRT, tau=s["tau"], s=W.mrt_rates(s["tau"]))
        o.set_interface(s["X"], model=orc.SPRING, kappa=s["kappa"], dX=s["dX"])
        o.step(40)
        os_.append(o)
    with iilbm.Batch(gs) as B:
        B.step(40)
        for g, o in zip(gs, os_):
            _, ug, vg = g.get_macros()
            _, uo, vo = o.current_macros()
            uref = max(np.abs(uo).max(), np.abs(vo).max(), 1e-6)
            assert max(rel_err(ug, uo, uref), rel_err(vg, vo, uref)) < 1e-5
            mo = o.markers()
            umax = max(np.abs(mo["U"]).max(), 1e-6)
            assert np.abs(g.get_markers()["X"] - mo["X"]).max() <= 40 * 1e-5 * umax


def test_batch_from_odd_state_and_readout_midway():
    """Lattices one step in (odd state) enter the batch; a read-out of one lattice midway
    does not disturb the others."""
    solo = lattices()
    batched = lattices()
    for g in solo:
        g.step(1)
        g.step(69)
    for g in batched:
        g.step(1)
    with iilbm.Batch(batched) as B:
        B.step(36)
        batched[2].get_macros()
        batched[5].iilbm_get_cut_link_count()
        B.step(33)
        for a, b in zip(batched, solo):
            assert max_vel_diff(a, b) < 1e-5
    # after the batch is gone the lattices step on their own again
    for g in batched + solo:
        g.step(3)
    for a, b in zip(batched, solo):
        assert max_vel_diff(a, b) < 1e-5


def test_autotune_picks_a_variant_and_keeps_the_trajectory():
    solo = lattices(empty=False)[:4]
    batched = lattices(empty=False)[:4]
    with iilbm.Batch(batched) as B:
        v, us = B.autotune(32)
        assert 0 <= v < len(iilbm.BATCH_VARIANTS) and us > 0
        # each variant: 32 warm-up steps + 32 timed steps from step 0 (even throughout)
        B.step(6)
    for g in solo:
        g.step(len(iilbm.BATCH_VARIANTS) * 64 + 6)
    for a, b in zip(batched, solo):
        assert max_vel_diff(a, b) < 1e-4


def test_batch_timing_counts():
    gs = lattices(empty=False)[:3]
    with iilbm.Batch(gs) as B:
        B.iilbm_batch_set_timing(True)
        B.step(5)
        ms, n, k = B.iilbm_batch_get_timing()
        # per step: lean and forced stream-collide, interpolation, marker and segment
        # passes of the next interface phase
        assert n == 5 and k == 5 * 5 and ms > 0


def test_batch_refuses_invalid_sets():
    a = membrane(SIMS[0])
    b = membrane(SIMS[1], "f16")
    c = iilbm.Lattice(64, 64, storage="f64", tau=0.8)
    d = iilbm.Lattice(70, 64, storage="f32", tau=0.8)
    e = iilbm.Lattice(64, 64, storage="f32", tau=0.8, collision=iilbm.SRT)
    for bad in ([a, a], [a, b], [c], [a, d], [a, e]):
        with pytest.raises(iilbm.IilbmError) as err:
            iilbm.Batch(bad)
        assert err.value.code == iilbm.ERR_INVALID_ARG
    f = membrane(SIMS[2])
    f.step(1)
    with pytest.raises(iilbm.IilbmError):
        iilbm.Batch([a, f])  # different parity
    with iilbm.Batch([a]) as B:
        with pytest.raises(iilbm.IilbmError):
            iilbm.Batch([a])  # already batched
        for call in (lambda: a.step(1), lambda: a.set_interface(SIMS[0]["X"]),
                     lambda: a.init_equilibrium(), lambda: a.set_option(iilbm.OPT_OVERLAP, 0)):
            with pytest.raises(iilbm.IilbmError) as err:
                call()
            assert err.value.code == iilbm.ERR_INVALID_ARG
        B.step(2)
    a.step(1)


# ------------------------------------------------------------ channels, direct forcing
def parabola(nx, ny, u_max=0.05):
    y = np.arange(ny) + 0.5
    return np.repeat((4 * u_max * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)


CHANNELS = [dict(nx=256, ny=64, D=12.0, n=38, cx=64.0, cy=32.3, tau=0.7),
            dict(nx=320, ny=96, D=16.0, n=50, cx=80.0, cy=47.8, tau=0.62)]


def channel(c, lib, storage="f32"):
    s = W.mrt_rates(c["tau"])
    X = W.circle_markers(c["cx"], c["cy"], c["D"] / 2, c["n"])
    dX = W.polygon_perimeter(X) / c["n"]
    if lib is iilbm:
        g = iilbm.Lattice(c["nx"], c["ny"], collision=iilbm.MRT, storage=storage, tau=c["tau"],
                          s=s, bc=iilbm.BC_CHANNEL, u_max=0.05)
        g.init_equilibrium(ux=parabola(c["nx"], c["ny"]))
        g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                        aux=np.zeros((c["n"], 2)))
        return g
    o = lib.Oracle(c["nx"], c["ny"], collision=lib.MRT, tau=c["tau"], s=s, bc=lib.BC_CHANNEL,
                   u_max=0.05)
    o.init_equilibrium(ux=parabola(c["nx"], c["ny"]))
    o.set_interface(X, model=lib.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                    UD=np.zeros((c["n"], 2)))
    return o


def test_channel_direct_forcing_batch(orc):
    """Two cylinder channels of different size under direct forcing (5 force updates per
    step), 40 steps in the batch: against the lattices alone and the FP64 oracle."""
    solo = [channel(c, iilbm) for c in CHANNELS]
    batched = [channel(c, iilbm) for c in CHANNELS]
    for g in solo:
        g.step(40)
    with iilbm.Batch(batched) as B:
        B.step(40)
        for a, b in zip(batched, solo):
            assert max_vel_diff(a, b) < 1e-5
            fa, fb = np.array(a.iilbm_get_body_force()), np.array(b.iilbm_get_body_force())
            assert np.linalg.norm(fa - fb) <= 1e-5 * np.linalg.norm(fb)
        o = channel(CHANNELS[0], orc)
        o.step(40)
        _, ug, vg = batched[0].get_macros()
        _, uo, vo = o.current_macros()
        assert max(rel_err(ug, uo, 0.05), rel_err(vg, vo, 0.05)) < 1e-5
