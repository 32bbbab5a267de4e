"""The three-dimensional (D3Q19) II-LBM on the GPU against the FP64 oracle: the lattice
alone, body forces, the uniform-traction sphere (exact fixed point), the jump field of a
triangulated surface, moving surface-tension surfaces in both forms, FP32 storage, graph
replay, and ragged sizes."""
import itertools

import numpy as np
import pytest

from oracle import oracle3d as o3
from paper_2003_12186_gb300 import iilbm3d
from paper_2003_12186_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm3d.load()


def pair(nx, ny, nz, collision="mrt", storage="f64", tau=0.8, jump=1, force="guo",
         body=(0.0, 0.0, 0.0)):
    cg = iilbm3d.MRT if collision == "mrt" else iilbm3d.SRT
    co = o3.MRT if collision == "mrt" else o3.SRT
    fg = iilbm3d.FORCE_SIMPLE if force == "simple" else iilbm3d.FORCE_GUO
    fo = o3.FORCE_SIMPLE if force == "simple" else o3.FORCE_GUO
    g = iilbm3d.Lattice3D(nx, ny, nz, collision=cg, storage=storage, tau=tau, jump=jump, force=fg,
                          body=body)
    o = o3.Oracle3D(nx, ny, nz, collision=co, tau=tau, jump=jump, force=fo, body=body)
    return g, o


def vel_err(g, o, uref):
    _, ug, vg, wg = g.get_macros()
    _, uo, vo, wo = o.current_macros()
    return max(np.abs(ug - uo).max(), np.abs(vg - vo).max(), np.abs(wg - wo).max()) / uref


@pytest.mark.parametrize("collision", ["srt", "mrt"])
@pytest.mark.parametrize("shape", [(16, 12, 10), (37, 29, 23), (150, 6, 5)])
def test_lattice_alone_fp64(collision, shape):
    """Random populations streamed and collided: equal to the oracle step by step, at
    both AA parities, on sizes with ragged tiles."""
    nx, ny, nz = shape
    g, o = pair(nx, ny, nz, collision)
    df = W.random_df3(nx, ny, nz, 1e-4, 11)
    g.set_populations(df)
    o.set_df(df)
    for n in (1, 1, 3, 6):
        g.step(n)
        o.step(n)
        assert np.abs(g.get_populations() - o.get_df()).max() < 1e-17


@pytest.mark.parametrize("force", ["guo", "simple"])
def test_body_force_fp64(force):
    g, o = pair(14, 11, 9, "mrt", force=force, body=(1e-5, -2e-5, 3e-6))
    df = W.random_df3(14, 11, 9, 1e-4, 12)
    g.set_populations(df)
    o.set_df(df)
    for n in (1, 4, 9):
        g.step(n)
        o.step(n)
        assert np.abs(g.get_populations() - o.get_df()).max() < 1e-17
    assert vel_err(g, o, 1e-4) < 1e-12


def _sphere(level=3, R=5.3, c=(12.21, 11.83, 12.47)):
    X, T = W.icosphere(level)
    return X * R + np.asarray(c), T


def _exact_sphere_state(X, T, n, F):
    """u = 0, rho0 - 3F inside (the pressure jump F), as the streamed state."""
    drho = np.zeros((n, n, n))
    for z, y, x in itertools.product(range(n), repeat=3):
        if o3.inside(X, T, x, y, z):
            drho[z, y, x] = -3.0 * F
    E, w = o3.lattice()
    return np.stack([w[i] * np.roll(drho, tuple(E[i][::-1]), axis=(0, 1, 2)) for i in range(19)])


@pytest.mark.parametrize("storage,tol", [("f64", 1e-16), ("f32", 2e-8)])
def test_uniform_traction_sphere_is_a_fixed_point(storage, tol):
    """Section 4.1 in three dimensions: a uniform normal traction on a closed surface,
    started from the exact solution (u = 0, pressure jump F), stays there in the II-LBM;
    the GPU's cut links are the oracle's (equal counts); the IB-LBM drives currents."""
    n, F = 24, -2e-3
    X, T = _sphere()
    nrm, _ = o3.surface_geometry(X, T)
    df = _exact_sphere_state(X, T, n, F)
    errs = {}
    for jump in (1, 0):
        g, o = pair(n, n, n, "mrt", storage=storage, jump=jump)
        g.set_populations(df)
        o.set_df(df)
        g.set_surface(X, T, model=iilbm3d.PRESCRIBED, G=F * nrm)
        o.set_surface(X, T, model=o3.PRESCRIBED, G=F * nrm)
        g.step(20)
        o.step(20)
        _, ux, uy, uz = g.get_macros()
        errs[jump] = max(np.abs(ux).max(), np.abs(uy).max(), np.abs(uz).max())
        if jump:
            assert g.get_cut_link_count() == o.cut_link_count() > 1000
    assert errs[1] < tol
    assert errs[0] > 1e-6


def test_jump_field_matches_the_oracles_records():
    """A rotated ellipsoid with a random prescribed force: the jump field (which links,
    which directions, how much) equals the oracle's."""
    n = 20
    X, T = W.ellipsoid_surface((9.7, 10.2, 10.05), (6.1, 4.3, 3.6), 2, seed=13)
    G = np.random.default_rng(13).uniform(-1e-3, 1e-3, X.shape)
    g, o = pair(n, n, n, "mrt")
    g.set_surface(X, T, model=iilbm3d.PRESCRIBED, G=G)
    o.set_surface(X, T, model=o3.PRESCRIBED, G=G)
    Jg = g.get_jump()
    Jo, cnt = o.jump_field()
    assert cnt > 1000 and g.get_cut_link_count() == cnt
    assert ((Jg != 0) == (Jo != 0)).all()
    assert np.abs(Jg - Jo).max() < 1e-15 * max(1e-6, np.abs(Jo).max()) * 100


@pytest.mark.parametrize("collision,jump,force", [("mrt", 1, "guo"), ("srt", 1, "guo"),
                                                  ("mrt", 0, "guo"), ("mrt", 1, "simple"),
                                                  ("mrt", 0, "simple")])
def test_moving_tension_surface_fp64(collision, jump, force):
    """A surface-tension ellipsoid relaxing with its vertices moving (Eq. 20): markers,
    forces and every population follow the oracle step by step."""
    n = 20
    X, T = W.ellipsoid_surface((10.1, 9.8, 10.3), (5.0, 4.0, 3.4), 2, seed=9)
    g, o = pair(n, n, n, collision, jump=jump, force=force)
    g.set_surface(X, T, model=iilbm3d.TENSION, moves=True, gamma=2e-3)
    o.set_surface(X, T, model=o3.TENSION, moves=True, gamma=2e-3)
    for k in (1, 2, 7, 20):
        g.step(k)
        o.step(k)
        mg, mo = g.get_markers(), o.markers()
        assert np.abs(mg["X"] - mo["X"]).max() < 1e-12
        assert np.abs(mg["Fn"] - mo["Fn"]).max() < 1e-12 * np.abs(mo["Fn"]).max()
        assert np.abs(g.get_populations() - o.get_df()).max() < 1e-15
    assert np.abs(mg["X"] - X).max() > 1e-4


def test_moving_tension_surface_fp32():
    n = 24
    X, T = W.ellipsoid_surface((12.1, 11.8, 12.3), (6.0, 4.8, 4.0), 2, seed=10)
    g, o = pair(n, n, n, "mrt", storage="f32")
    g.set_surface(X, T, model=iilbm3d.TENSION, moves=True, gamma=3e-3)
    o.set_surface(X, T, model=o3.TENSION, moves=True, gamma=3e-3)
    g.step(60)
    o.step(60)
    uref = max(np.abs(o.markers()["U"]).max(), 1e-6)
    assert vel_err(g, o, uref) < 1e-5
    assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-6


def test_graph_replay_and_read_outs_do_not_change_the_run():
    """Steps replayed from graphs equal eager steps (timing on runs eagerly); reading the
    macroscopic fields or the jump between steps, or a read-out followed by a fresh
    equilibrium before the first step, changes nothing: populations, vertices and the
    G and Fn the read-out returns (those of the last step's level)."""
    n = 16
    X, T = W.ellipsoid_surface((8.1, 7.9, 8.2), (4.0, 3.2, 2.8), 2, seed=14)
    runs = []
    for mode in ("graph", "eager", "reads", "restart"):
        g = iilbm3d.Lattice3D(n, n, n, storage="f64")
        g.set_surface(X, T, model=iilbm3d.TENSION, moves=True, gamma=2e-3)
        if mode == "restart":
            # a read-out runs the level's vertex pass; a fresh equilibrium keeps it valid
            g.get_jump()
            g.init_equilibrium()
        if mode == "eager":
            g.set_timing(True)
        for k in (5, 1, 8, 3):
            if mode == "reads":
                g.get_macros()
                g.get_jump()
                for _ in range(k):
                    g.step(1)
            else:
                g.step(k)
        m = g.get_markers()
        runs.append((g.get_populations(), m["X"], m["Fn"], m["G"]))
    for df, Xg, Fn, G in runs[1:]:
        assert np.abs(df - runs[0][0]).max() < 1e-17
        assert np.abs(Xg - runs[0][1]).max() < 1e-14
        assert np.abs(Fn - runs[0][2]).max() <= 1e-14 * np.abs(runs[0][2]).max()
        assert np.abs(G - runs[0][3]).max() <= 1e-14 * np.abs(runs[0][3]).max()


def test_surface_validation():
    g = iilbm3d.Lattice3D(16, 16, 16)
    X, T = _sphere(level=1, R=4.0, c=(8, 8, 8))
    bad = T.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(iilbm3d.IilbmError) as e:
        g.set_surface(X, bad, model=iilbm3d.TENSION, gamma=1e-3)
    assert e.value.code == -6
    big, Tb = _sphere(level=0, R=9.0, c=(8, 8, 8))  # edges of 9.5 nodes
    with pytest.raises(iilbm3d.IilbmError):
        g.set_surface(big, Tb, model=iilbm3d.TENSION, gamma=1e-3)
    with pytest.raises(iilbm3d.IilbmError):
        g.set_surface(X, T, model=iilbm3d.PRESCRIBED)  # no force given
    g.set_surface(X, T, model=iilbm3d.TENSION, gamma=1e-3)
    g.step(3)
    g.synchronize()


def test_surface_across_the_periodic_boundary_fp64():
    """A moving tension surface centred on the box's corner: its cut links, spreading and
    interpolation wrap on every axis, step by step like the oracle's."""
    n = 18
    X, T = W.ellipsoid_surface((0.37, 17.6, 0.21), (4.6, 3.9, 3.3), 2, seed=21)
    g, o = pair(n, n, n, "mrt")
    g.set_surface(X, T, model=iilbm3d.TENSION, moves=True, gamma=2e-3)
    o.set_surface(X, T, model=o3.TENSION, moves=True, gamma=2e-3)
    for k in (1, 3, 10):
        g.step(k)
        o.step(k)
        assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-12
        assert np.abs(g.get_populations() - o.get_df()).max() < 1e-15
    assert g.get_cut_link_count() == o.cut_link_count() > 500


@pytest.mark.parametrize("collision,force", [("srt", "simple"), ("mrt", "guo")])
def test_body_force_with_a_moving_surface(collision, force):
    """A uniform body force drives the box while a tension surface moves with it: the
    force reaches every node (lean tiles included) and the flagged tiles add it to the
    spread force."""
    n = 16
    X, T = W.ellipsoid_surface((8.1, 7.9, 8.2), (4.0, 3.2, 2.8), 2, seed=22)
    body = (2e-6, -1e-6, 5e-7)
    g, o = pair(n, n, n, collision, force=force, body=body)
    g.set_surface(X, T, model=iilbm3d.TENSION, moves=True, gamma=1e-3)
    o.set_surface(X, T, model=o3.TENSION, moves=True, gamma=1e-3)
    g.step(12)
    o.step(12)
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-15
    assert vel_err(g, o, 1e-5) < 1e-10


def test_surfaces_replaced_and_removed():
    """A surface can be replaced by another of a different size and removed; the lattice
    then streams alone, and every read-out works without a surface."""
    n = 16
    g, o = pair(n, n, n, "mrt")
    X1, T1 = W.ellipsoid_surface((8.0, 8.0, 8.0), (4.0, 3.5, 3.0), 1, seed=23)
    X2, T2 = W.ellipsoid_surface((7.7, 8.3, 8.1), (5.0, 4.0, 3.5), 2, seed=24)
    g.set_surface(X1, T1, model=iilbm3d.TENSION, moves=True, gamma=2e-3)
    o.set_surface(X1, T1, model=o3.TENSION, moves=True, gamma=2e-3)
    g.get_macros()  # a read-out before the first step (the level is prepared once)
    g.step(3)
    o.step(3)
    g.set_surface(X2, T2, model=iilbm3d.TENSION, moves=True, gamma=1e-3)
    o.set_surface(X2, T2, model=o3.TENSION, moves=True, gamma=1e-3)
    g.step(4)
    o.step(4)
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-15
    g.set_surface(None, None)
    df = g.get_populations()
    g2, o2 = pair(n, n, n, "mrt")
    g2.set_populations(df)
    o2.set_df(df)
    g.step(5)
    o2.step(5)
    assert np.abs(g.get_populations() - o2.get_df()).max() < 1e-17
    assert not np.abs(g.get_jump()).any()
    d, ux, uy, uz = g.get_macros()
    assert np.all(np.isfinite(ux))


def test_jump_field_fp32_matches_the_oracle():
    """The FP32 lattice forms each crossing's coefficient in FP32: the same links as the
    oracle's, values within FP32 rounding."""
    n = 20
    X, T = W.ellipsoid_surface((9.7, 10.2, 10.05), (6.1, 4.3, 3.6), 2, seed=13)
    G = np.random.default_rng(13).uniform(-1e-3, 1e-3, X.shape)
    g, o = pair(n, n, n, "mrt", storage="f32")
    g.set_surface(X, T, model=iilbm3d.PRESCRIBED, G=G)
    o.set_surface(X, T, model=o3.PRESCRIBED, G=G)
    Jg = g.get_jump()
    Jo, cnt = o.jump_field()
    assert g.get_cut_link_count() == cnt
    mask = (Jo != 0)
    assert (mask == (Jg != 0)).all()
    assert np.abs(Jg - Jo).max() < 1e-6 * np.abs(Jo).max()


def test_full_size_membrane_fp32_matches_the_oracle():
    """The benchmark's own workload and launch configuration (256^3 surface-tension
    ellipsoid, 40 962 vertices, FP32, MRT, graph replay of two steps): the first level's
    jump field crosses the same links as the oracle's (index work, exact); after four
    steps the cut-link count equals the oracle's, and the vertices and every population
    agree with the FP64 oracle to FP32 rounding."""
    w = W.membrane_3d(256)
    n = w["n"]
    g = iilbm3d.Lattice3D(n, n, n, collision=iilbm3d.MRT, storage="f32", tau=w["tau"])
    try:
        o = o3.Oracle3D(n, n, n, parallel=True, collision=o3.MRT, tau=w["tau"])
    except RuntimeError:  # no OpenMP build: the serial oracle
        o = o3.Oracle3D(n, n, n, collision=o3.MRT, tau=w["tau"])
    g.set_surface(w["X"], w["T"], model=iilbm3d.TENSION, moves=True, gamma=w["gamma"])
    o.set_surface(w["X"], w["T"], model=o3.TENSION, moves=True, gamma=w["gamma"])
    # the first level's jump field: the same links in every direction, values to FP32
    Jg = g.get_jump()
    Jo, cnt = o.jump_field()
    assert cnt > 500000 and g.get_cut_link_count() == cnt
    assert ((Jg != 0) == (Jo != 0)).all()
    assert np.abs(Jg - Jo).max() <= 1e-5 * np.abs(Jo).max()
    del Jg, Jo
    g.step(4)
    o.step(4)
    assert g.get_cut_link_count() == o.cut_link_count() > 500000
    mg, mo = g.get_markers(), o.markers()
    assert np.abs(mg["X"] - mo["X"]).max() < 1e-6
    dg, do = g.get_populations(), o.get_df()
    assert np.abs(dg - do).max() <= 1e-5 * np.abs(do).max()
