"""The cubic-spline interface of a flexible boundary (end of section 3.2: normals, |X_s|
and the jump strength from the spline through the markers, crossings on m chords per
segment), CUDA path against the FP64 oracle."""
import numpy as np
import pytest

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

from _pair import assert_jump_fields_agree, make_pair, oracle_jump_field, vel_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def ellipse_two_apart(n=128):
    """An ellipse membrane with markers about two lattice units apart (the marker
    spacing section 4.2 gives the II-LBM), stretched so that it moves."""
    X = W.ellipse_markers(63.7, 64.4, 38.0, 26.0, 100)
    dX = W.polygon_perimeter(X) / 100
    return X, dX * 0.9


@pytest.mark.parametrize("curve", [1, 4])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_spline_membrane_matches_oracle(orc, storage, curve):
    """A moving elastic membrane whose jump lives on the spline: the populations follow
    the oracle step by step (FP64 to 1e-12; FP32 velocity to 1e-5), the markers too, and
    the jump field's cut links are the oracle's exactly."""
    X, dX = ellipse_two_apart()
    g, o = make_pair(orc, 128, 128, collision="mrt", storage=storage, tau=0.7)
    g.set_interface(X, model=iilbm.SPRING, stiffness=0.02, dX=dX, curve=curve)
    o.set_interface(X, model=orc.SPRING, kappa=0.02, dX=dX, curve=curve)
    Jo, _ = oracle_jump_field(orc, o, curve)
    assert_jump_fields_agree(g.iilbm_get_jump(), Jo, 1e-11 if storage == "f64" else 2e-6)
    umax = 0.0
    for _ in range(3):
        g.step(40)
        o.step(40)
        umax = max(umax, np.abs(o.markers()["U"]).max())
        if storage == "f64":
            assert np.abs(g.get_populations() - o.get_df()).max() < 1e-13
            assert np.abs(g.get_markers()["X"] - o.markers()["X"]).max() < 1e-11
    assert umax > 1e-5  # the membrane moves
    assert vel_error(g, o, umax) < (1e-11 if storage == "f64" else 1e-5)
    Jo, count = oracle_jump_field(orc, o, curve)
    assert_jump_fields_agree(g.iilbm_get_jump(), Jo, 1e-10 if storage == "f64" else 2e-6)
    assert g.iilbm_get_cut_link_count() == count


def test_spline_uniform_normal_force_is_a_fixed_point(orc):
    """Section 4.1's exact solution with the jump on the spline: a uniform normal force
    on a circle of markers and the piecewise-constant pressure of the spline's chords is
    kept by the GPU step to rounding (FP64), as by the oracle."""
    nx = ny = 40
    R, F, n, m = 10.0, -2e-3, 64, 4
    c0 = np.array([20.3, 19.8])
    X = W.circle_markers(c0[0], c0[1], R, n)
    nrm = (X - c0) / np.linalg.norm(X - c0, axis=1, keepdims=True)
    cx, cy = orc.spline_coeffs(X[:, 0]), orc.spline_coeffs(X[:, 1])
    s = np.arange(n * m) / m
    P = np.stack([[orc.spline_eval(cx, t) for t in s], [orc.spline_eval(cy, t) for t in s]], 1)
    wind = np.array([[orc.winding(P, x, y) for x in range(nx)] for y in range(ny)])
    rho = 1.0 - wind * F * 3
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    WT = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    df = np.stack([WT[i] * (np.roll(rho, (ey, ex), axis=(0, 1)) - 1.0)
                   for i, (ex, ey) in enumerate(E)])
    g, o = make_pair(orc, nx, ny, collision="mrt", storage="f64", tau=0.8)
    g.set_populations(df)
    o.set_df(df)
    dX = W.polygon_perimeter(X) / n
    g.set_interface(X, model=iilbm.PRESCRIBED, moves=False, dX=dX, aux=F * nrm, curve=m)
    o.set_interface(X, model=orc.PRESCRIBED, moves=False, dX=dX, G=F * nrm, curve=m)
    g.step(30)
    o.step(30)
    _, u, v = g.get_macros()
    assert max(np.abs(u).max(), np.abs(v).max()) < 1e-15
    assert np.abs(g.get_populations() - o.get_df()).max() < 1e-16


def test_spline_interface_is_refused_where_it_does_not_apply():
    """Direct forcing keeps the polygon (a rigid body), the chord count is bounded, and a
    batch takes only polygon interfaces."""
    g = iilbm.Lattice(64, 64, collision=iilbm.MRT, storage="f32", tau=0.8)
    X = W.circle_markers(32.2, 31.7, 10.0, 40)
    with pytest.raises(iilbm.IilbmError):
        g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=1.5, eta=2.0, mdf_iters=5,
                        aux=np.zeros((40, 2)), curve=2)
    with pytest.raises(iilbm.IilbmError):
        g.set_interface(X, model=iilbm.SPRING, stiffness=0.01, dX=1.5, curve=17)
    g.set_interface(X, model=iilbm.SPRING, stiffness=0.01, dX=1.5, curve=2)
    with pytest.raises(iilbm.IilbmError):
        iilbm.Batch([g])
