"""Helpers that set up the same seeded case on the CUDA library and on the oracle."""
import numpy as np

from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W


def rates(collision, tau):
    return W.mrt_rates(tau) if collision == "mrt" else [1.0 / tau] * 9


def make_pair(orc, nx, ny, collision="mrt", storage="f64", tau=0.8, s=None, bc="periodic",
              jump=1, body=(0.0, 0.0), rho0=1.0):
    s = s if s is not None else rates(collision, tau)
    bcg = {"periodic": iilbm.BC_PERIODIC, "walls": iilbm.BC_WALLS_Y}[bc]
    bco = {"periodic": orc.BC_PERIODIC, "walls": orc.BC_WALLS_Y}[bc]
    g = iilbm.Lattice(nx, ny, collision=iilbm.SRT if collision == "srt" else iilbm.MRT,
                      storage=storage, tau=tau, s=s, bc=bcg, jump=jump, body=body, rho0=rho0)
    o = orc.Oracle(nx, ny, collision=orc.SRT if collision == "srt" else orc.MRT, tau=tau, s=s,
                   bc=bco, jump=jump, body=body, rho0=rho0)
    return g, o


def set_membrane(orc, g, o, X, model="spring", kappa=0.05, dX=1.0, l0=1.0, moves=True, G=None):
    mg = {"spring": iilbm.SPRING, "spring_rest": iilbm.SPRING_REST,
          "prescribed": iilbm.PRESCRIBED}[model]
    mo = {"spring": orc.SPRING, "spring_rest": orc.SPRING_REST,
          "prescribed": orc.PRESCRIBED}[model]
    g.set_interface(X, model=mg, moves=moves, stiffness=kappa, dX=dX, rest_length=l0, aux=G)
    o.set_interface(X, model=mo, moves=moves, kappa=kappa, dX=dX, l0=l0, G=G)


def rel_err(u_gpu, u_orc, uref):
    """||a - b||_inf / max(||b||_inf, uref)."""
    return float(np.abs(u_gpu - u_orc).max() / max(np.abs(u_orc).max(), uref))


def vel_error(g, o, uref=1e-6):
    _, ug, vg = g.get_macros()
    _, uo, vo = o.current_macros()
    return max(rel_err(ug, uo, uref), rel_err(vg, vo, uref))


def oracle_jump_field(orc, o, curve=0):
    """The oracle's jump of the current state, J[i-1][y][x] (i = 1..8): its cut-link
    records summed per link (a link crossed twice carries both records); curve = m for
    the spline interface on m chords per segment."""
    o.current_macros()  # runs the current state's interface phase
    m = o.markers()
    if curve > 0:
        cell, d, coef = orc.cut_links_spline(o.cfg, m["X"], m["Fn"], curve)
    else:
        cell, d, coef = orc.cut_links(o.cfg, m["X"], m["Fn"])
    J = np.zeros((8, o.ny * o.nx))
    np.add.at(J, (d - 1, cell), coef)
    return J.reshape(8, o.ny, o.nx), len(cell)


def assert_jump_fields_agree(Jg, Jo, rel):
    """Same cut links (the set of (direction, node) carrying a jump, compared exactly)
    and the same values within rel of the largest."""
    sg, so = Jg != 0, Jo != 0
    assert np.array_equal(sg, so), (f"cut-link sets differ: {int((sg & ~so).sum())} only on "
                                    f"the GPU, {int((so & ~sg).sum())} only in the oracle")
    assert so.sum() > 0
    d = float(np.abs(Jg - Jo).max() / np.abs(Jo).max())
    assert d <= rel, f"jump values differ by {d:.3e} of the largest (bound {rel:.1e})"
