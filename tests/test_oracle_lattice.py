"""Pins of the oracle's lattice part (equilibrium, Guo forcing, SRT/MRT collision,
streaming, walls) against closed forms and invariants fixed by the paper and by
lattice Boltzmann theory.  CPU only."""
import math

import numpy as np
import pytest

from paper_2003_12186_gb300 import workloads as W

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_mrt_basis_is_orthogonal_with_textbook_norms(orc):
    """Lallemand-Luo basis: rows mutually orthogonal with squared norms
    (9, 36, 36, 6, 12, 6, 12, 4, 4); M^-1 M = I; the rest state w*rho0 has moments
    rho0 (1, -2, 1, 0, ..., 0)."""
    M, Mi = orc.mrt_matrix()
    G = M @ M.T
    assert np.allclose(G, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]), atol=0, rtol=0)
    assert np.abs(Mi @ M - np.eye(9)).max() < 1e-15
    assert np.abs(Mi - orc.invert9(M)).max() < 1e-15
    assert np.abs(Mi - np.linalg.inv(M)).max() < 1e-15
    assert np.allclose(M @ WT, [1, -2, 1, 0, 0, 0, 0, 0, 0], atol=1e-16)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.05, -0.02), (0.97, -0.1, 0.07)])
def test_equilibrium_moments(orc, rho, ux, uy):
    """Eq. 23: sum f_eq = rho, sum e f_eq = rho u, sum e_a e_b f_eq = rho c_s^2 d_ab +
    rho u_a u_b (Maxwellian moments the equilibrium is built to match)."""
    rho0 = 1.0
    f = orc.feq_shifted(rho, rho0, ux, uy) + WT * rho0
    u = np.array([ux, uy])
    assert abs(f.sum() - rho) < 1e-15
    assert np.abs(E.T @ f - rho * u).max() < 1e-16
    P = np.einsum("i,ia,ib->ab", f, E, E)
    assert np.abs(P - (rho / 3 * np.eye(2) + rho * np.outer(u, u))).max() < 1e-15


def test_guo_source_moments(orc):
    """Eq. 21 source: zeroth moment 0, first moment g, second moment u g + g u."""
    u = np.array([0.04, -0.03])
    g = np.array([2e-4, 5e-5])
    Gt = orc.guo_source(u[0], u[1], g[0], g[1])
    assert abs(Gt.sum()) < 1e-19
    assert np.abs(E.T @ Gt - g).max() < 1e-19
    P = np.einsum("i,ia,ib->ab", Gt, E, E)
    assert np.abs(P - (np.outer(u, g) + np.outer(g, u))).max() < 1e-19


@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_rest_state_is_preserved_bitwise(orc, collision):
    o = orc.Oracle(12, 10, collision=orc.SRT if collision == "srt" else orc.MRT, tau=0.7,
                   s=W.mrt_rates(0.7))
    o.step(15)
    assert np.all(o.get_df() == 0.0)


@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_uniform_flow_is_preserved(orc, collision):
    """A uniform-velocity equilibrium in a periodic box is a steady solution."""
    nx, ny = 8, 6
    o = orc.Oracle(nx, ny, collision=orc.SRT if collision == "srt" else orc.MRT, tau=0.9,
                   s=W.mrt_rates(0.9))
    o.init_equilibrium(np.full(nx * ny, 1.02), np.full(nx * ny, 0.06), np.full(nx * ny, -0.03))
    df0 = o.get_df()
    o.step(20)
    assert np.abs(o.get_df() - df0).max() < 1e-15


def test_mrt_with_equal_rates_equals_srt(orc):
    """M^-1 (I/tau) M = I/tau: MRT with every rate 1/tau is SRT (with Guo forcing:
    M^-1 (I - I/(2 tau)) M = (1 - 1/(2 tau)) I)."""
    rng = np.random.default_rng(3)
    tau = 0.77
    for _ in range(20):
        df = 1e-2 * rng.standard_normal(9)
        g = 1e-3 * rng.standard_normal(2)
        a = orc.collide_cell(orc.make_cfg(1, 1, collision=orc.SRT, tau=tau), df, *g)
        b = orc.collide_cell(orc.make_cfg(1, 1, collision=orc.MRT, tau=tau, s=[1 / tau] * 9),
                             df, *g)
        assert np.abs(a - b).max() < 1e-15


def test_mrt_conserved_rates_do_not_matter(orc):
    """With Guo's forcing the conserved-moment rates s0, s3, s5 drop out: the mass and
    momentum moments are unchanged by the relaxation term, while the forcing term
    adds exactly g to j.  So the paper's rates with s1=s2=s4=s6=s7=s8=1/tau give SRT."""
    rng = np.random.default_rng(4)
    tau = 0.6
    s = [0, 1 / tau, 1 / tau, 0, 1 / tau, 0, 1 / tau, 1 / tau, 1 / tau]
    for _ in range(20):
        df = 1e-2 * rng.standard_normal(9)
        g = 1e-3 * rng.standard_normal(2)
        a = orc.collide_cell(orc.make_cfg(1, 1, collision=orc.SRT, tau=tau), df, *g)
        b = orc.collide_cell(orc.make_cfg(1, 1, collision=orc.MRT, tau=tau, s=s), df, *g)
        assert np.abs(a - b).max() < 1e-15


@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_shear_wave_decays_at_the_viscosity_of_eq7(orc, collision):
    """Eq. 7: nu = c_s^2 (tau - 1/2).  A shear wave u_x = U sin(k y) decays as
    exp(-nu k^2 t); with ny = 128 the lattice's O(k^2) error is far below 1%."""
    nx, ny, tau, U, T = 4, 128, 0.8, 1e-4, 400
    o = orc.Oracle(nx, ny, collision=orc.SRT if collision == "srt" else orc.MRT, tau=tau,
                   s=W.mrt_rates(tau))
    k = 2 * math.pi / ny
    y = np.repeat(np.arange(ny), nx)
    o.init_equilibrium(None, U * np.sin(k * y), None)
    o.step(T + 1)
    _, ux, _ = o.step_macros()  # velocity at time T
    amp = 2 * np.mean(ux[:, 0] * np.sin(k * np.arange(ny)))
    nu = (tau - 0.5) / 3
    assert abs(amp / (U * math.exp(-nu * k * k * T)) - 1) < 1e-2
    # a wrong viscosity relation (e.g. nu = c_s^2 tau) would miss by > 50 %
    assert abs(math.exp(-tau / 3 * k * k * T) / math.exp(-nu * k * k * T) - 1) > 0.05


@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_body_force_adds_exact_momentum(orc, collision):
    """Guo forcing (Eqs. 21-24): a uniform body force g in a periodic box adds exactly
    g of momentum per cell per step, and u(t) = (t + 1/2) g / rho0."""
    nx, ny, g = 6, 5, (3e-5, -1e-5)
    o = orc.Oracle(nx, ny, collision=orc.SRT if collision == "srt" else orc.MRT, tau=0.7,
                   s=W.mrt_rates(0.7), body=g)
    for t in range(30):
        o.step(1)
        r, ux, uy = o.step_macros()
        assert np.abs(ux - (t + 0.5) * g[0]).max() < 1e-17 + 1e-13 * abs(g[0]) * t
        assert np.abs(uy - (t + 0.5) * g[1]).max() < 1e-17 + 1e-13 * abs(g[1]) * t
        assert np.abs(r - 1.0).max() < 1e-15
    df = o.get_df()
    jx = np.tensordot(E[:, 0], df, axes=(0, 0)).sum()
    assert abs(jx - 30 * g[0] * nx * ny) < 1e-15


def _poiseuille(orc, collision, tau, s=None, ny=8, steps=12000):
    g = 1e-6
    o = orc.Oracle(2, ny, collision=collision, tau=tau, s=s, bc=orc.BC_WALLS_Y, body=(g, 0.0))
    o.step(steps)
    _, ux, _ = o.step_macros()
    y = np.arange(ny) + 0.5  # walls at y = -1/2 and ny - 1/2
    nu = (tau - 0.5) / 3 if collision == orc.SRT else (1 / s[7] - 0.5) / 3
    exact = g / (2 * nu) * y * (ny - y)
    return ux[:, 0], exact


def test_poiseuille_exact_at_magic_parameter(orc):
    """Halfway bounce-back puts the wall exactly midway when (tau - 1/2)^2 = 3/16
    (SRT), so the body-force channel flow is the exact parabola u = g y (H - y)/(2 nu)
    with H = ny and y measured from the wall."""
    tau = 0.5 + math.sqrt(3 / 16)
    u, ex = _poiseuille(orc, orc.SRT, tau)
    assert np.abs(u / ex - 1).max() < 1e-8


def test_poiseuille_mrt_exact_at_magic_parameter(orc):
    """MRT: (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 gives the exact parabola as well."""
    tau = 0.9
    sq = 1 / (0.5 + (3 / 16) / (tau - 0.5))
    s = [0, 1.63, 1.14, 0, sq, 0, sq, 1 / tau, 1 / tau]
    u, ex = _poiseuille(orc, orc.MRT, tau, s=s, steps=9000)
    assert np.abs(u / ex - 1).max() < 1e-8


def test_poiseuille_second_order_away_from_magic(orc):
    """At other tau the wall-slip error is O(1/ny^2): the error ratio between ny = 8
    and ny = 16 is about 4."""
    tau = 1.0
    errs = []
    for ny in (8, 16):
        u, ex = _poiseuille(orc, orc.SRT, tau, ny=ny, steps=int(2.2 * ny * ny / ((tau - 0.5) / 3)))
        errs.append(np.abs(u - ex).max() / ex.max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_channel_inflow_sets_the_prescribed_velocity(orc):
    """Non-equilibrium extrapolation keeps the neighbour's non-equilibrium part, whose
    first moment is zero, so the inflow node carries exactly u_in(y) and rho(1, y)."""
    nx, ny, um = 16, 10, 0.05
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.8, s=W.mrt_rates(0.8), bc=orc.BC_CHANNEL,
                   u_max=um)
    o.step(40)
    o.step(1)
    r, ux, uy = o.step_macros()
    y = np.arange(ny) + 0.5
    uin = 4 * um * y * (ny - y) / ny ** 2
    assert np.abs(ux[:, 0] - uin).max() < 1e-15
    assert np.abs(uy[:, 0]).max() < 1e-16
    assert np.abs(r[:, 0] - r[:, 1]).max() < 1e-15


def test_channel_outflow_copies_exactly_the_unknown_populations(orc):
    """Zero-gradient outflow pinned by a one-step computation from the (separately pinned)
    collision.  From a random state, one step of an empty channel must give:
    (1) at column nx - 1, the populations with e_x < 0 (the ones no node streams in)
        equal to those of column nx - 2, bitwise;
    (2) every other population of column nx - 1 equal to the post-collision value of its
        source node x - e_i (the node's own opposite population where the source lies
        beyond a wall: halfway bounce-back), computed here cell by cell;
    (3) the e_x < 0 populations of column nx - 2 likewise streamed in from column
        nx - 1, not copied.
    A copy of the wrong set (e_x > 0), from the wrong column, or onto the wrong column
    fails one of the three."""
    nx, ny, tau = 12, 9, 0.8
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=tau, s=W.mrt_rates(tau), bc=orc.BC_CHANNEL,
                   u_max=0.03)
    df = W.random_df(nx, ny, 1e-3, 5)
    o.set_df(df)
    post = np.array([[orc.collide_cell(o.cfg, df[:, y, x]) for x in range(nx)]
                     for y in range(ny)])  # [ny][nx][9]
    o.step(1)
    d = o.get_df()
    EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]

    def streamed(i, x, y):
        sx, sy = x - EX[i], y - EY[i]
        return post[y, x, OPP[i]] if not 0 <= sy < ny else post[sy, sx, i]

    for y in range(ny):
        for i in range(9):
            if EX[i] < 0:
                assert d[i, y, nx - 1] == d[i, y, nx - 2]                  # (1)
                assert d[i, y, nx - 2] == streamed(i, nx - 2, y)           # (3)
            else:
                assert d[i, y, nx - 1] == streamed(i, nx - 1, y)           # (2)
    # the copy is not vacuous: the two columns' unknown populations differ before it
    assert any(streamed(i, nx - 1 - 1, y) != post[y, nx - 1, i]
               for y in range(ny) for i in (3, 6, 7))


# ------------------------------------------------- the paper's boxes, simple force
@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_simple_force_adds_exact_momentum(orc, collision):
    """The simple external force term (Eq. 16: (1/c_s^2) w_i e_i . g per population)
    adds exactly g to the momentum each step and the velocity is sum e f / rho, so a
    uniform body force in a periodic box gives u(t) = t g / rho0 at the collision of step
    t (the Guo form gives (t + 1/2) g / rho0, pinned above)."""
    c = orc.MRT if collision == "mrt" else orc.SRT
    for g in ((1e-5, 0.0), (2e-6, -3e-6)):
        o = orc.Oracle(12, 10, collision=c, tau=0.7, s=W.mrt_rates(0.7), body=g,
                       force=orc.FORCE_SIMPLE)
        for t in (1, 4, 9):
            o.step(1 if t == 1 else (t - (1 if t == 4 else 4)))
            _, ux, uy = o.current_macros()
            assert np.allclose(ux, t * g[0], rtol=1e-12, atol=0)
            assert np.allclose(uy, t * g[1], rtol=1e-12, atol=1e-22)


def _box_macros(o, x, y):
    df = o.get_df()[:, y, x]
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    d = df.sum()
    ux = sum(e[0] * f for e, f in zip(E, df)) / (1.0 + d)
    uy = sum(e[1] * f for e, f in zip(E, df)) / (1.0 + d)
    return d, ux, uy


@pytest.mark.parametrize("bc", ["wall", "outflow"])
def test_box_boundary_nodes_carry_the_prescribed_values(orc, bc):
    """Non-equilibrium extrapolation on the four sides of a box: the non-equilibrium part
    copied from the inward neighbour has zero mass and momentum, so every edge node
    carries exactly (to rounding) u = 0 and the neighbour's density on a wall, and the
    reference density with the neighbour's velocity at an outflow; corners take the
    diagonal neighbour.  From a random state, after every step."""
    nx, ny = 13, 9
    kind = orc.BC_BOX_WALL if bc == "wall" else orc.BC_BOX_OUTFLOW
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.75, s=W.mrt_rates(0.75), bc=kind)
    o.set_df(W.random_df(nx, ny, 1e-3, 11))
    for _ in range(3):
        o.step(1)
        for y in range(ny):
            for x in range(nx):
                if 0 < x < nx - 1 and 0 < y < ny - 1:
                    continue
                px, py = x + (x == 0) - (x == nx - 1), y + (y == 0) - (y == ny - 1)
                d, ux, uy = _box_macros(o, x, y)
                dn, uxn, uyn = _box_macros(o, px, py)
                if bc == "wall":
                    assert abs(ux) < 1e-17 and abs(uy) < 1e-17 and abs(d - dn) < 1e-17
                else:
                    assert abs(d) < 1e-17 and abs(ux - uxn) < 1e-16 and abs(uy - uyn) < 1e-16


def test_box_wall_keeps_rest_and_damps_a_disturbance(orc):
    """A wall box at rest stays at rest bitwise; a disturbance inside it decays (the
    walls take its momentum: no node keeps a velocity above 1% of the start's after
    2000 steps)."""
    nx, ny = 24, 20
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.7, s=W.mrt_rates(0.7), bc=orc.BC_BOX_WALL)
    o.step(20)
    assert np.all(o.get_df() == 0.0)
    yy, xx = np.mgrid[0:ny, 0:nx]
    u0 = 0.01 * np.sin(np.pi * xx / (nx - 1)) * np.sin(np.pi * yy / (ny - 1))
    o.init_equilibrium(None, u0, None)
    o.step(2000)
    _, ux, uy = o.step_macros()
    assert np.hypot(ux, uy).max() < 0.01 * 0.01
