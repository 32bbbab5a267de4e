"""Pins of the oracle's immersed-interface part: the Peskin delta kernel, spreading /
interpolation, Lagrangian forces, the normal split, the cut-link list of the jump
(against an independent exact-rational brute force), and whole-step invariants of
the II-LBM (mass, the exact fixed point of a uniform normal force, Laplace's law).
CPU only."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2003_12186_gb300 import workloads as W

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WT = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4


# ---------------------------------------------------------------- delta kernel
def test_phi_closed_form_values(orc):
    assert orc.phi(0.0) == 0.5
    assert orc.phi(1.0) == 0.25 and orc.phi(-1.0) == 0.25
    assert orc.phi(2.0) == 0.0 and orc.phi(2.5) == 0.0
    assert abs(orc.phi(0.5) - (2 + math.sqrt(2)) / 8) < 1e-16
    assert abs(orc.phi(1.5) - (2 - math.sqrt(2)) / 8) < 1e-16


def test_phi_moment_conditions(orc):
    """Peskin's four-point kernel satisfies, for every shift r: sum_j phi(r-j) = 1,
    sum_j (r-j) phi(r-j) = 0 and sum_j phi(r-j)^2 = 3/8."""
    for r in np.random.default_rng(0).uniform(0, 1, 200):
        v = [orc.phi(r - j) for j in range(-3, 4)]
        d = [r - j for j in range(-3, 4)]
        assert abs(sum(v) - 1) < 1e-15
        assert abs(sum(a * b for a, b in zip(v, d))) < 1e-15
        assert abs(sum(a * a for a in v) - 3 / 8) < 1e-15


def test_spread_and_interp_are_adjoint(orc):
    """<spread(P), u> = <P, interp(u)> (Eqs. 17 and 20 use one kernel), spreading
    conserves the total force and its first moment."""
    rng = np.random.default_rng(1)
    cfg = orc.make_cfg(24, 20)
    X = np.stack([rng.uniform(0, 24, 30), rng.uniform(0, 20, 30)], 1)
    P = rng.standard_normal((30, 2))
    ux, uy = rng.standard_normal((20, 24)), rng.standard_normal((20, 24))
    gx, gy = orc.spread(cfg, X, P)
    U = orc.interp(cfg, X, ux, uy)
    lhs = (gx * ux).sum() + (gy * uy).sum()
    assert abs(lhs - (P * U).sum()) < 1e-12
    assert abs(gx.sum() - P[:, 0].sum()) < 1e-12
    Xi = X[(X[:, 0] > 3) & (X[:, 0] < 20) & (X[:, 1] > 3) & (X[:, 1] < 16)]
    Pi = rng.standard_normal(Xi.shape)
    gx, gy = orc.spread(cfg, Xi, Pi)
    xs = np.arange(24)[None, :]
    assert abs((gx * xs).sum() - (Pi[:, 0] * Xi[:, 0]).sum()) < 1e-12


# -------------------------------------------------------------------- forces
def test_zero_rest_spring_on_regular_polygon(orc):
    """Eq. 19 on a regular N-gon of radius R: G_k = -kappa 2R(1-cos(2 pi/N))/dX^2 r_hat."""
    N, R, kappa, dX = 64, 10.0, 0.3, 0.9
    X = W.circle_markers(5, -2, R, N)
    G = orc.spring_forces(X, orc.SPRING, kappa, dX)
    mag = kappa * 2 * R * (1 - math.cos(2 * math.pi / N)) / dX ** 2
    rhat = (X - [5, -2]) / R
    assert np.abs(G + mag * rhat).max() < 1e-14
    assert np.abs(G.sum(0)).max() < 1e-13


def test_rest_length_spring_on_regular_polygon(orc):
    """Rest-length springs on a regular N-gon: net point force 2 T sin(pi/N) inward with
    segment tension T = kappa (l/l0 - 1)."""
    N, R, kappa = 128, 16.0, 0.01
    X = W.circle_markers(32, 32, R, N)
    l = 2 * R * math.sin(math.pi / N)
    dX, l0 = l, 0.9 * l
    G = orc.spring_forces(X, orc.SPRING_REST, kappa, dX, l0)
    T = kappa * (l / l0 - 1)
    rhat = (X - 32) / R
    assert np.abs(G * dX + 2 * T * math.sin(math.pi / N) * rhat).max() < 1e-15


def test_normal_split(orc):
    """Outward normal of a CCW circle is radial; |X_s| = R sin(2 pi/N)/dX; the split
    rebuilds G; Gpar is orthogonal to n; rigid bodies use |X_s| = 1."""
    N, R, dX = 50, 7.0, 0.8
    X = W.circle_markers(0, 0, R, N)
    rng = np.random.default_rng(2)
    G = rng.standard_normal((N, 2))
    Fn, Gpar, n = orc.normal_split(X, G, moves=True, dX=dX)
    assert np.abs(n - X / R).max() < 1e-14
    Xs = R * math.sin(2 * math.pi / N) / dX
    Gn = (G * n).sum(1)
    assert np.abs(Fn - Gn / Xs).max() < 1e-14
    assert np.abs((Gpar * n).sum(1)).max() < 1e-15
    assert np.abs(Gpar + Gn[:, None] * n - G).max() < 1e-15
    Fn1, _, _ = orc.normal_split(X, G, moves=False, dX=dX)
    assert np.abs(Fn1 - Gn).max() < 1e-15


# ----------------------------------------------------------------- cut links
def _q(v):
    """Snap to the 2^-24 grid (round half to even, as llrint) -- exact Fraction."""
    return Fr(int(np.rint(v * 2 ** 24)), 2 ** 24)


def _brute_cut_links(X, Fn, nx, ny):
    """Every link x-e_i -> x of an (unbounded) lattice window against every polygon
    segment, in exact rational arithmetic, with every lattice node displaced by a
    small explicit (eps, eps^2), eps = 2^-80.  Returns {(cell, i): [(sign, t), ...]}."""
    eps = Fr(1, 2 ** 80)
    n = len(X)
    Q = [(_q(x), _q(y)) for x, y in X]

    def cross(ax, ay, bx, by):
        return ax * by - ay * bx

    out = {}
    xs = [p[0] for p in Q]
    ys = [p[1] for p in Q]
    x0, x1 = math.floor(min(xs)) - 2, math.ceil(max(xs)) + 2
    y0, y1 = math.floor(min(ys)) - 2, math.ceil(max(ys)) + 2
    for k in range(n):
        A, B = Q[k], Q[(k + 1) % n]
        for qy in range(y0, y1 + 1):
            for qx in range(x0, x1 + 1):
                for i in range(1, 9):
                    ex, ey = E[i]
                    P = (qx - ex + eps, qy - ey + eps * eps)
                    R = (qx + eps, qy + eps * eps)
                    d1 = cross(B[0] - A[0], B[1] - A[1], P[0] - A[0], P[1] - A[1])
                    d2 = cross(B[0] - A[0], B[1] - A[1], R[0] - A[0], R[1] - A[1])
                    d3 = cross(ex, ey, A[0] - P[0], A[1] - P[1])
                    d4 = cross(ex, ey, B[0] - P[0], B[1] - P[1])
                    assert d1 != 0 and d2 != 0 and d3 != 0 and d4 != 0
                    if (d1 > 0) == (d2 > 0) or (d3 > 0) == (d4 > 0):
                        continue
                    t = d3 / (d3 - d4)
                    cell = (qy % ny) * nx + (qx % nx)
                    out.setdefault((cell, i), []).append((1 if d1 > 0 else -1, t, k))
    return out


def _check_against_brute(orc, X, nx, ny, seed):
    rng = np.random.default_rng(seed)
    Fn = rng.uniform(-1, 1, len(X))
    cfg = orc.make_cfg(nx, ny)
    cell, d, coef = orc.cut_links(cfg, X, Fn)
    got = {}
    for c, i, v in zip(cell, d, coef):
        got.setdefault((int(c), int(i)), []).append(v)
    ref = _brute_cut_links(X, Fn, nx, ny)
    assert set(got) == set(ref)
    n = len(X)
    for key, lst in ref.items():
        i = key[1]
        want = sorted(float(s * WT[i] * 3 * ((1 - t) * Fr(Fn[k]) + t * Fr(Fn[(k + 1) % n])))
                      for s, t, k in lst)
        have = sorted(got[key])
        assert len(want) == len(have)
        assert np.abs(np.array(want) - np.array(have)).max() < 1e-15
    return len(cell)


def test_cut_links_match_exact_rational_bruteforce(orc):
    """Random generic polygons on a small periodic lattice."""
    total = 0
    for seed in range(4):
        X = W.wobbly_polygon(8.3, 7.7, 4.2, 13, 0.35, seed)
        total += _check_against_brute(orc, X, 18, 16, seed)
    assert total > 100


def test_cut_links_degenerate_contacts_match_bruteforce(orc):
    """Vertices on lattice nodes, on links, and edges along lattice lines and
    diagonals: the symbolic (eps, eps^2) rule must agree with the explicit one."""
    polys = [
        np.array([[2, 2], [7, 2], [7, 6], [4, 6], [2, 4]], float),
        np.array([[2.5, 2], [6, 2.5], [6, 6], [3, 6], [3, 3]], float),
        np.array([[3, 3], [6, 3], [6, 6], [5, 5], [4, 6], [3, 6]], float),
        np.array([[2, 2], [4, 2], [6, 4], [6, 6], [4, 6], [2, 4]], float),
        np.array([[2.25, 2.0], [6.0, 2.0], [6.0, 5.5], [4.0, 7.0], [2.0, 5.0]], float),
    ]
    for s, X in enumerate(polys):
        _check_against_brute(orc, X, 12, 12, 10 + s)


def test_cut_link_signs_follow_the_winding_number(orc):
    """Signed crossings on every link equal winding(x - e_i) - winding(x): the jump is
    added once per net passage from interior to exterior, on any polygon, including a
    strongly non-convex one with links crossed twice."""
    th = np.linspace(0, 2 * np.pi, 61)[:-1]
    r = 9 + 4 * np.sin(5 * th)
    X = np.stack([16.2 + r * np.cos(th), 15.9 + r * np.sin(th)], 1)
    nx = ny = 34
    cfg = orc.make_cfg(nx, ny)
    cell, d, coef = orc.cut_links(cfg, X, np.ones(len(X)))
    net = {}
    for c, i, v in zip(cell, d, coef):
        s = int(np.sign(v))
        net[(int(c), int(i))] = net.get((int(c), int(i)), 0) + s
    wind = np.array([[orc.winding(X, x, y) for x in range(nx)] for y in range(ny)])
    assert wind.sum() > 100 and set(np.unique(wind)) <= {0, 1}
    for y in range(1, ny - 1):
        for x in range(1, nx - 1):
            for i in range(1, 9):
                ex, ey = E[i]
                want = wind[y - ey, x - ex] - wind[y, x]
                assert net.get((y * nx + x, i), 0) == want


def test_winding_matches_exact_ray_cast(orc):
    """orc_winding against a plain even-odd ray cast in exact rationals with the node
    displaced by (eps, eps^2)."""
    X = W.wobbly_polygon(10.1, 9.9, 6.0, 17, 0.4, 7)
    Q = [(_q(a), _q(b)) for a, b in X]
    eps = Fr(1, 2 ** 80)
    for y in range(20):
        for x in range(20):
            px, py = x + eps, y + eps * eps
            inside = False
            for k in range(len(Q)):
                (ax, ay), (bx, by) = Q[k], Q[(k + 1) % len(Q)]
                if (ay > py) != (by > py):
                    xc = ax + (py - ay) * (bx - ax) / (by - ay)
                    if xc > px:
                        inside = not inside
            assert orc.winding(X, x, y) == (1 if inside else 0)


def test_cut_link_hand_computed_values(orc):
    """A CCW square with its right edge on x = 0.5 (outward normal +x) and uniform
    Fn = F: the link (0,0) -> (1,0) (i=1) leaves the interior, so it carries
    +w_1/c_s^2 F = F/3; the diagonal (0,-1) -> (1,0) (i=5) carries F/12; the links
    (1,0) -> (0,0) (i=3) and (1,1) -> (0,0) (i=7) carry -F/3 and -F/12."""
    X = np.array([[-5.5, -5.0], [0.5, -5.0], [0.5, 5.0], [-5.5, 5.0]])
    F = 0.37
    nx = ny = 32
    cfg = orc.make_cfg(nx, ny)
    cell, d, coef = orc.cut_links(cfg, X, np.full(4, F))
    rec = {(int(c), int(i)): v for c, i, v in zip(cell, d, coef)}
    at = lambda x, y: (y % ny) * nx + (x % nx)  # noqa: E731
    assert abs(rec[(at(1, 0), 1)] - F / 3) < 1e-16
    assert abs(rec[(at(1, 0), 5)] - F / 12) < 1e-16
    assert abs(rec[(at(0, 0), 3)] + F / 3) < 1e-16
    assert abs(rec[(at(0, 0), 7)] + F / 12) < 1e-16
    assert (at(1, 0), 2) not in rec  # a link parallel to the edge never crosses it


def test_cut_links_are_translation_invariant(orc):
    X = W.wobbly_polygon(11.3, 10.6, 5.0, 19, 0.3, 3)
    Fn = np.random.default_rng(5).uniform(-1, 1, 19)
    cfg = orc.make_cfg(40, 40)
    a = orc.cut_links(cfg, X, Fn)
    b = orc.cut_links(cfg, X + [7, 12], Fn)
    ka = sorted(((int(c) // 40 + 12) * 40 + (int(c) % 40 + 7), int(i), v) for c, i, v in zip(*a))
    kb = sorted((int(c), int(i), v) for c, i, v in zip(*b))
    assert ka == kb


def _link_image(cell, i, L, node, dirmap):
    x, y = int(cell) % L, int(cell) // L
    X, Y = node(x, y)
    return (Y % L) * L + (X % L), dirmap[int(i)]


def test_cut_links_rotate_with_the_polygon(orc):
    """A quarter turn of a generic polygon about a lattice node maps its cut links onto
    those of the turned polygon: destinations turned, directions E->N->W->S, NE->NW->SW->SE,
    the same coefficients (the crossing tests are exact integer arithmetic on snapped
    coordinates, which a quarter turn maps exactly)."""
    L = 40
    X = W.wobbly_polygon(17.3, 21.6, 8.0, 23, 0.3, 8)
    Fn = np.random.default_rng(9).uniform(-1, 1, 23)
    cfg = orc.make_cfg(L, L)
    a = orc.cut_links(cfg, X, Fn)
    Xr = np.stack([L - X[:, 1], X[:, 0]], axis=1)  # (x, y) -> (L - y, x), still CCW
    b = orc.cut_links(cfg, Xr, Fn)
    quarter = [0, 2, 3, 4, 1, 6, 7, 8, 5]
    ka = sorted(_link_image(c, i, L, lambda x, y: (L - y, x), quarter) + (v,)
                for c, i, v in zip(*a))
    kb = sorted((int(c), int(i), v) for c, i, v in zip(*b))
    assert len(ka) > 100 and ka == kb


def test_cut_links_mirror_with_the_polygon(orc):
    """The mirror image x -> L - x (marker order reversed to stay counter-clockwise, with
    its Fn) has the mirrored cut links: E <-> W, NE <-> NW, SW <-> SE, the same
    coefficients up to the rounding of the crossing parameter (t becomes 1 - t)."""
    L = 40
    X = W.wobbly_polygon(17.3, 21.6, 8.0, 23, 0.3, 10)
    Fn = np.random.default_rng(12).uniform(-1, 1, 23)
    cfg = orc.make_cfg(L, L)
    a = orc.cut_links(cfg, X, Fn)
    Xm = np.stack([L - X[:, 0], X[:, 1]], axis=1)[::-1].copy()
    b = orc.cut_links(cfg, Xm, Fn[::-1].copy())
    mirror = [0, 3, 2, 1, 4, 6, 5, 8, 7]
    ra = {}
    for c, i, v in zip(*a):
        k = _link_image(c, i, L, lambda x, y: (L - x, y), mirror)
        ra[k] = ra.get(k, 0.0) + v
    rb = {}
    for c, i, v in zip(*b):
        rb[(int(c), int(i))] = rb.get((int(c), int(i)), 0.0) + v
    assert len(ra) > 100 and set(ra) == set(rb)
    assert max(abs(ra[k] - rb[k]) for k in ra) < 1e-15


def test_jump_records_cancel_in_pairs(orc):
    """Each crossed link x - e_i -> x has its reverse x -> x - e_i crossed at the same
    point with the opposite sign and w_i = w_opp(i): the jump adds no mass."""
    X = W.wobbly_polygon(20.4, 19.7, 9.0, 40, 0.3, 11)
    Fn = np.random.default_rng(6).uniform(-1, 1, 40)
    cfg = orc.make_cfg(48, 48)
    cell, d, coef = orc.cut_links(cfg, X, Fn)
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    rec = {}
    for c, i, v in zip(cell, d, coef):
        rec.setdefault((int(c), int(i)), []).append(v)
    for (c, i), vs in rec.items():
        x, y = c % 48, c // 48
        src = ((y - E[i][1]) % 48) * 48 + (x - E[i][0]) % 48
        back = rec[(src, opp[i])]
        assert abs(sum(vs) + sum(back)) < 1e-15
    assert abs(coef.sum()) < 1e-13


# ----------------------------------------------------------- whole-step pins
@pytest.mark.parametrize("collision", ["srt", "mrt"])
def test_mass_is_conserved_with_the_jump(orc, collision):
    nx = ny = 40
    X = W.wobbly_polygon(20.2, 19.6, 9.0, 60, 0.15, 2)
    o = orc.Oracle(nx, ny, collision=orc.SRT if collision == "srt" else orc.MRT, tau=0.7,
                   s=W.mrt_rates(0.7))
    o.set_df(W.random_df(nx, ny, 1e-4, 9))
    m0 = o.get_df().sum()
    o.set_interface(X, model=orc.SPRING, kappa=0.05, dX=W.polygon_perimeter(X) / 60)
    o.step(25)
    assert abs(o.get_df().sum() - m0) < 1e-14


def _spline_points(orc, X, m):
    """The points X(k + j / m) of the periodic spline through the markers."""
    cx, cy = orc.spline_coeffs(X[:, 0]), orc.spline_coeffs(X[:, 1])
    s = np.arange(len(X) * m) / m
    return np.stack([[orc.spline_eval(cx, t) for t in s], [orc.spline_eval(cy, t) for t in s]], 1)


def _uniform_normal_force_case(orc, jump, init_exact, steps, curve=0):
    nx = ny = 40
    R, F = 10.0, -2e-3
    X = W.circle_markers(20.3, 19.8, R, 64)
    n = X - [20.3, 19.8]
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.8, s=W.mrt_rates(0.8), jump=jump)
    if init_exact:
        # f_i(x) = w_i rho(x); the stored state is the streamed part f_i - [[f_i]],
        # which for uniform Fn equals w_i rho(x - e_i).  rho_out - rho_in = Fn/c_s^2.
        # The interface is the polygon, or (curve = m) the polygon of the spline's points
        inside = np.array([[1 if (x - 20.3) ** 2 + (y - 19.8) ** 2 < (R - 1) ** 2 else 0
                            for x in range(nx)] for y in range(ny)])
        P = X if curve == 0 else _spline_points(orc, X, curve)
        wind = np.array([[orc.winding(P, x, y) for x in range(nx)] for y in range(ny)])
        assert np.all(wind[inside == 1] == 1)
        rho = 1.0 - wind * F * 3
        df = np.zeros((9, ny, nx))
        for i, (ex, ey) in enumerate(E):
            df[i] = float(WT[i]) * (np.roll(rho, (ey, ex), axis=(0, 1)) - 1.0)
        o.set_df(df)
    o.set_interface(X, model=orc.PRESCRIBED, moves=False, dX=W.polygon_perimeter(X) / 64,
                    G=F * n, curve=curve)
    o.step(steps)
    return o


@pytest.mark.parametrize("curve", [0, 4])
def test_uniform_normal_force_exact_fixed_point(orc, curve):
    """Section 4.1's exact solution u = 0 with a piecewise-constant pressure: with the
    jump of Eq. 32 on the cut links of the interface (the marker polygon, or the cubic
    spline through the markers taken on 4 chords per segment), the exact state is a
    fixed point of the II-LBM step (to rounding)."""
    o = _uniform_normal_force_case(orc, 1, True, 30, curve)
    r, ux, uy = o.step_macros()
    assert max(np.abs(ux).max(), np.abs(uy).max()) < 1e-16
    inside = r[20, 20]
    assert abs((inside - r[0, 0]) / 3 - 2e-3) < 1e-15  # [[p]] = Fn: p_in - p_out = -F


def test_uniform_normal_force_ii_beats_ib(orc):
    """Started from the exact solution (u = 0, piecewise-constant pressure), the II-LBM
    keeps it to rounding, while the IB-LBM (the same force spread by the delta kernel,
    no jump) cannot hold a sharp pressure jump and develops currents many orders of
    magnitude larger -- the contrast of section 4.1, Table 1."""
    ii = _uniform_normal_force_case(orc, 1, True, 200)
    ib = _uniform_normal_force_case(orc, 0, True, 200)
    _, ux, uy = ii.step_macros()
    e_ii = np.hypot(ux, uy).max()
    _, ux, uy = ib.step_macros()
    e_ib = np.hypot(ux, uy).max()
    assert e_ii < 1e-15 and e_ib > 1e-6


def test_laplace_law_membrane64(orc):
    """64^2 SRT membrane (R = 16, 128 markers, rest-length springs): once the slow
    breathing mode has decayed (6000 steps; at 2000 steps it still holds the ratio near
    0.92), the pressure jump c_s^2 (<rho>_in - <rho>_out), averaged over cells more than
    three lattice units from the polygon, matches Laplace's law T / R_c with the tension
    and circumradius measured at the end.  Area drift is small."""
    w = W.membrane_64()
    o = orc.Oracle(64, 64, collision=orc.SRT, tau=w["tau"])
    o.set_interface(w["X"], model=orc.SPRING_REST, kappa=w["kappa"], dX=w["dX"], l0=w["l0"])
    a0 = orc.polygon_area(w["X"])
    o.step(6000)
    m = o.markers()
    X = m["X"]
    r, _, _ = o.step_macros()
    c = X.mean(0)
    seg = np.linalg.norm(np.roll(X, -1, 0) - X, axis=1)
    T = w["kappa"] * (seg.mean() / w["l0"] - 1)
    Rc = seg.mean() / (2 * math.sin(math.pi / 128))
    yy, xx = np.mgrid[0:64, 0:64]
    d = np.hypot(xx - c[0], yy - c[1])
    dp = ((r[d < Rc - 3].mean() - r[d > Rc + 3].mean()) / 3)
    assert abs(dp / (T / Rc) - 1) < 2e-3
    assert abs(orc.polygon_area(X) / a0 - 1) < 1e-3


def test_translation_by_lattice_vector_shifts_fields_exactly(orc):
    """Shifting a moving membrane by a lattice vector shifts every field exactly.
    The polygon is snapped to a dyadic grid and the shift keeps every coordinate in
    the same binary exponent range, so each rounding is the same before and after."""
    nx = ny = 48
    X = W.wobbly_polygon(23.5, 23.7, 6.0, 44, 0.1, 4)
    X = np.round(X * 2 ** 20) / 2 ** 20
    assert X.min() > 16.5 and X.max() < 30.5
    outs = []
    for sh in ((0, 0), (1, 1)):
        o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.65, s=W.mrt_rates(0.65))
        o.set_interface(X + sh, model=orc.SPRING, kappa=0.05, dX=0.84)
        o.step(6)
        outs.append((o.get_df(), o.markers()["X"]))
    assert np.array_equal(np.roll(outs[0][0], (1, 1), axis=(1, 2)), outs[1][0])
    assert np.array_equal(outs[0][1] + 1, outs[1][1])


def _df_case(orc, iters, tol, jump=1, oracle=False, n=50):
    nx = ny = 48
    X = W.circle_markers(24.2, 23.9, 8.0, n)
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.8, s=W.mrt_rates(0.8), jump=jump)
    o.init_equilibrium(None, np.full(nx * ny, 0.02), None)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=W.polygon_perimeter(X) / n, eta=2.0,
                    mdf_iters=iters, mdf_tol=tol, UD=np.zeros((n, 2)))
    o.step(1)
    return o if oracle else o.mdf_stats()


@pytest.mark.parametrize("jump", [0, 1])
def test_direct_forcing_iteration_converges_to_no_slip(orc, jump):
    """Eq. 18 repeated: for a fixed cylinder in a uniform stream u = 0.02 the first pass
    sees the full slip 0.02, the residual max_k |U^D - U_k| then falls every pass (the
    IB form below 3% of the slip in 10 passes; the II-LBM form, whose passes carry the
    normal part through the jump, below 10%), and a run with a tolerance stops at the
    first pass below it."""
    it1, r1 = _df_case(orc, 1, 0.0, jump)
    assert it1 == 1 and abs(r1 - 0.02) < 1e-15
    res = [_df_case(orc, m, 0.0, jump)[1] for m in (2, 5, 10, 20)]
    assert all(a > b for a, b in zip([r1] + res, res))
    assert res[2] < (0.03 if jump == 0 else 0.1) * r1
    it, r = _df_case(orc, 200, 1e-3, jump)
    assert r < 1e-3 and 3 < it < (10 if jump == 0 else 20)


@pytest.mark.parametrize("jump", [0, 1])
def test_direct_forcing_meets_no_slip_in_the_collision_velocity(orc, jump):
    """The iteration interpolates the velocity the step's collision will use: once it
    stops below the tolerance, the velocity the oracle then interpolates at the markers
    from the collision's own fields (u of Eq. 24 with the jump on the cut links and the
    spread tangential force, the U of the step) meets the no-slip condition within that
    tolerance, in II-LBM as in IB-LBM.  (An iteration that spread the whole G and then
    moved its normal part into the jump would leave a slip of the order of the jump's
    effect here.)  Markers 1.5 apart, where the iteration reaches 1e-7."""
    o = _df_case(orc, 400, 1e-7, jump, oracle=True, n=34)
    it, r = o.mdf_stats()
    assert r < 1e-7 and it < 400
    U = o.markers()["U"]  # interpolated from the collision velocity of the step
    assert np.abs(U).max() < 1e-7


@pytest.mark.slow
def test_rigid_cylinder_channel_stays_bounded_at_re100(orc):
    """The cylinder channel at Re 100 (reduced replica: 512 x 128, D = 20, u_max 0.05,
    tau = 0.53 from Re, MRT, normal force through the jump, five force updates a step),
    impulsively started from the parabolic profile: 1000 steps stay bounded (|u| below
    3 u_max, |rho - rho0| below 0.15; the coupling that spread the whole G in the
    passes reached |u| 0.39 and |rho - rho0| 0.97 by step 250), the force iteration
    keeps the slip near 1e-4 of
    the stream, and the drag is positive.  The paper runs its II-LBM cylinder at Re 100
    and 200 stably (section 4.3)."""
    try:
        orc.lib(parallel=True)
        par = True
    except RuntimeError:
        par = False
    w = W.cylinder_channel(100.0, nx=512, ny=128, D=20.0, cx=128.0, cy=64.5, n=63)
    nx, ny = w["nx"], w["ny"]
    o = orc.Oracle(nx, ny, parallel=par, collision=orc.MRT, tau=w["tau"],
                   s=W.mrt_rates(w["tau"]), bc=orc.BC_CHANNEL, u_max=w["u_max"])
    y = np.arange(ny) + 0.5
    o.init_equilibrium(None, np.repeat((4 * 0.05 * y * (ny - y) / ny ** 2)[:, None], nx, axis=1),
                       None)
    o.set_interface(w["X"], model=orc.DIRECT, moves=False, dX=w["dX"], eta=2.0, mdf_iters=5,
                    UD=np.zeros((63, 2)))
    for _ in range(4):
        o.step(250)
        r, ux, uy = o.step_macros(deviation=True)
        assert np.isfinite(ux).all() and np.abs(ux).max() < 0.15 and np.abs(uy).max() < 0.15
        assert np.abs(r).max() < 0.15
        _, res = o.mdf_stats()
        assert res < 5e-3
    assert res < 2e-4
    Fx = -o.markers()["G"][:, 0].sum() * w["dX"]
    assert Fx > 0


# ------------------------------------------------------------ spline interface
def test_spline_interpolates_and_solves_its_system(orc):
    """The periodic spline passes through every value (v(k) = v_k), its coefficients
    satisfy the defining cyclic system (c_{k-1} + 4 c_k + c_{k+1}) / 6 = v_k, and it
    has period n."""
    for n in (3, 4, 7, 64):
        v = np.random.default_rng(n).normal(size=n)
        c = orc.spline_coeffs(v)
        assert np.allclose((np.roll(c, 1) + 4 * c + np.roll(c, -1)) / 6, v, rtol=0, atol=1e-14)
        assert max(abs(orc.spline_eval(c, k) - v[k]) for k in range(n)) < 1e-14
        for s in (0.3, 1.7):
            assert abs(orc.spline_eval(c, s) - orc.spline_eval(c, s + n)) < 1e-13


def test_spline_converges_at_fourth_order(orc):
    """For samples of a smooth periodic function the spline between the samples (at
    half-integer parameters) and its derivative converge at least at the cubic spline's
    orders on refinement: value error ~h^4, derivative error ~h^3 (at the half-integers
    of a uniform periodic spline the derivative is superconvergent, ~h^4)."""
    ev, ed = [], []
    for n in (16, 32, 64):
        k = np.arange(n)
        f = lambda t: np.sin(2 * np.pi * t / n) + 0.5 * np.cos(4 * np.pi * t / n)
        df = lambda t: (2 * np.pi / n) * (np.cos(2 * np.pi * t / n)
                                          - np.sin(4 * np.pi * t / n))
        c = orc.spline_coeffs(f(k))
        s = k + 0.5
        ev.append(max(abs(orc.spline_eval(c, t) - f(t)) for t in s))
        ed.append(max(abs(orc.spline_eval(c, t, 1) / (2 * np.pi / n)
                          - df(t) / (2 * np.pi / n)) for t in s))
    for e, order in ((ev, 4), (ed, 3)):
        rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
        assert all(r > order - 0.3 for r in rates), (e, rates)
    assert ev[-1] < 1e-5 and ed[-1] < 1e-4


def test_spline_normals_of_an_ellipse_converge_faster_than_the_polygons(orc):
    """Markers equally spaced in arc length on an ellipse: the normal split's normals
    from the spline tangent approach the ellipse's exact normals at the markers at
    fourth order; the polygon's central difference only at second order.  (Equal steps
    in the ellipse's angle parameter would make the central difference exactly tangent,
    so the markers follow arc length.)"""
    errs = {0: [], 1: []}
    for n in (32, 64, 128):
        a, b = 20.0, 11.0
        X = W.ellipse_markers(0.0, 0.0, a, b, n)
        nex = np.stack([X[:, 0] / a ** 2, X[:, 1] / b ** 2], 1)
        nex /= np.linalg.norm(nex, axis=1, keepdims=True)
        for curve in (0, 1):
            _, _, nrm = orc.normal_split(X, np.zeros((n, 2)), True, 1.0, curve=curve)
            errs[curve].append(np.abs(nrm - nex).max())
    r_poly = np.log2(errs[0][-2] / errs[0][-1])
    r_spl = np.log2(errs[1][-2] / errs[1][-1])
    assert abs(r_poly - 2) < 0.3 and abs(r_spl - 4) < 0.4, (errs, r_poly, r_spl)
    assert errs[1][-1] < 0.01 * errs[0][-1]


def test_spline_cut_links_follow_the_curve(orc):
    """The cut links of the spline interface (8 chords per segment) of a circle sampled
    by 40 markers: every link whose ends lie on opposite sides of the exact circle by
    more than the spline's distance from it carries one record, signed by the side of
    its source (interior to exterior +1), and no link with both ends on one side does;
    a constant Fn gives s w_i/c_s^2 Fn exactly."""
    nx = ny = 48
    c0, R, n, Fn = np.array([23.6, 24.3]), 11.2, 40, -1.5e-3
    X = W.circle_markers(c0[0], c0[1], R, n)
    cfg = orc.make_cfg(nx, ny)
    cell, d, coef = orc.cut_links_spline(cfg, X, np.full(n, Fn), 8)
    P = _spline_points(orc, X, 8)
    dev = np.abs(np.linalg.norm(P - c0, axis=1) - R).max()
    assert dev < 2e-4  # the spline hugs the circle (the polygon is 0.03 inside it)
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    WT = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    rec = {}
    for cl, i, cf in zip(cell, d, coef):
        rec.setdefault((int(cl), int(i)), []).append(cf)
    margin = 3 * dev + 1e-9
    for y in range(ny):
        for x in range(nx):
            r1 = np.hypot(x - c0[0], y - c0[1]) - R
            for i in range(1, 9):
                xs, ys = x - E[i][0], y - E[i][1]
                r0 = np.hypot(xs - c0[0], ys - c0[1]) - R
                key = (y * nx + x, i)
                if r0 < -margin and r1 > margin:
                    assert len(rec.get(key, [])) == 1
                    assert abs(rec[key][0] - 3 * WT[i] * Fn) < 1e-14 * abs(Fn)
                elif r0 > margin and r1 < -margin:
                    assert len(rec.get(key, [])) == 1
                    assert abs(rec[key][0] + 3 * WT[i] * Fn) < 1e-14 * abs(Fn)
                elif (r0 > margin and r1 > margin) or (r0 < -margin and r1 < -margin):
                    assert key not in rec


# ---------------------------------------------------------------- rigid bodies
def _body_case(orc, mode, jump=0, dof=3, u0=0.01, D=10.0, n=32, rho_s=2.0, steps=0):
    nx = ny = 48
    X = W.circle_markers(23.7, 24.2, D / 2, n)
    dX = W.polygon_perimeter(X) / n
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=0.8, s=W.mrt_rates(0.8), jump=jump)
    o.init_equilibrium(None, np.full(nx * ny, u0), None)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=5,
                    UD=np.zeros((n, 2)))
    Vs = np.pi * D * D / 4
    m = rho_s * Vs
    o.set_body(mode, dof=dof, A=3.0, umax=0.02, mass=m, inertia=m * D * D / 8, volume=Vs)
    o.step(steps)
    return o, X, m, Vs


def _fluid_momentum(o):
    df = o.get_df()
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    return np.array([sum(e[0] * df[i].sum() for i, e in enumerate(E)),
                     sum(e[1] * df[i].sum() for i, e in enumerate(E))])


def test_free_body_conserves_momentum_with_the_fluid(orc):
    """A free rigid body (section 2.3) in a periodic box with a uniform stream, the whole
    force spread (IB form): the fluid gains exactly sum_k G_k dX each step (the delta
    kernel's partition of unity; Guo's term adds exactly g), and the body's Eq. 25 (with
    its internal-fluid inertia term) and Eqs. 27-29 then make
        Q(t) = P_fluid(t) + m U_c(t) - rho_f V_s U_c(t - 1)
    constant to rounding.  A sign error in the force, or a missing or misplaced inertia
    term, breaks it.  The stream drags the body along (U_x > 0).  Density ratio 10: the
    explicit inertia term of Eq. 25 lets light bodies oscillate unstably (this IB form at
    rho_s / rho_f <= 2.55, the II-LBM form at 1.5 but not at 2.55)."""
    o, X, m, Vs = _body_case(orc, orc.BODY_FREE, rho_s=10.0)
    Q0 = _fluid_momentum(o)
    Ucp = np.zeros(2)
    for _ in range(60):
        o.step(1)
        Uc = o.body()[3:5]
        Q = _fluid_momentum(o) + m * Uc - Vs * Ucp
        assert np.abs(Q - Q0).max() < 1e-13 * np.abs(Q0).max()
        Ucp = Uc
    assert Uc[0] > 1e-5 and abs(Uc[1]) < 1e-3 * Uc[0]


def test_prescribed_translation_moves_the_markers_rigidly(orc):
    """Section 4.4's prescribed harmonic translation: after t steps the centre sits at
    X_c0 - A sin(U_max t / A), every marker keeps its offset from the centre exactly, and
    the body's velocity is -U_max cos(U_max t / A)."""
    o, X, _, _ = _body_case(orc, orc.BODY_PRESCRIBED_X, jump=1, u0=0.0)
    c0 = X.mean(0)
    T = 38
    o.step(T)
    b = o.body()
    A, um = 3.0, 0.02
    assert abs(b[0] - (c0[0] - A * np.sin(um * T / A))) < 1e-12
    assert abs(b[3] + um * np.cos(um * T / A)) < 1e-15 and b[1] == c0[1]
    Xt = o.markers()["X"]
    assert np.abs((Xt - b[:2]) - (X - c0)).max() < 1e-12


def test_free_body_at_the_papers_density_ratio_is_stable(orc):
    """At the density ratio of section 4.5 (8 / pi) a free body carried by a stream in the
    II-LBM settles into a smooth drift (no growing oscillation of its velocity over 300
    steps)."""
    o, _, _, _ = _body_case(orc, orc.BODY_FREE, jump=1, rho_s=8 / np.pi)
    u = []
    for _ in range(300):
        o.step(1)
        u.append(o.body()[3])
    u = np.array(u)
    assert np.all(np.isfinite(u)) and 0 < u[-1] < 0.02
    assert np.abs(np.diff(u[-100:])).max() < 1e-4


def test_free_body_at_rest_stays_at_rest(orc):
    """A free body in fluid at rest feels no force: it, and the fluid, stay at rest."""
    o, X, _, _ = _body_case(orc, orc.BODY_FREE, jump=1, u0=0.0, dof=7, steps=40)
    b = o.body()
    assert np.abs(b[3:9]).max() == 0.0 and np.abs(o.markers()["X"] - X).max() == 0.0
    assert np.abs(o.get_df()).max() == 0.0
