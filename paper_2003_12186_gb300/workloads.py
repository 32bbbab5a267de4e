"""Seeded synthetic inputs (marker polygons, lattice parameters, perturbed states).

This module builds inputs only: shapes, sizes, rates and seeds of the workloads the
paper's section 4 experiments are shaped like.  It holds none of the method's
arithmetic and imports neither the CUDA library nor the CPU oracle, so both sides
can draw identical inputs from it.

All marker polygons are closed, counter-clockwise, returned as float64 [n, 2] arrays
in lattice units (node (i, j) sits at coordinate (i, j)).
"""
from __future__ import annotations

import math

import numpy as np

# Lallemand-Luo D2Q9 rates quoted in section 2.2.1 of the paper; s7 = s8 = 1/tau.
PAPER_MRT_RATES = (0.0, 1.63, 1.14, 0.0, 1.92, 0.0, 1.92)


def mrt_rates(tau: float) -> list:
    return list(PAPER_MRT_RATES) + [1.0 / tau, 1.0 / tau]


def circle_markers(cx: float, cy: float, R: float, n: int, phase: float = 0.0) -> np.ndarray:
    th = phase + 2.0 * np.pi * np.arange(n) / n
    return np.stack([cx + R * np.cos(th), cy + R * np.sin(th)], axis=1)


def ellipse_markers(cx: float, cy: float, a: float, b: float, n: int,
                    angle: float = 0.0) -> np.ndarray:
    """n markers equally spaced in arc length on an ellipse (semi-axes a, b)."""
    m = max(64 * n, 4096)
    t = np.linspace(0.0, 2.0 * np.pi, m + 1)
    px, py = a * np.cos(t), b * np.sin(t)
    seg = np.hypot(np.diff(px), np.diff(py))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    targets = s[-1] * np.arange(n) / n
    tt = np.interp(targets, s, t)
    x, y = a * np.cos(tt), b * np.sin(tt)
    ca, sa = math.cos(angle), math.sin(angle)
    return np.stack([cx + ca * x - sa * y, cy + sa * x + ca * y], axis=1)


def polygon_perimeter(X: np.ndarray) -> float:
    d = np.roll(X, -1, axis=0) - X
    return float(np.hypot(d[:, 0], d[:, 1]).sum())


def ramanujan_perimeter(a: float, b: float) -> float:
    return math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))


def random_df(nx: int, ny: int, amp: float, seed: int) -> np.ndarray:
    """Random shifted populations df[9, ny, nx] of amplitude amp (a perturbed state)."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((9, ny, nx))


def wobbly_polygon(cx: float, cy: float, R: float, n: int, amp: float, seed: int) -> np.ndarray:
    """A star-shaped CCW polygon with random radial wobble (generic positions)."""
    rng = np.random.default_rng(seed)
    th = 2.0 * np.pi * (np.arange(n) + 0.3 * rng.uniform(-1, 1, n)) / n
    th = np.sort(th)
    r = R * (1.0 + amp * rng.uniform(-1, 1, n))
    return np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], axis=1)


# ------------------------------------------------------------------ workloads
def membrane_64():
    """64x64 periodic SRT membrane: circle R=16 at the centre, 128 markers, linear
    rest-length springs (stiffness 0.01, rest length 0.9 x the initial segment)."""
    X = circle_markers(32.0, 32.0, 16.0, 128)
    seg = 2 * 16.0 * math.sin(math.pi / 128)
    return dict(name="membrane64_srt_f64", nx=64, ny=64, collision="srt", tau=0.8,
                storage="f64", X=X, model="spring_rest", kappa=0.01, dX=seg, l0=0.9 * seg,
                steps=2000)


def ellipse_2048(storage: str = "f32"):
    """2048^2 periodic MRT membrane: ellipse a=400, b=250 centred, 2048 markers equally
    spaced in arc length, zero-rest-length springs (Eq. 19) of stiffness 0.05, tau 0.6."""
    X = ellipse_markers(1024.0, 1024.0, 400.0, 250.0, 2048)
    return dict(name=f"ellipse2048_mrt_{storage}", nx=2048, ny=2048, collision="mrt", tau=0.6,
                storage=storage, X=X, model="spring", kappa=0.05,
                dX=polygon_perimeter(X) / 2048, l0=0.0, steps=20000)


def ellipse_scaled(n: int, storage: str = "f32", markers: int | None = None):
    """The 2048^2 ellipse membrane scaled to an n x n lattice (same aspect, same tau)."""
    s = n / 2048.0
    nm = markers or max(32, int(round(2048 * s)))
    X = ellipse_markers(n / 2.0, n / 2.0, 400.0 * s, 250.0 * s, nm)
    return dict(name=f"ellipse{n}_mrt_{storage}", nx=n, ny=n, collision="mrt", tau=0.6,
                storage=storage, X=X, model="spring", kappa=0.05,
                dX=polygon_perimeter(X) / nm, l0=0.0)


def cylinder_channel(re: float = 100.0, nx: int = 1024, ny: int = 256, D: float = 40.0,
                     cx: float = 256.0, cy: float = 128.5, n: int = 126, u_max: float = 0.05):
    """Rigid cylinder in a channel with a parabolic inflow; tau from Re = u_max D / nu."""
    nu = u_max * D / re
    tau = 0.5 + 3.0 * nu
    X = circle_markers(cx, cy, D / 2.0, n)
    return dict(name=f"cylinder{nx}x{ny}_re{re:g}", nx=nx, ny=ny, collision="mrt", tau=tau,
                storage="f32", X=X, model="direct", u_max=u_max, D=D,
                dX=polygon_perimeter(X) / n, steps=50000)


def batched_membranes(count: int = 256, seed: int = 0):
    """Independent membrane lattices of uneven size: n in {64..512}, ellipse aspect in
    [1, 2.5], perimeter 0.6 n, one marker per 0.5 lattice unit, stiffness log-uniform
    in [1e-3, 1e-1], tau uniform in [0.55, 1.0]."""
    rng = np.random.default_rng(seed)
    sizes = (64, 96, 128, 192, 256, 384, 512)
    sims = []
    for k in range(count):
        n = int(sizes[rng.integers(len(sizes))])
        asp = float(rng.uniform(1.0, 2.5))
        kappa = float(10 ** rng.uniform(-3, -1))
        tau = float(rng.uniform(0.55, 1.0))
        per = 0.6 * n
        b = per / ramanujan_perimeter(asp, 1.0)
        a = asp * b
        nm = int(round(per / 0.5))
        X = ellipse_markers(n / 2.0, n / 2.0, a, b, nm)
        sims.append(dict(nx=n, ny=n, tau=tau, kappa=kappa, X=X,
                         dX=polygon_perimeter(X) / nm))
    return sims


# ------------------------------------------------------------- learned warm start
MLP_SHAPES = [((64, 30), True), ((64,), False), ((64, 64), True), ((64,), False),
              ((64, 64), True), ((64,), False), ((2, 64), True), ((2,), False)]


def mlp_init_params(seed: int) -> np.ndarray:
    """Initial parameters of the 30-64-64-64-2 network in its packed order (W1, b1, W2,
    b2, W3, b3, W4, b4; weights [out][in]): weights uniform in +-sqrt(6 / fan_in)
    (+-sqrt(3 / fan_in) for the output layer), biases zero; FP32 values."""
    rng = np.random.default_rng(seed)
    parts = []
    for q, (shape, is_w) in enumerate(MLP_SHAPES):
        if is_w:
            bound = np.sqrt((3.0 if q == 6 else 6.0) / shape[1])
            parts.append(rng.uniform(-bound, bound, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


def learned_channels(count: int = 64, seed: int = 0, nx: int = 512, ny: int = 128,
                     spacing: float = 1.5, u_max: float = 0.05):
    """Rigid-cylinder channels of the learned warm start: D uniform in [16, 32], centre x
    uniform in [96, 160], y = ny/2 + uniform(-4, 4), Re uniform in [10, 150] (tau from
    Re with u_max), markers every `spacing` lattice units along the circle."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        D = float(rng.uniform(16.0, 32.0))
        xc = float(rng.uniform(96.0, 160.0))
        yc = ny / 2.0 + float(rng.uniform(-4.0, 4.0))
        re = float(rng.uniform(10.0, 150.0))
        n = int(round(np.pi * D / spacing))
        X = circle_markers(xc, yc, D / 2.0, n, phase=float(rng.uniform(0.0, 2.0 * np.pi / n)))
        out.append(dict(nx=nx, ny=ny, D=D, xc=xc, yc=yc, re=re, n=n, X=X, u_max=u_max,
                        tau=0.5 + 3.0 * u_max * D / re, dX=polygon_perimeter(X) / n))
    return out


# ------------------------------------------------------------ three dimensions
# Closed triangulated surfaces for the D3Q19 lattice: vertices float64 [n, 3] in lattice
# units, triangles int32 [m, 3] ordered counter-clockwise seen from outside.

def d3q19_rates(tau: float) -> list:
    """The D3Q19 MRT rates of section 2.2.1 (d'Humieres moment order): s1 = 1.19,
    s2 = s10 = s12 = 1.4, s4 = s6 = s8 = 1.2, s9 = s11 = s13..s15 = 1/tau,
    s16..s18 = 1.98; the conserved moments' rates 0."""
    s = [0.0] * 19
    s[1] = 1.19
    s[2] = s[10] = s[12] = 1.4
    s[4] = s[6] = s[8] = 1.2
    s[9] = s[11] = s[13] = s[14] = s[15] = 1.0 / tau
    s[16] = s[17] = s[18] = 1.98
    return s


def icosphere(level: int):
    """Unit sphere: the icosahedron with each triangle split into four `level` times,
    new vertices pushed out to the sphere.  Returns (vertices [n, 3], triangles [m, 3]),
    10 * 4**level + 2 vertices."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[key] = len(V) - 1
            return mid[key]

        G = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            G += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = G
    X = np.array(V)
    T = np.array(F, np.int32)
    # orient every triangle outward (its normal along its centroid)
    A, B, C = X[T[:, 0]], X[T[:, 1]], X[T[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(B - A, C - A), A + B + C) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return X, T


def ellipsoid_surface(centre, axes, level: int, seed: int | None = None):
    """An icosphere scaled to the semi-axes (a, b, c) and moved to centre; with a seed,
    turned by a random rotation first (generic position against the lattice)."""
    X, T = icosphere(level)
    X = X * np.asarray(axes, float)
    if seed is not None:
        rng = np.random.default_rng(seed)
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q * np.sign(np.diag(r))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        X = X @ q.T
    return X + np.asarray(centre, float), T


def random_df3(nx: int, ny: int, nz: int, amp: float, seed: int) -> np.ndarray:
    """Random shifted D3Q19 populations df[19, nz, ny, nx] of amplitude amp."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((19, nz, ny, nx))


def membrane_3d(n: int = 256, seed: int = 17):
    """The three-dimensional membrane workload: an n^3 periodic D3Q19 box (MRT, tau 0.6)
    holding a surface-tension ellipsoid with semi-axes 0.31 n, 0.25 n, 0.22 n at the box's
    centre (offset from the nodes), turned by a seeded rotation, triangulated so that its
    edges are about one lattice unit (icosphere level 6 at n = 256, 40 962 vertices), at
    rest; gamma = 1e-3 lattice units."""
    level = max(3, int(round(math.log2(n / 256.0))) + 6)
    c = (n / 2 + 0.37, n / 2 + 0.21, n / 2 + 0.13)
    X, T = ellipsoid_surface(c, (0.31 * n, 0.25 * n, 0.22 * n), level, seed=seed)
    return {"name": f"membrane3d_{n}", "n": n, "X": X, "T": T, "tau": 0.6, "gamma": 1e-3,
            "level": level}
