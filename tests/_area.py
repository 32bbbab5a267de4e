"""Enclosed area of a closed interface, for the area-loss comparison of section 4.2.

The polygon through the markers is the IB-LBM's interface; the II-LBM's is the periodic
cubic spline through them (end of section 3.2).  Markers two lattice units apart on a
curve of radius 20 cut its area by about 1e-3 as a polygon, and that cut changes as an
ellipse relaxes to a circle, so the comparison measures every method on the spline.
"""
import numpy as np


def polygon_area(X):
    """Shoelace area of the closed polygon X[n][2] (positive counter-clockwise)."""
    x, y = X[:, 0], X[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def spline_area(X):
    """Area enclosed by the periodic interpolating cubic spline through X[n][2],
    parametrised by the marker index: (c_{k-1} + 4 c_k + c_{k+1}) / 6 = X_k for its
    uniform B-spline coefficients, then 1/2 * integral of (x y' - y x') ds, a degree-5
    polynomial on each segment, exact with 3-point Gauss-Legendre quadrature."""
    X = np.asarray(X, dtype=np.float64)
    n = len(X)
    M = np.zeros((n, n))
    idx = np.arange(n)
    M[idx, (idx - 1) % n] += 1.0 / 6
    M[idx, idx] += 4.0 / 6
    M[idx, (idx + 1) % n] += 1.0 / 6
    c = np.linalg.solve(M, X)
    nodes = 0.5 + 0.5 * np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    weights = np.array([5.0, 8.0, 5.0]) / 18.0
    total = 0.0
    for t, w in zip(nodes, weights):
        u = 1.0 - t
        b = (u ** 3 / 6, (3 * t ** 3 - 6 * t ** 2 + 4) / 6, (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6,
             t ** 3 / 6)
        d = (-0.5 * u * u, 1.5 * t * t - 2 * t, -1.5 * t * t + t + 0.5, 0.5 * t * t)
        P = sum(b[j] * c[(idx - 1 + j) % n] for j in range(4))
        D = sum(d[j] * c[(idx - 1 + j) % n] for j in range(4))
        total += w * float(np.sum(P[:, 0] * D[:, 1] - P[:, 1] * D[:, 0]))
    return 0.5 * total
