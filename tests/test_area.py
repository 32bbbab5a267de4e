"""Pins of the area measures used by the area-loss comparison (section 4.2)."""
import numpy as np
import pytest

from paper_2003_12186_gb300 import workloads as W

from _area import polygon_area, spline_area


def test_spline_area_equals_scipys_periodic_spline():
    """The periodic C2 cubic interpolant through given points is unique, so scipy's
    CubicSpline (periodic, same index parametrisation) must enclose the same area;
    integrated there with its own antiderivative of x y' - y x'."""
    interpolate = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(5)
    n = 23
    th = 2 * np.pi * np.arange(n) / n
    r = 10 + rng.uniform(-1.5, 1.5, n)
    X = np.stack([3.1 + r * np.cos(th), -2.4 + r * np.sin(th)], axis=1)
    s = np.arange(n + 1, dtype=np.float64)
    sx = interpolate.CubicSpline(s, np.append(X[:, 0], X[0, 0]), bc_type="periodic")
    sy = interpolate.CubicSpline(s, np.append(X[:, 1], X[0, 1]), bc_type="periodic")
    ss = np.linspace(0, n, 200 * n + 1)
    f = sx(ss) * sy(ss, 1) - sy(ss) * sx(ss, 1)
    ref = 0.5 * float(np.sum((f[1:] + f[:-1]) * 0.5 * np.diff(ss)))  # trapezoid, h = 1/200
    ss2 = np.linspace(0, n, 400 * n + 1)
    f2 = sx(ss2) * sy(ss2, 1) - sy(ss2) * sx(ss2, 1)
    ref_fine = 0.5 * float(np.sum((f2[1:] + f2[:-1]) * 0.5 * np.diff(ss2)))
    ref = ref_fine + (ref_fine - ref) / 3  # Richardson: the trapezoid's h^2 term removed
    assert abs(spline_area(X) - ref) < 1e-9 * abs(ref)


def test_spline_area_of_a_circle_converges_at_fourth_order():
    R = 20.0
    errs = [abs(spline_area(W.circle_markers(40.13, 40.07, R, n)) / (np.pi * R * R) - 1)
            for n in (16, 32, 64)]
    assert errs[2] < 1e-6
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20
    # the polygon's deficit is second order and far larger
    p = abs(polygon_area(W.circle_markers(40.13, 40.07, R, 64)) / (np.pi * R * R) - 1)
    assert p > 1000 * errs[2]


def test_spline_area_orientation_and_translation():
    X = W.ellipse_markers(30.0, 25.0, 12.0, 7.0, 40)
    a = spline_area(X)
    assert a > 0 and abs(spline_area(X[::-1]) + a) < 1e-12 * a
    assert abs(spline_area(X + np.array([117.25, -33.5])) - a) < 1e-11 * a
