"""Pins of the learned warm start's oracle (oracle/mlp.py): values the definitions fix,
finite differences for every derivative, closed forms of the optimiser and geometry."""

import numpy as np
import pytest

from oracle import mlp as M
from paper_2003_12186_gb300 import workloads as W

PHI1 = 0.8413447460685429  # standard normal distribution function at 1


def norm_ident():
    return dict(in_mean=np.zeros(30), in_istd=np.ones(30), out_mean=np.zeros(2),
                out_scale=np.ones(2))


def test_parameter_count_and_layout():
    assert M.N_PARAMS == 10434
    theta = np.arange(M.N_PARAMS, dtype=np.float64)
    p = M.unpack(theta)
    assert p["W1"].shape == (64, 30) and p["W1"][1, 0] == 30  # [out][in], row major
    assert p["b4"][-1] == M.N_PARAMS - 1
    assert np.array_equal(M.pack(p), theta)
    assert W.mlp_init_params(0).size == M.N_PARAMS


def test_gelu_values():
    assert M.gelu(0.0) == 0.0
    assert abs(M.gelu(1.0) - PHI1) < 1e-15
    assert abs(M.gelu(-1.0) + (1.0 - PHI1)) < 1e-15
    assert abs(M.gelu(8.0) - 8.0) < 1e-12 and abs(M.gelu(-8.0)) < 1e-12
    assert abs(M.gelu_prime(0.0) - 0.5) < 1e-15


def test_gelu_prime_against_finite_differences():
    z = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.abs(fd - M.gelu_prime(z)).max() < 1e-8


@pytest.fixture(scope="module")
def small_problem():
    rng = np.random.default_rng(7)
    theta = W.mlp_init_params(3).astype(np.float64)
    theta += rng.normal(0, 0.05, theta.size)  # nonzero biases too
    X = rng.normal(0, 1, (7, 30))
    T = rng.normal(0, 1, (7, 2))
    norm = dict(in_mean=rng.normal(0, 0.1, 30), in_istd=rng.uniform(0.5, 2.0, 30),
                out_mean=rng.normal(0, 0.1, 2), out_scale=rng.uniform(0.5, 2.0, 2))
    return theta, X, T, norm


def test_gradient_against_finite_differences(small_problem):
    """Central differences on every bias and weight of the output layer and on 300
    weights drawn from the hidden layers: relative agreement within 1e-6."""
    theta, X, T, norm = small_problem
    L, g = M.loss_and_grad(theta, X, T, norm)
    rng = np.random.default_rng(1)
    idx = np.concatenate([np.arange(M.N_PARAMS - 130, M.N_PARAMS),  # W4, b4
                          np.arange(1920, 1984),                     # b1
                          rng.choice(M.N_PARAMS - 130, 300, replace=False)])
    h = 1e-6
    scale = np.abs(g).max()
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (M.loss_and_grad(theta + e, X, T, norm)[0] -
              M.loss_and_grad(theta - e, X, T, norm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * scale), i


def test_loss_of_a_constant_network(small_problem):
    """W4 = 0: the output is b4 for every input, the loss and its b4-gradient are the
    mean squared / mean error of the normalised targets."""
    theta, X, T, norm = small_problem
    p = M.unpack(theta.copy())
    p["W4"][:] = 0.0
    p["b4"][:] = [0.3, -0.2]
    th = M.pack(p)
    G, _ = M.forward(th, X, norm)
    assert np.allclose(G, np.array([0.3, -0.2]) * norm["out_scale"] + norm["out_mean"])
    t = (T - norm["out_mean"]) / norm["out_scale"]
    e = np.array([0.3, -0.2]) - t
    L, g = M.loss_and_grad(th, X, T, norm)
    assert abs(L - np.mean(e * e)) < 1e-14
    assert np.allclose(g[-2:], e.sum(0) / X.shape[0], atol=1e-14)


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    new, m, v = M.adam_step(theta, np.zeros(50), np.zeros(50), g, 1, lr=1e-3)
    # bias correction makes the first moments g and g^2: the step is lr g / (|g| + eps),
    # within lr eps / |g| of lr sign(g)
    assert np.all(np.abs((new - theta) + 1e-3 * np.sign(g)) <= 1e-3 * 1e-8 / np.abs(g) * 1.001)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_of_a_regular_polygon():
    """Regular n-gon of circumradius R: normals are radial and the discrete curvature is
    1/R exactly; the blocks are ordered k-2 .. k+2."""
    R, n, c = 11.0, 40, np.array([50.0, 30.0])
    X = W.circle_markers(c[0], c[1], R, n)
    dX = W.polygon_perimeter(X) / n
    nrm, kappa = M.marker_geometry(X, dX)
    radial = (X - c) / R
    assert np.abs(nrm - radial).max() < 1e-13
    assert np.abs(kappa - 1.0 / R).max() < 1e-12
    Us = np.arange(2 * n, dtype=float).reshape(n, 2)
    F = M.features(X, Us, np.zeros((n, 2)), dX, 42.0)
    assert F.shape == (n, 30)
    k = 5
    for q, j in enumerate(range(k - 2, k + 3)):
        assert np.array_equal(F[k, 6 * q:6 * q + 2], -Us[j % n])
        assert np.allclose(F[k, 6 * q + 2:6 * q + 4], nrm[j % n])
        assert F[k, 6 * q + 5] == 42.0
    assert np.array_equal(F[0, 0:2], -Us[n - 2])  # cyclic
