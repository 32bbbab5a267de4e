"""Learned warm start on the GPU: the network's forward pass, its gradient and Adam steps
against the FP64 oracle (oracle/mlp.py), the features the library forms from a force
iteration, and the network's proposal as the start of direct forcing."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2003_12186_gb300 import iilbm
from paper_2003_12186_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    iilbm.load()


def problem(seed, N=200):
    rng = np.random.default_rng(seed)
    theta = W.mlp_init_params(seed).astype(np.float64) + rng.normal(0, 0.05, M.N_PARAMS)
    theta = theta.astype(np.float32)
    X = rng.normal(0, 1, (N, 30)).astype(np.float32)
    T = rng.normal(0, 1, (N, 2)).astype(np.float32)
    norm = dict(in_mean=rng.normal(0, 0.1, 30).astype(np.float32),
                in_istd=rng.uniform(0.5, 2.0, 30).astype(np.float32),
                out_mean=rng.normal(0, 0.1, 2).astype(np.float32),
                out_scale=rng.uniform(0.5, 2.0, 2).astype(np.float32))
    return theta, X, T, norm


def network(theta, norm):
    m = iilbm.Mlp(theta)
    m.iilbm_mlp_set_normalization(norm["in_mean"], norm["in_istd"], norm["out_mean"],
                                  norm["out_scale"])
    return m


def as64(norm):
    return {k: v.astype(np.float64) for k, v in norm.items()}


def test_forward_matches_oracle():
    theta, X, _, norm = problem(1, N=333)  # a ragged last block of samples
    m = network(theta, norm)
    Y = m.forward(X)
    G, _ = M.forward(theta.astype(np.float64), X.astype(np.float64), as64(norm))
    assert np.abs(Y - G).max() <= 1e-5 * np.abs(G).max()


def test_gradient_matches_oracle():
    theta, X, T, norm = problem(2)
    m = network(theta, norm)
    loss, g = m.gradient(X, T)
    Lo, go = M.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                             T.astype(np.float64), as64(norm))
    assert abs(loss - Lo) <= 1e-5 * Lo
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()
    # every layer's block, not just the largest entries
    o = 0
    for name, shape in M.SHAPES:
        size = int(np.prod(shape))
        blk, blko = g[o:o + size], go[o:o + size]
        assert np.abs(blk - blko).max() <= 1e-4 * max(np.abs(blko).max(), 1e-12), name
        o += size


def test_adam_steps_follow_the_oracle():
    theta, X, T, norm = problem(3)
    m = network(theta, norm)
    rng = np.random.default_rng(4)
    order = np.concatenate([rng.permutation(200)[:64] for _ in range(3)]).astype(np.int32)
    losses = m.train(X, T, order, batch=64, lr=1e-3)
    th = theta.astype(np.float64)
    mo, vo = np.zeros_like(th), np.zeros_like(th)
    for s in range(3):
        b = order[s * 64:(s + 1) * 64]
        L, g = M.loss_and_grad(th, X[b].astype(np.float64), T[b].astype(np.float64), as64(norm))
        assert abs(losses[s] - L) <= 1e-5 * L
        th, mo, vo = M.adam_step(th, mo, vo, g, s + 1, lr=1e-3)
    got = m.iilbm_mlp_get_params().astype(np.float64)
    moved = np.abs(th - theta)
    assert np.median(np.abs(got - th)) <= 1e-6
    assert np.abs(got - th).max() <= 6e-3  # at most a few sign flips of tiny gradients
    assert np.median(moved) > 5e-4  # the steps did move the parameters


def test_training_reduces_the_loss():
    rng = np.random.default_rng(5)
    X = rng.normal(0, 1, (4096, 30)).astype(np.float32)
    A = rng.normal(0, 0.3, (30, 2))
    T = (np.tanh(X @ A) + 0.1 * X[:, :2] ** 2).astype(np.float32)
    m = iilbm.Mlp(W.mlp_init_params(5))
    order = np.concatenate([rng.permutation(4096) for _ in range(40)]).astype(np.int32)
    losses = m.train(X, T, order, batch=256, lr=1e-3)
    assert losses.size == 640
    assert losses[-40:].mean() < 0.1 * losses[:10].mean()


# -------------------------------------------------------------- in the step
def cylinder(storage, n, iters, tol, lib, orc=None):
    nx, ny, D, tau = 160, 64, 16.0, 0.7
    s = W.mrt_rates(tau)
    y = np.arange(ny) + 0.5
    u0 = np.repeat((4 * 0.05 * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)
    X = W.circle_markers(48.0, 32.5, D / 2, n)
    dX = W.polygon_perimeter(X) / n
    if lib == "gpu":
        g = iilbm.Lattice(nx, ny, collision=iilbm.MRT, storage=storage, tau=tau, s=s,
                          bc=iilbm.BC_CHANNEL, u_max=0.05)
        g.init_equilibrium(None, u0, None)
        g.set_interface(X, model=iilbm.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=iters,
                        mdf_tol=tol, aux=np.zeros((n, 2)))
        return g, X, dX
    o = orc.Oracle(nx, ny, collision=orc.MRT, tau=tau, s=s, bc=orc.BC_CHANNEL, u_max=0.05)
    o.init_equilibrium(None, u0, None)
    o.set_interface(X, model=orc.DIRECT, moves=False, dX=dX, eta=2.0, mdf_iters=iters,
                    mdf_tol=tol, UD=np.zeros((n, 2)))
    return o, X, dX


def test_features_match_oracle(orc):
    g, X, dX = cylinder("f64", 34, 5, 0.0, "gpu")
    o, _, _ = cylinder("f64", 34, 5, 0.0, "oracle", orc)
    g.step(12)
    o.step(12)
    F = g.iilbm_get_df_features(63.0)
    Fo = M.features(X, o.unforced_velocity(), np.zeros((34, 2)), dX, 63.0)
    scale = np.abs(Fo).max(0)
    assert np.all(np.abs(F - Fo) <= 1e-6 * np.maximum(scale, 1e-3))
    assert np.abs(Fo[:, 0:2]).max() > 1e-3  # the flow meets the body


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_proposal_is_the_networks_output(storage):
    """With no update pass, the force of the step is the network's proposal from the
    features of that step: compare with the network applied to the features the library
    reports."""
    theta, _, _, _ = problem(6)
    norm = dict(in_mean=np.zeros(30, np.float32), in_istd=np.full(30, 20.0, np.float32),
                out_mean=np.zeros(2, np.float32), out_scale=np.full(2, 0.01, np.float32))
    m = network(theta, norm)
    g, _, _ = cylinder(storage, 34, 0, 0.0, "gpu")
    g.step(8)
    g.iilbm_set_warm_start_mlp(m, 55.0)
    g.step(1)
    F = g.iilbm_get_df_features(55.0)
    G0 = m.forward(F).astype(np.float64)
    G = g.get_markers()["G"]
    assert np.abs(G - G0).max() <= 1e-5 * np.abs(G0).max()
    assert g.iilbm_get_mdf_stats()[0] == 0


def test_learned_start_converges_to_the_plain_answer():
    """A proposal only moves the start: run to the tolerance, the force and the flow
    agree with the plain iteration's to within what the tolerance leaves open.  The
    network here is untrained (random weights) with a normalisation that brings its
    inputs to O(1) and its proposals to the size of the body's force (~0.01); the
    iteration, which includes the jump's change of density near the body, converges
    from starts of that size (a start a hundred times larger can leave its region of
    convergence)."""
    theta, _, _, _ = problem(7)
    in_mean = np.zeros(30, np.float32)
    in_istd = np.ones(30, np.float32)
    in_istd[0::6] = in_istd[1::6] = 20.0   # U^D - U*, a few hundredths
    in_mean[5::6], in_istd[5::6] = 40.0, 0.05  # Re
    norm = dict(in_mean=in_mean, in_istd=in_istd, out_mean=np.zeros(2, np.float32),
                out_scale=np.full(2, 0.01, np.float32))
    m = network(theta, norm)
    a, _, _ = cylinder("f32", 34, 400, 1e-6, "gpu")
    b, _, _ = cylinder("f32", 34, 400, 1e-6, "gpu")
    b.iilbm_set_warm_start_mlp(m, 40.0)
    for _ in range(6):
        a.step(1)
        b.step(1)
        assert a.iilbm_get_mdf_stats()[1] < 1e-6 and b.iilbm_get_mdf_stats()[1] < 1e-6
    _, ua, va = a.get_macros()
    _, ub, vb = b.get_macros()
    assert max(np.abs(ua - ub).max(), np.abs(va - vb).max()) < 1e-4
