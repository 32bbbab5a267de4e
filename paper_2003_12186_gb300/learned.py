"""The learned warm start of direct forcing, end to end: data from the method itself,
training with the library's kernels, and the gain measured against the plain iteration.

* generate(): rigid-cylinder channels (workloads.learned_channels) advanced by the
  batched executor with the force iteration run to the no-slip tolerance; at recorded
  steps every marker contributes one sample (its 30 features from that step's
  unforced velocity U*, and the force the iteration converged to).
* train(): normalisation from the training split, Adam on shuffled batches (the order
  is drawn here, on the host, and passed to the kernels), the held-out loss.
* evaluate(): the same kind of channels from another seed, three starts of the force
  iteration (zero, the previous step's force, the network's proposal) under the same
  stopping rule: mean passes per step, the residual reached, and throughput.

Host code only orchestrates; every step of the method and of the network runs in the
CUDA library through its C ABI.
"""
from __future__ import annotations

import time

import numpy as np

from . import iilbm
from . import workloads as W

TOL = 1e-6        # no-slip residual max_k |U^D - U_k| that ends the force iteration
MAX_PASSES = 500  # the iteration's cap


def _parabola(nx, ny, u_max):
    y = np.arange(ny) + 0.5
    return np.repeat((4.0 * u_max * y * (ny - y) / ny ** 2)[:, None], nx, axis=1)


def make_channel(sim, tol=TOL, max_passes=MAX_PASSES):
    """FP32 MRT channel with the cylinder of `sim`, started from the parabolic inflow:
    II-LBM, the normal part of the body force through the jump and the tangential part
    spread; the force iteration sees the force through that same operator, so run to
    the tolerance it gives the step's collision velocity no slip at the markers."""
    g = iilbm.Lattice(sim["nx"], sim["ny"], collision=iilbm.MRT, storage="f32", tau=sim["tau"],
                      s=W.mrt_rates(sim["tau"]), bc=iilbm.BC_CHANNEL, u_max=sim["u_max"],
                      jump=1)
    g.init_equilibrium(None, _parabola(sim["nx"], sim["ny"], sim["u_max"]), None)
    g.set_interface(sim["X"], model=iilbm.DIRECT, moves=False, dX=sim["dX"], eta=2.0,
                    mdf_iters=max_passes, mdf_tol=tol, aux=np.zeros((sim["n"], 2)))
    return g


def generate(count=64, seed=1, spin_up=400, records=64, every=100, nx=512, ny=128):
    """Samples (X [N][30] FP32 features, T [N][2] FP32 converged forces) from `records`
    recorded steps of `count` channels; returns X, T and the channel of each sample."""
    sims = W.learned_channels(count, seed, nx=nx, ny=ny)
    # the label is the force the plain iteration (zero start) reaches at the tolerance:
    # the operator of the iteration has near-null directions, along which the converged
    # force depends on the start -- a previous-step start carries an arbitrary, drifting
    # component there that no network can predict from the features
    lat = [make_channel(s) for s in sims]
    Xs, Ts, Ss = [], [], []
    with iilbm.Batch(lat) as B:
        B.step(spin_up)
        for _ in range(records):
            B.step(every)
            B.synchronize()
            for k, (g, s) in enumerate(zip(lat, sims)):
                Xs.append(g.iilbm_get_df_features(s["re"]))
                Ts.append(g.get_markers()["G"].astype(np.float32))
                Ss.append(np.full(s["n"], k, dtype=np.int32))
    return np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ss)


def normalization(X, T):
    """Per-feature mean and reciprocal deviation, per-output mean and deviation."""
    sd = X.std(0)
    return dict(in_mean=X.mean(0).astype(np.float32),
                in_istd=(1.0 / np.where(sd > 0, sd, 1.0)).astype(np.float32),
                out_mean=T.mean(0).astype(np.float32),
                out_scale=np.where(T.std(0) > 0, T.std(0), 1.0).astype(np.float32))


def train(X, T, epochs=30, batch=1024, lr=1e-3, seed=0, val_frac=0.2, init_seed=0):
    """Train a network on (X, T); returns the network, its normalisation and a report
    (per-epoch training losses, held-out MSE of the normalised outputs)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(X))
    nval = int(round(val_frac * len(X)))
    val, tr = perm[:nval], perm[nval:]
    norm = normalization(X[tr], T[tr])
    m = iilbm.Mlp(W.mlp_init_params(init_seed))
    m.iilbm_mlp_set_normalization(norm["in_mean"], norm["in_istd"], norm["out_mean"],
                                  norm["out_scale"])
    Xt, Tt = np.ascontiguousarray(X[tr]), np.ascontiguousarray(T[tr])
    per_epoch = len(tr) // batch
    order = np.concatenate([rng.permutation(len(tr))[:per_epoch * batch] for _ in range(epochs)])
    t0 = time.perf_counter()
    losses = m.train(Xt, Tt, order.astype(np.int32), batch=batch, lr=lr)
    train_s = time.perf_counter() - t0
    val_mse = None
    if nval:
        Y = m.forward(np.ascontiguousarray(X[val]))
        val_mse = float(np.mean(((Y - T[val]) / norm["out_scale"]) ** 2))
    report = dict(samples=len(X), train=len(tr), held_out=nval, epochs=epochs, batch=batch,
                  lr=lr, steps=len(losses), seconds=train_s,
                  first_loss=float(losses[:per_epoch].mean()) if per_epoch else None,
                  last_loss=float(losses[-per_epoch:].mean()) if per_epoch else None,
                  val_mse=val_mse)
    return m, norm, report


def evaluate(mlp, count=64, seed=2, spin_up=400, count_steps=32, timed_steps=256, nx=512,
             ny=128, modes=("plain", "previous", "mlp")):
    """Force passes per step and throughput of the three starts on the same channels."""
    import torch

    sims = W.learned_channels(count, seed, nx=nx, ny=ny)
    cells = sum(s["nx"] * s["ny"] for s in sims)
    out = {}
    for mode in modes:
        lat = [make_channel(s) for s in sims]
        for g, s in zip(lat, sims):
            if mode == "previous":
                g.iilbm_set_warm_start_mode(iilbm.WS_PREVIOUS)
            elif mode == "mlp":
                g.iilbm_set_warm_start_mlp(mlp, s["re"])
        with iilbm.Batch(lat) as B:
            B.step(spin_up)
            B.autotune(32)  # the stream-collide variant for these lattices (the run advances)
            B.synchronize()
            passes, worst, capped = [], 0.0, 0
            for _ in range(count_steps):
                B.step(1)
                for g in lat:
                    it, res = g.iilbm_get_mdf_stats()
                    passes.append(it)
                    worst = max(worst, res)
                    capped += it >= MAX_PASSES
            B.synchronize()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.step(timed_steps)
            B.synchronize()
            dt = time.perf_counter() - t0
        out[mode] = dict(passes_per_step=float(np.mean(passes)), worst_residual=worst,
                         capped=int(capped), mlups=cells * timed_steps / dt / 1e6,
                         us_per_step=dt / timed_steps * 1e6)
        del lat
    return out
