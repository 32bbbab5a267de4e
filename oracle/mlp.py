"""Oracle of the learned warm start for direct forcing: a plain FP64 numpy statement of
the features, the network, its loss, gradient and optimiser step.

TEST INFRASTRUCTURE: only tests/, the smoke check and the benchmark's CPU baseline use
this module; the CUDA library shares no code with it.

The paper's direct forcing (Eq. 18, repeated) starts from G = 0; the learned part
proposes the starting force G^(0)_k of every marker from local, method-generated
quantities.  Definitions (readings, stated once here):

* Features of marker k, 6 for each of the markers j = k-2 .. k+2 (indices cyclic along
  the closed polygon), 30 in all, in the order j = k-2, ..., k+2:
    dU_j = U^D_j - U*_j   (2)  U* = the velocity interpolated at the markers (Eq. 20)
                               from the state without the body's force
    n_j                   (2)  outward unit normal: the tangent X_{j+1} - X_{j-1}
                               rotated by -90 degrees (counter-clockwise polygon)
    kappa_j               (1)  signed curvature -(X_{j+1} - 2 X_j + X_{j-1}) . n_j / dX^2
                               (1/R on a regular polygon of circumradius R)
    Re                    (1)  the flow's Reynolds number
* Network: xh = (x - mu) * istd;  h1 = gelu(W1 xh + b1), h2 = gelu(W2 h1 + b2),
  h3 = gelu(W3 h2 + b3) (width 64);  yh = W4 h3 + b4;  G^(0) = yh * s_o + mu_o.
  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (the exact form).
* Loss on a batch of B samples with targets G: L = mean over samples and the two
  components of (yh - (G - mu_o) / s_o)^2.
* Optimiser: Adam with bias correction (lr, beta1, beta2, eps).
* Parameter vector (float32 on the GPU): W1 [64][30], b1 [64], W2 [64][64], b2, W3
  [64][64], b3, W4 [2][64], b4 [2] -- 10434 values.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf as _erf

N_IN, N_HID, N_OUT = 30, 64, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Parameter vector -> dict of arrays (views, FP64)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[o:o + size].reshape(shape)
        o += size
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


# ---------------------------------------------------------------- activation
def gelu(z):
    """z Phi(z), Phi the standard normal distribution function (erf form)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    Phi = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return Phi + z * phi


# ------------------------------------------------------------------ network
def forward(theta, X, norm):
    """Outputs G^(0) [B][2] and the cache of the pass (pre-activations, activations)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    xh = (X - norm["in_mean"]) * norm["in_istd"]
    z1 = xh @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    z3 = a2 @ p["W3"].T + p["b3"]
    a3 = gelu(z3)
    yh = a3 @ p["W4"].T + p["b4"]
    G = yh * norm["out_scale"] + norm["out_mean"]
    return G, dict(xh=xh, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, yh=yh)


def loss_and_grad(theta, X, T, norm):
    """Mean squared error of the normalised outputs, and its gradient (backpropagation
    written out layer by layer)."""
    p = unpack(theta)
    _, c = forward(theta, X, norm)
    th = (np.asarray(T, dtype=np.float64) - norm["out_mean"]) / norm["out_scale"]
    B = th.shape[0]
    e = c["yh"] - th
    L = float(np.mean(e * e))
    dyh = 2.0 * e / (B * N_OUT)
    g = {}
    g["W4"] = dyh.T @ c["a3"]
    g["b4"] = dyh.sum(0)
    dz3 = (dyh @ p["W4"]) * gelu_prime(c["z3"])
    g["W3"] = dz3.T @ c["a2"]
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * gelu_prime(c["z2"])
    g["W2"] = dz2.T @ c["a1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_prime(c["z1"])
    g["W1"] = dz1.T @ c["xh"]
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1, bias-corrected); returns new theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------------- features
def marker_geometry(X, dX):
    """Outward unit normals and signed curvature of a closed counter-clockwise polygon."""
    X = np.asarray(X, dtype=np.float64)
    Xp, Xm = np.roll(X, -1, axis=0), np.roll(X, 1, axis=0)
    t = Xp - Xm
    nrm = np.stack([t[:, 1], -t[:, 0]], axis=1) / np.linalg.norm(t, axis=1)[:, None]
    d2 = Xp - 2.0 * X + Xm
    kappa = -(d2 * nrm).sum(1) / (dX * dX)
    return nrm, kappa


def features(X, Ustar, UD, dX, Re):
    """[n][30] features of every marker (see the module docstring)."""
    nrm, kappa = marker_geometry(X, dX)
    dU = np.asarray(UD, dtype=np.float64) - np.asarray(Ustar, dtype=np.float64)
    per = np.concatenate([dU, nrm, kappa[:, None], np.full((len(kappa), 1), float(Re))], axis=1)
    return np.concatenate([np.roll(per, 2 - q, axis=0) for q in range(5)], axis=1)
