"""Learned warm start: the density-profile MLP, FP64 oracle (test infrastructure only).

The network is not part of the paper: it predicts the steady density profile of a
liquid column (the set-up of Sec. IV) from six column descriptors, and its output
only initialises the lattice Boltzmann run, which alone decides the result.

Definition (plain FP64, in this order):
    x  = (T/T_c, log10|g|, form, <rho>/rho_c, z/H, log2 H) mapped by the fixed
         affine normalisation FEATURE_CENTER / FEATURE_SCALE
    Z1 = x W1^T + b1,  H1 = silu(Z1)          (W1: 128 x 6)
    Z2 = H1 W2^T + b2, H2 = silu(Z2)          (W2: 128 x 128)
    Z3 = H2 W3^T + b3, H3 = silu(Z3)          (W3: 128 x 128)
    y  = H3 w4 + b4                           (predicted rho / rho_c)
    loss = mean over the batch of (y - t)^2
with silu(z) = z sigmoid(z). Gradients by the chain rule (backward), Adam with bias
correction for the update.

``bf16=True`` applies the mixed-precision storage points of the GPU path: the inputs x,
the weights W1..W3 and the activations H1, H2 used as matrix operands are rounded to
bfloat16 (round to nearest even), and so are the error signals dZ1..dZ3 used as matrix
operands; everything else (biases, w4, b4, Z, H3, y, bias gradients) stays at full
precision. Rounding follows the bfloat16 format definition (the top 16 bits of an IEEE
binary32 value).

Pins: finite-difference gradients, closed forms of silu and of special networks, the
first Adam step, and known bfloat16 roundings (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

WIDTH = 128
N_IN = 6
# x_norm = (x - center) / scale: T/T_c in [0.70, 0.95], log10|g| in [-6, -4], form in
# {1, 2}, <rho>/rho_c in ~[0.3, 2.5], z/H in (0, 1), log2 H in [6, 10]
FEATURE_CENTER = np.array([0.825, -5.0, 1.5, 1.4, 0.5, 8.0])
FEATURE_SCALE = np.array([0.125, 1.0, 0.5, 1.1, 0.5, 2.0])


def to_bf16(a):
    """Round to the nearest bfloat16 (ties to even) and return the value as float64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def normalise(raw):
    """raw: (n, 6) column descriptors -> network inputs."""
    return (np.asarray(raw, dtype=np.float64) - FEATURE_CENTER) / FEATURE_SCALE


def init_params(u):
    """Parameters from uniform draws u (a dict of arrays in [0, 1) with the shapes of
    the parameters): every weight uniform in +-sqrt(6/(fan_in + fan_out)), biases 0."""
    def glorot(x, fan_in, fan_out):
        return (2.0 * x - 1.0) * np.sqrt(6.0 / (fan_in + fan_out))

    return {
        "W1": glorot(u["W1"], N_IN, WIDTH), "b1": np.zeros(WIDTH),
        "W2": glorot(u["W2"], WIDTH, WIDTH), "b2": np.zeros(WIDTH),
        "W3": glorot(u["W3"], WIDTH, WIDTH), "b3": np.zeros(WIDTH),
        "w4": glorot(u["w4"], WIDTH, 1), "b4": np.zeros(1),
    }


def forward(x, P, bf16=False):
    """Returns y and the cache of the forward pass (x: normalised inputs, (n, 6))."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = r(x)
    Z1 = X @ r(P["W1"]).T + P["b1"]
    H1 = silu(Z1)
    Z2 = r(H1) @ r(P["W2"]).T + P["b2"]
    H2 = silu(Z2)
    Z3 = r(H2) @ r(P["W3"]).T + P["b3"]
    H3 = silu(Z3)
    y = H3 @ P["w4"] + P["b4"][0]
    return y, dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3)


def loss_and_grads(x, t, P, bf16=False):
    """Mean squared error over the batch and its gradient with respect to every parameter."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(x, P, bf16)
    n = len(t)
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    g = {"w4": c["H3"].T @ dy, "b4": np.array([np.sum(dy)])}
    dZ3 = np.outer(dy, P["w4"]) * dsilu(c["Z3"])
    g["W3"] = r(dZ3).T @ r(c["H2"])
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = (r(dZ3) @ r(P["W3"])) * dsilu(c["Z2"])
    g["W2"] = r(dZ2).T @ r(c["H1"])
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (r(dZ2) @ r(P["W2"])) * dsilu(c["Z1"])
    g["W1"] = r(dZ1).T @ c["X"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def adam_step(P, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected, step number t >= 1); returns new P, m, v."""
    P2, m2, v2 = {}, {}, {}
    for k in P:
        m2[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v2[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mh = m2[k] / (1.0 - beta1**t)
        vh = v2[k] / (1.0 - beta2**t)
        P2[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P2, m2, v2
