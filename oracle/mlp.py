"""FP64 CPU oracle of the learned closure's network (test infrastructure only).

The learned closure replaces KC-MP's SGS second moment m_sgs = m_neq - m_CE
(App. F.3) by the output of a small multilayer perceptron evaluated per cell:

    x  (10 inputs) -> standardise: xs = (x - mu_x) / sd_x
    h1 = silu(W1 xs + b1)   (64)
    h2 = silu(W2 h1 + b2)   (64)
    h3 = silu(W3 h2 + b3)   (64)
    ys = W4 h3 + b4         (6, standardised m_sgs / rho)
    y  = ys * sd_y + mu_y

silu(a) = a / (1 + exp(-a)).  Training minimises the mean squared error of the
standardised outputs, L = mean over samples and the 6 outputs of (ys - ts)^2,
with AdamW (decoupled weight decay on the weight matrices only).

Plain numpy, written for checking by eye: forward, the chain-rule backward and
one AdamW step.  Pins: tests/test_oracle_mlp.py (central finite differences of
the loss, the closed-form silu derivative, the first AdamW step).
"""
from __future__ import annotations

import numpy as np

SIZES = (10, 64, 64, 64, 6)


def init_params(seed: int = 0):
    """Kaiming-uniform-like initialisation: W_l ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), b_l = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for l in range(4):
        fi, fo = SIZES[l], SIZES[l + 1]
        p[f"W{l + 1}"] = rng.uniform(-1.0, 1.0, size=(fo, fi)) / np.sqrt(fi)
        p[f"b{l + 1}"] = np.zeros(fo)
    return p


def silu(a):
    return a / (1.0 + np.exp(-a))


def silu_grad(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def forward(p, xs):
    """xs [n, 10] (standardised) -> ys [n, 6]; also the pre-activations for backward."""
    a1 = xs @ p["W1"].T + p["b1"]
    h1 = silu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(a2)
    a3 = h2 @ p["W3"].T + p["b3"]
    h3 = silu(a3)
    ys = h3 @ p["W4"].T + p["b4"]
    return ys, (xs, a1, h1, a2, h2, a3, h3)


def loss(p, xs, ts):
    ys, _ = forward(p, xs)
    return float(np.mean((ys - ts) ** 2))


def backward(p, xs, ts):
    """Gradients of L = mean((ys - ts)^2) with respect to every parameter."""
    ys, (x, a1, h1, a2, h2, a3, h3) = forward(p, xs)
    n = xs.shape[0]
    dy = 2.0 * (ys - ts) / (n * ys.shape[1])
    g = {}
    g["W4"] = dy.T @ h3
    g["b4"] = dy.sum(axis=0)
    d3 = (dy @ p["W4"]) * silu_grad(a3)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"]) * silu_grad(a2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * silu_grad(a1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return g


def adamw_step(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (Loshchilov & Hutter): m, v moment estimates with bias
    correction at step t (1-based); weight decay lr*wd*W applied to weight
    matrices only.  Updates p, m, v in place."""
    for k in p:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mh = m[k] / (1.0 - beta1 ** t)
        vh = v[k] / (1.0 - beta2 ** t)
        if k.startswith("W") and wd:
            p[k] = p[k] - lr * wd * p[k]
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def flat(p):
    """Parameters in the flat order W1 b1 W2 b2 W3 b3 W4 b4 (row-major W[out][in])."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel()
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")])


def unflat(v):
    p, o = {}, 0
    for l in range(4):
        fi, fo = SIZES[l], SIZES[l + 1]
        p[f"W{l + 1}"] = np.asarray(v[o:o + fo * fi], dtype=np.float64).reshape(fo, fi)
        o += fo * fi
        p[f"b{l + 1}"] = np.asarray(v[o:o + fo], dtype=np.float64).copy()
        o += fo
    return p


NPARAM = sum(SIZES[l] * SIZES[l + 1] + SIZES[l + 1] for l in range(4))
