"""Oracle of the learned form's network: forward pass, loss and exact gradients.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy in float64,
each step written out as its definition.  The network is the multilayer
perceptron the library trains on the GPU:

    a_0 = x,   z_l = a_{l-1} W_l^T + b_l,   a_l = relu(z_l) (l < L),   y = z_L,

with the loss the mean over the batch and the outputs of the squared error,

    loss = sum_{b,o} (y_{bo} - t_{bo})^2 / (B * n_out).

The library computes its forward and backward passes with weights rounded to
bfloat16 (the masters stay FP32); gradients(bf16_weights=True) evaluates the
same function, so the two differ by FP32 accumulation only.  Backward pass by
the chain rule:

    dL/dy = 2 (y - t) / (B n_out),   dL/dz_l = dL/da_l * [z_l > 0] (l < L),
    dL/dW_l = (dL/dz_l)^T a_{l-1},   dL/db_l = sum_b dL/dz_l,   dL/da_{l-1} = dL/dz_l W_l.
"""
from __future__ import annotations

import numpy as np

from . import bf16 as _bf16


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Elementwise rounding to bfloat16 (nearest, ties to even) with the oracle's rounding."""
    flat = np.asarray(a, dtype=np.float64).reshape(-1)
    return np.array([_bf16(float(v)) for v in flat]).reshape(np.shape(a))


def forward(params, x, bf16_weights: bool = True):
    """params: list of (W [out, in], b [out]).  Returns (y, cache of (a_{l-1}, z_l, W_l))."""
    a = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        Wl = bf16_round(W) if bf16_weights else np.asarray(W, dtype=np.float64)
        z = a @ Wl.T + np.asarray(b, dtype=np.float64)
        cache.append((a, z, Wl))
        a = np.maximum(z, 0.0) if l < len(params) - 1 else z
    return a, cache


def loss(params, x, t, bf16_weights: bool = True) -> float:
    y, _ = forward(params, x, bf16_weights)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.sum(d * d) / d.size)


def gradients(params, x, t, bf16_weights: bool = True):
    """Exact gradients [(dW_l, db_l)] of loss() with respect to the weights the
    forward pass uses (the bfloat16-rounded ones when bf16_weights)."""
    y, cache = forward(params, x, bf16_weights)
    t = np.asarray(t, dtype=np.float64)
    g = 2.0 * (y - t) / y.size
    grads = []
    for l in range(len(params) - 1, -1, -1):
        a_prev, z, Wl = cache[l]
        if l < len(params) - 1:
            g = g * (z > 0.0)
        grads.append((g.T @ a_prev, g.sum(axis=0)))
        g = g @ Wl
    return grads[::-1]
