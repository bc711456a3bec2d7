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

Inputs of a column T of one multigrid level (n_r cells, vertical index k):
point values p_Tk = f_Tk / (|T| v_k) of the right-hand side (cell integrals
over cell volumes), their root mean square s over the level, and

    x_T = [ p_T / s ,  (sum_e g_e p_{n_e}) / (s sum_e g_e) ],

the column and the mean over its three edge neighbours n_e weighted by the
two-point flux factors g_e of the finite-volume scheme.  The network predicts
u_T / s; the predicted solution is u_T = s y_T.  Adam (Kingma & Ba, 2015) is
the update of the training.
"""
from __future__ import annotations

import numpy as np

from . import bf16 as _bf16


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Elementwise rounding to bfloat16 (nearest, ties to even) with the oracle's rounding."""
    flat = np.asarray(a, dtype=np.float64).reshape(-1)
    return np.array([_bf16(float(v)) for v in flat]).reshape(np.shape(a))


def forward(params, x, bf16_weights: bool = True, bf16_acts: bool = False):
    """params: list of (W [out, in], b [out]).  Returns (y, cache of (a_{l-1}, z_l, W_l)).
    bf16_acts: every layer's input (x and the hidden activations) is rounded to
    bfloat16 first, as in the library's fused tensor-core inference."""
    a = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        Wl = bf16_round(W) if bf16_weights else np.asarray(W, dtype=np.float64)
        if bf16_acts:
            a = bf16_round(a)
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


def features(f, area, vol, nbr, g, cells=None):
    """Network inputs [rows, 2 n_r] of the field f ([n_cells * n_r], cell
    integrals) on a level with cell areas `area` [n], vertical volume factors
    `vol` [n_r], neighbours `nbr` [n, 3] and flux factors `g` [n, 3]; returns
    (x, s).  `cells` selects rows (default: every cell in order)."""
    area = np.asarray(area, dtype=np.float64)
    vol = np.asarray(vol, dtype=np.float64)
    n, n_r = area.shape[0], vol.shape[0]
    p = np.asarray(f, dtype=np.float64).reshape(n, n_r) / np.outer(area, vol)
    s = float(np.sqrt(np.mean(p * p)))
    w = np.asarray(g, dtype=np.float64)
    nbr = np.asarray(nbr)
    mean = np.zeros_like(p)
    for e in range(3):
        mean += w[:, e:e + 1] * p[nbr[:, e]]
    mean /= w.sum(axis=1, keepdims=True)
    x = np.concatenate([p, mean], axis=1)
    x = x / s if s > 0.0 else np.zeros_like(x)
    if cells is not None:
        x = x[np.asarray(cells)]
    return x, s


def targets(u, s, n_r, cells=None):
    """Training targets [rows, n_r] = u / s."""
    t = np.asarray(u, dtype=np.float64).reshape(-1, n_r)
    t = t / s if s > 0.0 else np.zeros_like(t)
    return t[np.asarray(cells)] if cells is not None else t


def predict(params, f, area, vol, nbr, g, bf16_weights: bool = True, bf16_acts: bool = False):
    """u = s network(x) for every column of the level: the learned coarse solve
    or warm start as the library computes it."""
    x, s = features(f, area, vol, nbr, g)
    y, _ = forward(params, x, bf16_weights, bf16_acts)
    return (s * y).reshape(-1)


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (step number t >= 1) on lists of arrays;
    returns (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p_, g_, m_, v_ in zip(params, grads, m, v):
        m1 = b1 * m_ + (1.0 - b1) * g_
        v1 = b2 * v_ + (1.0 - b2) * g_ * g_
        mh = m1 / (1.0 - b1 ** t)
        vh = v1 / (1.0 - b2 ** t)
        out_p.append(p_ - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(m1)
        out_v.append(v1)
    return out_p, out_m, out_v
