"""Pins of the oracle network (oracle/mlp.py) against the mathematics, on CPU.

The learned form's GPU training is checked against these gradients, so they are
pinned here to something other than themselves: central finite differences of
the loss, and the identity that the bfloat16-weight gradients are the plain
gradients at the rounded weights."""
import numpy as np

from oracle import mlp


def small_net(rng, sizes=(6, 5, 5, 5, 3)):
    return [(rng.uniform(-0.7, 0.7, (o, i)), rng.uniform(-0.2, 0.2, o)) for i, o in zip(sizes[:-1], sizes[1:])]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(31)
    params = small_net(rng)
    x, t = rng.uniform(-1, 1, (7, 6)), rng.uniform(-1, 1, (7, 3))
    grads = mlp.gradients(params, x, t, bf16_weights=False)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.loss(params, x, t, bf16_weights=False)
                arr[idx] = old - h
                lm = mlp.loss(params, x, t, bf16_weights=False)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-7 + 1e-6 * abs(fd), (l, idx, fd, g[idx])


def test_bf16_gradients_are_plain_gradients_at_rounded_weights():
    rng = np.random.default_rng(32)
    params = small_net(rng)
    x, t = rng.uniform(-1, 1, (5, 6)), rng.uniform(-1, 1, (5, 3))
    rounded = [(mlp.bf16_round(W), b) for W, b in params]
    a = mlp.gradients(params, x, t, bf16_weights=True)
    b = mlp.gradients(rounded, x, t, bf16_weights=False)
    for (ga, gb), (ha, hb) in zip(a, b):
        np.testing.assert_array_equal(ga, ha)
        np.testing.assert_array_equal(gb, hb)
    assert mlp.loss(params, x, t) != mlp.loss(params, x, t, bf16_weights=False)


def test_forward_is_the_composition_of_layers():
    """A 1-layer net is affine; hidden layers clip negative pre-activations."""
    rng = np.random.default_rng(33)
    W, b = rng.uniform(-1, 1, (3, 4)), rng.uniform(-1, 1, 3)
    x = rng.uniform(-1, 1, (6, 4))
    y, _ = mlp.forward([(W, b)], x, bf16_weights=False)
    np.testing.assert_allclose(y, x @ W.T + b, rtol=1e-15)
    y2, cache = mlp.forward([(W, b), (np.eye(3), np.zeros(3))], x, bf16_weights=False)
    np.testing.assert_allclose(y2, np.maximum(x @ W.T + b, 0.0), rtol=1e-15)
