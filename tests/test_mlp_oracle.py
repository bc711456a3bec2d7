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


def _level(o, level):
    grid = o.grid(o.level_ref(level))
    return grid["area"], o.vertical()["vol"], grid["nbr"], grid["g"]


def test_features_of_constant_point_values():
    """p = c everywhere: s = |c| and every input is sign(c)."""
    import oracle
    o = oracle.Oracle(refinement=2, n_levels=2, n_r=5, grading=1.1)
    area, vol, nbr, g = _level(o, 1)
    for c in (2.5, -0.75):
        f = c * np.outer(area, vol).reshape(-1)
        x, s = mlp.features(f, area, vol, nbr, g)
        assert abs(s - abs(c)) <= 1e-15 * abs(c)
        np.testing.assert_allclose(x, np.sign(c), rtol=1e-14)


def test_features_of_a_single_cell_pick_the_flux_weights():
    """A unit point value in one cell: its own input is 1/s at its level, and each
    edge neighbour sees it in the mean block with weight g_e / sum g of the
    neighbour's edge that faces it; every other input is zero."""
    import oracle
    o = oracle.Oracle(refinement=2, n_levels=2, n_r=4, grading=1.2)
    area, vol, nbr, g = _level(o, 1)
    n, n_r = area.shape[0], vol.shape[0]
    T0, k0 = 17, 2
    p = np.zeros((n, n_r))
    p[T0, k0] = 1.0
    f = (p * np.outer(area, vol)).reshape(-1)
    x, s = mlp.features(f, area, vol, nbr, g)
    assert abs(s - 1.0 / np.sqrt(n * n_r)) < 1e-15
    expect = np.zeros((n, 2 * n_r))
    expect[T0, k0] = 1.0 / s
    for T in range(n):
        for e in range(3):
            if nbr[T, e] == T0:
                expect[T, n_r + k0] += g[T, e] / g[T].sum() / s
    assert np.count_nonzero(expect[:, n_r:]) == 3
    np.testing.assert_allclose(x, expect, rtol=1e-13, atol=1e-13)


def test_features_are_odd_and_scale_free():
    import oracle
    o = oracle.Oracle(refinement=2, n_levels=2, n_r=3)
    area, vol, nbr, g = _level(o, 1)
    f = np.random.default_rng(5).uniform(-1, 1, area.shape[0] * 3)
    x, s = mlp.features(f, area, vol, nbr, g)
    x2, s2 = mlp.features(-4.0 * f, area, vol, nbr, g)
    assert abs(s2 - 4.0 * s) <= 1e-14 * s2
    np.testing.assert_allclose(x2, -x, rtol=1e-13, atol=1e-15)
    x0, s0 = mlp.features(0.0 * f, area, vol, nbr, g)
    assert s0 == 0.0 and not np.any(x0)


def test_adam_first_step_is_the_sign_of_the_gradient():
    """With zero moments, bias correction makes the first Adam step
    lr g / (|g| + eps) = lr sign(g) for |g| >> eps."""
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([3.0, -0.01, 1e-3])]
    z = [np.zeros(3)]
    p1, m1, v1 = mlp.adam_step(p, g, z, z, t=1, lr=0.1)
    np.testing.assert_allclose(p1[0], p[0] - 0.1 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(p1[0], p[0] - 0.1 * np.sign(g[0]), rtol=1e-5)
    np.testing.assert_allclose(m1[0], 0.1 * g[0], rtol=1e-15)
    np.testing.assert_allclose(v1[0], 0.001 * g[0] ** 2, rtol=1e-12)


def test_oracle_coarse_solve_hook():
    """The coarsest-level solve replaced through the hook by a guess and one
    block-Jacobi sweep: with a single level, a zero guess is exactly one Jacobi
    sweep from zero (the V-cycle of a Jacobi-smoothed oracle with nu_coarse 1);
    with two levels, the exact dense solve as guess is left unchanged by the
    sweep and equals converged sweeps."""
    import oracle
    r1 = np.random.default_rng(6).uniform(-1, 1, 320 * 6)
    o = oracle.Oracle(refinement=2, n_levels=1, n_r=6, grading=1.1)
    o.set_coarse_solve(lambda f: np.zeros_like(f))
    np.testing.assert_array_equal(o.vcycle(r1), oracle.Oracle(refinement=2, n_levels=1, n_r=6, grading=1.1,
                                                              smoother=1, nu_coarse=1).vcycle(r1))
    kw = dict(refinement=3, n_levels=2, n_r=6, grading=1.1, courant_c=8.0)
    r = np.random.default_rng(7).uniform(-1, 1, 1280 * 6)
    o = oracle.Oracle(**kw)
    A0 = o.dense_operator(level=0)
    o.set_coarse_solve(lambda f: np.linalg.solve(A0, f))
    z, z_ref = o.vcycle(r), oracle.Oracle(nu_coarse=40, **kw).vcycle(r)
    # the sweep re-solves the stiff columns from a residual of rounding size
    assert np.max(np.abs(z - z_ref)) <= 1e-10 * np.max(np.abs(z_ref))
    o.set_coarse_solve(None)
    np.testing.assert_array_equal(o.vcycle(r), oracle.Oracle(**kw).vcycle(r))


def test_bf16_activations_round_every_layer_input():
    """forward(bf16_acts=True) rounds x and each hidden activation to bfloat16
    before the product: for one layer it is the plain forward of bf16(x), for
    two layers the second layer sees bf16(relu(.))."""
    rng = np.random.default_rng(34)
    W1, b1 = rng.uniform(-1, 1, (5, 4)), rng.uniform(-1, 1, 5)
    W2, b2 = rng.uniform(-1, 1, (3, 5)), rng.uniform(-1, 1, 3)
    x = rng.uniform(-1, 1, (6, 4))
    y, _ = mlp.forward([(W1, b1)], x, bf16_acts=True)
    y_ref, _ = mlp.forward([(W1, b1)], mlp.bf16_round(x))
    np.testing.assert_array_equal(y, y_ref)
    y2, _ = mlp.forward([(W1, b1), (W2, b2)], x, bf16_acts=True)
    h = np.maximum(mlp.bf16_round(x) @ mlp.bf16_round(W1).T + b1, 0.0)
    np.testing.assert_array_equal(y2, mlp.bf16_round(h) @ mlp.bf16_round(W2).T + b2)
    assert not np.array_equal(y2, mlp.forward([(W1, b1), (W2, b2)], x)[0])
