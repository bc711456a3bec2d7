"""The learned form on the GPU, through the C ABI (tpmg_learned.h), against the
oracle (oracle/mlp.py, the oracle V-cycle with its coarse-solve hook).

* the network's forward pass, loss and gradients against the float64 oracle
  with the same bfloat16 weights (FP32 accumulation on the GPU);
* one Adam step against the oracle's Adam;
* features and targets against the oracle's definition on the oracle's mesh;
* the V-cycle with the network as coarsest-level solve against the oracle
  V-cycle with the same network hooked in;
* the learned solve: equal to plain flexible CG when no network is attached,
  the judge rejecting useless guesses, the fallback finishing a solve the
  network cannot, and what a trained network gains (reported).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1408_2981_gb300 import binding, build, inputs, learned

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)
SMALL = dict(refinement=4, n_levels=3, n_r=16, grading=1.05, courant_c=8.0, nu_pre=2, nu_post=2, nu_coarse=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def random_net(n_r, hidden, seed, scale=1.0):
    net = binding.Net(n_r, hidden)
    flat = learned.init_params(net.sizes, seed)
    # non-zero biases so that the bias paths are exercised
    off = 0
    for i, o in zip(net.sizes[:-1], net.sizes[1:]):
        off += o * i
        flat[off:off + o] = inputs.uniform_pm1(seed + 99 + off, o) * 0.1
        off += o
    flat = (flat * np.float32(scale)).astype(np.float32)
    net.set_params(flat)
    return net, flat


def cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("rows", [1, 63, 300])
def test_forward_and_gradients_match_the_oracle(rows):
    n_r, hidden = 12, 64
    net, flat = random_net(n_r, hidden, seed=inputs.SEED_LEARNED + rows)
    params = net.unflatten(flat.astype(np.float64))
    x = inputs.uniform_pm1(inputs.SEED_LEARNED + 1, rows * 2 * n_r).reshape(rows, 2 * n_r)
    t = inputs.uniform_pm1(inputs.SEED_LEARNED + 2, rows * n_r).reshape(rows, n_r)
    xg, tg = cuda32(x), cuda32(t)
    # the GPU sees x, t rounded to FP32: give the oracle the same numbers
    x32, t32 = xg.cpu().double().numpy(), tg.cpu().double().numpy()
    y = torch.empty((rows, n_r), dtype=torch.float32, device="cuda")
    net.forward(xg, y)
    y_ref, _ = mlp.forward(params, x32)
    assert np.max(np.abs(y.cpu().double().numpy() - y_ref)) <= 1e-5 * max(1.0, np.max(np.abs(y_ref)))
    grad = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    loss = net.gradients(xg, tg, grad)
    assert abs(loss - mlp.loss(params, x32, t32)) <= 1e-5 * abs(loss)
    g = net.unflatten(grad.cpu().double().numpy())
    for l, ((dW, db), (rW, rb)) in enumerate(zip(g, mlp.gradients(params, x32, t32))):
        for got, ref in ((dW, rW), (db, rb)):
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(got - ref)) <= 2e-4 * scale + 1e-12, (l, np.max(np.abs(got - ref)), scale)


def test_adam_step_matches_the_oracle():
    n_r, hidden, rows = 8, 64, 200
    net, flat = random_net(n_r, hidden, seed=inputs.SEED_LEARNED + 5)
    x = cuda32(inputs.uniform_pm1(inputs.SEED_LEARNED + 6, rows * 2 * n_r).reshape(rows, 2 * n_r))
    t = cuda32(inputs.uniform_pm1(inputs.SEED_LEARNED + 7, rows * n_r).reshape(rows, n_r))
    grad = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    net.gradients(x, t, grad)
    g = grad.cpu().double().numpy()
    net.train_step(x, t, lr=1e-3)
    after = net.get_params().astype(np.float64)
    # the update from the GPU's own gradient, in float64 (same gradient, so only
    # the update's arithmetic is compared)
    p1, _, _ = mlp.adam_step([flat.astype(np.float64)], [g], [np.zeros_like(g)], [np.zeros_like(g)], t=1, lr=1e-3)
    assert np.max(np.abs(after - p1[0])) <= 1e-6 * max(1.0, np.max(np.abs(p1[0])))
    assert not np.array_equal(after, flat)


def test_training_reduces_the_loss():
    """A network fitted to a fixed linear map of its inputs: the loss falls by 20x."""
    n_r, hidden, rows = 8, 64, 4096
    net, _ = random_net(n_r, hidden, seed=inputs.SEED_LEARNED + 8)
    x = inputs.uniform_pm1(inputs.SEED_LEARNED + 9, rows * 2 * n_r).reshape(rows, 2 * n_r)
    M = inputs.uniform_pm1(inputs.SEED_LEARNED + 10, 2 * n_r * n_r).reshape(2 * n_r, n_r) / np.sqrt(2 * n_r)
    xg, tg = cuda32(x), cuda32(x @ M)
    before = learned.full_loss(net, xg, tg)
    out = learned.train(net, xg, tg, steps=600, seed=inputs.SEED_LEARNED + 11, batch=512, lr=3e-3)
    assert out["final"] < before / 20, (before, out["final"])


def test_features_and_targets_match_the_oracle():
    s = binding.Solver(**SMALL, **MIXED)
    o = oracle.Oracle(**{k: v for k, v in SMALL.items()})
    n_r = s.n_r
    for level in (0, s.n_levels - 1):
        grid = o.grid(o.level_ref(level))
        vol = o.vertical()["vol"]
        n = grid["area"].shape[0]
        assert n == s.query(level)[0]
        f = inputs.uniform_pm1(inputs.SEED_LEARNED + 20 + level, n * n_r)
        u = inputs.uniform_pm1(inputs.SEED_LEARNED + 30 + level, n * n_r)
        cells = (inputs.splitmix64(inputs.SEED_LEARNED + 40, 37) % np.uint64(n)).astype(np.int32)
        x_ref, s_ref = mlp.features(f, grid["area"], vol, grid["nbr"], grid["g"], cells=cells)
        t_ref = mlp.targets(u, s_ref, n_r, cells=cells)
        fg, ug = torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()
        x = torch.empty((37, 2 * n_r), dtype=torch.float32, device="cuda")
        t = torch.empty((37, n_r), dtype=torch.float32, device="cuda")
        sg = s.net_features(level, fg, x, cells=torch.from_numpy(cells).cuda())
        s.net_targets(level, fg, ug, t, cells=torch.from_numpy(cells).cuda())
        assert abs(sg - s_ref) <= 1e-6 * s_ref   # point values in FP32, sums in double
        np.testing.assert_allclose(x.cpu().double().numpy(), x_ref, rtol=1e-6, atol=1e-6 * np.max(np.abs(x_ref)))
        np.testing.assert_allclose(t.cpu().double().numpy(), t_ref, rtol=1e-6, atol=1e-7)
        # all columns in order when no cells are given
        xa = torch.empty((n, 2 * n_r), dtype=torch.float32, device="cuda")
        s.net_features(level, fg, xa)
        xa_ref, _ = mlp.features(f, grid["area"], vol, grid["nbr"], grid["g"])
        np.testing.assert_allclose(xa.cpu().double().numpy(), xa_ref, rtol=1e-6, atol=1e-6 * np.max(np.abs(xa_ref)))


def test_vcycle_with_network_coarse_solve_matches_the_oracle():
    """B r with the network's guess and one line relaxation as coarsest-level
    solve: FP32 V-cycle on the BF16 stencil against the oracle's V-cycle
    (BF16-rounded coefficients, FP64) with the same network (bfloat16 weights,
    float64 activations) hooked in."""
    s = binding.Solver(**SMALL, **MIXED)
    o = oracle.Oracle(**SMALL)
    o.set_vcycle_bf16(True)
    net, flat = random_net(s.n_r, 64, seed=inputs.SEED_LEARNED + 50, scale=0.5)
    params = net.unflatten(flat.astype(np.float64))
    grid0 = o.grid(o.level_ref(0))
    vol = o.vertical()["vol"]
    o.set_coarse_solve(lambda f0: mlp.predict(params, f0, grid0["area"], vol, grid0["nbr"], grid0["g"],
                                              bf16_acts=True))
    s.attach_net(binding.TPMG_NET_COARSE, net)
    r = inputs.uniform_pm1(inputs.SEED_LEARNED + 51, s.N)
    z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.vcycle_learned(torch.from_numpy(r).cuda(), z)
    z_ref = o.vcycle(r)
    err = np.max(np.abs(z.cpu().numpy() - z_ref)) / np.max(np.abs(z_ref))
    assert err <= 5e-3, err
    # the network changed the result: the plain V-cycle differs by much more
    o.set_coarse_solve(None)
    z_plain = o.vcycle(r)
    assert np.max(np.abs(z_plain - z_ref)) / np.max(np.abs(z_ref)) > 10 * err


@pytest.mark.parametrize("hidden", [64, 48])
def test_network_prediction_matches_the_oracle(hidden):
    """The attached network's prediction u = s network(features(f)) on the
    coarsest and the finest level.  Hidden width 64 runs the fused tensor-core
    kernel (inputs and activations rounded to bfloat16: the oracle rounds the
    same way; a rounding boundary crossed differently moves a value by one
    bfloat16 step, hence the tolerance); width 48 runs layer by layer in FP32."""
    s = binding.Solver(**SMALL, **MIXED)
    o = oracle.Oracle(**SMALL)
    vol = o.vertical()["vol"]
    net, flat = random_net(s.n_r, hidden, seed=inputs.SEED_LEARNED + 80 + hidden)
    params = net.unflatten(flat.astype(np.float64))
    for role, level in ((binding.TPMG_NET_COARSE, 0), (binding.TPMG_NET_WARM, s.n_levels - 1)):
        s.attach_net(role, net)
        grid = o.grid(o.level_ref(level))
        n = grid["area"].shape[0] * s.n_r
        f = inputs.uniform_pm1(inputs.SEED_LEARNED + 81 + level, n)
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.net_predict(role, torch.from_numpy(f).cuda(), u)
        ref = mlp.predict(params, f, grid["area"], vol, grid["nbr"], grid["g"], bf16_acts=hidden == 64)
        got = u.cpu().numpy()
        err = np.abs(got - ref)
        scale = np.max(np.abs(ref))
        assert np.max(err) <= (2e-2 if hidden == 64 else 1e-5) * scale, (role, np.max(err) / scale)
        assert np.mean(err) <= (2e-3 if hidden == 64 else 1e-6) * np.mean(np.abs(ref)), (role, np.mean(err))
        s.attach_net(role, None)


@pytest.mark.parametrize("n_r", [16, 32, 64, 128])
def test_tcgen05_network_matches_the_mma_sync_kernel(n_r):
    """The network on tcgen05 (tiles of 128 columns, accumulators in tensor memory)
    against the mma.sync kernel: the same bfloat16 roundings of inputs and
    activations, FP32 accumulation in another order, so values agree up to an
    occasional rounding boundary crossed differently.  Level 0 has 320 columns
    (a ragged third tile), the finest 5120; the kernel reports no timeout."""
    kw = dict(refinement=4, n_levels=3, n_r=n_r, grading=1.05, courant_c=8.0, **MIXED)
    tc, ms = binding.Solver(net_tcgen05=1, **kw), binding.Solver(net_tcgen05=0, **kw)
    net, _ = random_net(n_r, 64, seed=inputs.SEED_LEARNED + 90 + n_r)
    for role, level in ((binding.TPMG_NET_COARSE, 0), (binding.TPMG_NET_WARM, kw["n_levels"] - 1)):
        n = tc.query(level)[0] * n_r
        f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_LEARNED + 91 + level, n)).cuda()
        outs = []
        for s in (tc, ms):
            s.attach_net(role, net)
            u = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            s.net_predict(role, f, u)
            torch.cuda.synchronize()
            outs.append(u.cpu().numpy())
            s.attach_net(role, None)
        a, b = outs
        assert np.all(np.isfinite(a))
        scale = np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= 2e-2 * scale, (role, np.max(np.abs(a - b)) / scale)
        assert np.mean(np.abs(a - b)) <= 1e-3 * np.mean(np.abs(b)), (role, np.mean(np.abs(a - b)))
    assert not tc.net_fault()


def _smooth_rhs(s, seed):
    fields = learned.SmoothFields(s, l_max=8)
    return fields, fields.field(seed)


def test_learned_solve_without_networks_equals_flexible_cg():
    """No network attached and u = 0: the learned solve is the mixed form's
    flexible CG with the same kernels in the same order -- bit for bit."""
    s = binding.Solver(**SMALL, **MIXED)
    _, f = _smooth_rhs(s, inputs.SEED_LEARNED + 60)
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    st1, it1, rel1, _ = s.solve(f, u1, rtol=1e-7, max_iter=100)
    st2, it2, rel2, info, fb, launches = s.solve_learned(f, u2, rtol=1e-7, max_iter=100)
    assert (st1, it1) == (st2, it2) and fb == 0 and info == 0 and launches > 0
    # ||r_0||^2 (plain) and ||f||^2 (learned) are the same number summed by two kernels
    assert abs(rel1 - rel2) <= 1e-12 * rel1
    assert torch.equal(u1, u2)


def test_learned_host_loop_matches_device_loop():
    """graphs 0 (or a timed kernel class) runs the learned solve kernel by
    kernel from the host: same kernels, same order, same bits."""
    warm, _ = random_net(16, 64, seed=inputs.SEED_LEARNED + 90, scale=0.3)
    coarse, _ = random_net(16, 64, seed=inputs.SEED_LEARNED + 91, scale=0.3)
    outs = []
    for graphs in (1, 0):
        s = binding.Solver(graphs=graphs, **SMALL, **MIXED)
        _, f = _smooth_rhs(s, inputs.SEED_LEARNED + 92)
        s.attach_net(binding.TPMG_NET_WARM, warm)
        s.attach_net(binding.TPMG_NET_COARSE, coarse)
        u = torch.zeros_like(f)
        res = s.solve_learned(f, u, rtol=1e-8, max_iter=60)
        torch.cuda.synchronize()
        outs.append((res[:5], u.cpu().numpy()))
    assert outs[0][0] == outs[1][0], (outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_judge_rejects_a_useless_warm_start():
    """A network predicting a wildly wrong field: the judge replaces the guess
    by zero and the solve is the plain one, bit for bit.  A network predicting
    zero leaves one line relaxation from zero as the guess, which beats u = 0
    and is kept."""
    s = binding.Solver(**SMALL, **MIXED)
    _, f = _smooth_rhs(s, inputs.SEED_LEARNED + 61)
    ref = torch.zeros_like(f)
    _, it_ref, _, _ = s.solve(f, ref, rtol=1e-7, max_iter=100)
    net, _ = random_net(s.n_r, 64, seed=inputs.SEED_LEARNED + 62, scale=300.0)
    s.attach_net(binding.TPMG_NET_WARM, net)
    u = torch.full_like(f, 7.0)   # ignored: the network gives the initial guess
    st, it, rel, info, fb, _ = s.solve_learned(f, u, rtol=1e-7, max_iter=100)
    assert st == binding.TPMG_OK and info == binding.TPMG_LEARNED_WARM_REJECTED and fb == 0
    assert it == it_ref and rel <= 1e-7
    assert torch.equal(u, ref)
    zero, _ = random_net(s.n_r, 64, seed=inputs.SEED_LEARNED + 62, scale=0.0)
    s.attach_net(binding.TPMG_NET_WARM, zero)
    u = torch.zeros_like(f)
    st, it, rel, info, fb, _ = s.solve_learned(f, u, rtol=1e-7, max_iter=100)
    assert st == binding.TPMG_OK and info == binding.TPMG_LEARNED_WARM_USED and fb == 0 and rel <= 1e-7
    print(f"\nzero network + one line relaxation as initial guess: {it} iterations (plain {it_ref})")
    s.attach_net(binding.TPMG_NET_WARM, None)


def test_fallback_after_a_breakdown_restarts_plain_tpmg():
    """A coarse network whose output overflows FP32 makes the preconditioned
    residual non-finite in the first iteration (breakdown): plain TPMG-PCG
    restarts from u = 0 and reaches the tolerance relative to ||f||."""
    s = binding.Solver(**SMALL, **MIXED)
    _, f = _smooth_rhs(s, inputs.SEED_LEARNED + 63)
    ref = torch.zeros_like(f)
    _, it_ref, _, _ = s.solve(f, ref, rtol=1e-8, max_iter=50)
    net, _ = random_net(s.n_r, 64, seed=inputs.SEED_LEARNED + 64, scale=1e15)
    s.attach_net(binding.TPMG_NET_COARSE, net)
    u = torch.zeros_like(f)
    st, it, rel, info, fb, _ = s.solve_learned(f, u, rtol=1e-8, max_iter=50)
    assert st == binding.TPMG_OK and info == binding.TPMG_LEARNED_FALLBACK
    assert fb == it_ref and it == fb + 1 and rel <= 1e-8
    assert torch.equal(u, ref)   # the fallback is the plain solve from zero


def test_fallback_finishes_what_the_network_cannot():
    """An untrained coarse network: the learned phase either converges or, after
    max_iter iterations, plain TPMG-PCG continues from its iterate; either way
    the true residual meets the tolerance relative to ||f||."""
    s = binding.Solver(**SMALL, **MIXED)
    _, f = _smooth_rhs(s, inputs.SEED_LEARNED + 65)
    net, _ = random_net(s.n_r, 64, seed=inputs.SEED_LEARNED + 66)
    s.attach_net(binding.TPMG_NET_COARSE, net)
    u = torch.zeros_like(f)
    st, it, rel, info, fb, _ = s.solve_learned(f, u, rtol=1e-8, max_iter=12)
    print(f"\nuntrained coarse network: {it} iterations, {fb} of them in the fallback, info {info}")
    assert st == binding.TPMG_OK and rel <= 1e-8
    assert (fb > 0) == bool(info & binding.TPMG_LEARNED_FALLBACK)
    r = torch.zeros_like(f)
    s.apply_operator(u, r)
    assert float(torch.linalg.norm(f - r) / torch.linalg.norm(f)) <= 1e-7


def test_trained_networks_reach_the_tolerance_and_report_their_gain():
    """Networks trained on solves of the method (small grid, 64 pairs): the
    learned solve reaches the same ||r|| <= 1e-5 ||f|| on held-out smooth
    right-hand sides; the warm start beats u = 0 on its initial residual.
    Iterations with and without the networks are printed."""
    kw = dict(SMALL, **MIXED)
    data_solver = binding.Solver(graphs=0, **kw)
    fields = learned.SmoothFields(data_solver, l_max=8)
    data = learned.generate(data_solver, fields, n_pairs=64, seed=inputs.SEED_LEARNED + 1000, cells_per_pair=256,
                            coarse_per_pair=2)
    warm = binding.Net(data_solver.n_r, 64)
    warm.set_params(learned.init_params(warm.sizes, inputs.SEED_LEARNED + 70))
    tw = learned.train(warm, data["xw"], data["tw"], steps=800, seed=inputs.SEED_LEARNED + 71, batch=1024)
    coarse = binding.Net(data_solver.n_r, 64)
    coarse.set_params(learned.init_params(coarse.sizes, inputs.SEED_LEARNED + 72))
    tc = learned.train(coarse, data["xc"], data["tc"], steps=800, seed=inputs.SEED_LEARNED + 73, batch=1024)
    var_w = float(data["tw"].double().pow(2).mean())
    var_c = float(data["tc"].double().pow(2).mean())
    print(f"\nwarm: loss {tw['history'][0][1]:.3e} -> {tw['final']:.3e} (target mean square {var_w:.3e}); "
          f"coarse: loss {tc['history'][0][1]:.3e} -> {tc['final']:.3e} (target mean square {var_c:.3e})")
    assert tw["final"] < tw["history"][0][1] and tc["final"] < tc["history"][0][1]
    s = binding.Solver(**kw)
    rows = []
    for j in range(4):
        f = fields.field(inputs.SEED_LEARNED + 5000 + j)   # held out
        u = torch.zeros_like(f)
        _, it_plain, rel_plain, _ = s.solve(f, u, rtol=1e-5, max_iter=100)
        res = {}
        for name, nets in (("warm", (None, warm)), ("coarse", (coarse, None)), ("both", (coarse, warm))):
            s.attach_net(binding.TPMG_NET_COARSE, nets[0])
            s.attach_net(binding.TPMG_NET_WARM, nets[1])
            u = torch.zeros_like(f)
            st, it, rel, info, fb, _ = s.solve_learned(f, u, rtol=1e-5, max_iter=100)
            assert st == binding.TPMG_OK and rel <= 1e-5
            r = torch.zeros_like(f)
            s.apply_operator(u, r)
            assert float(torch.linalg.norm(f - r) / torch.linalg.norm(f)) <= 2e-5
            res[name] = (it, info, fb)
        s.attach_net(binding.TPMG_NET_COARSE, None)
        s.attach_net(binding.TPMG_NET_WARM, None)
        # initial residual of the warm start alone
        s.attach_net(binding.TPMG_NET_WARM, warm)
        u = torch.zeros_like(f)
        s.solve_learned(f, u, rtol=1.0, max_iter=1)
        s.attach_net(binding.TPMG_NET_WARM, None)
        r = torch.zeros_like(f)
        s.apply_operator(u, r)
        r0 = float(torch.linalg.norm(f - r) / torch.linalg.norm(f))
        rows.append((it_plain, res, r0))
    print("\nplain iterations | warm / coarse / both (iters, info, fallback) | warm-start ||r0||/||f||")
    for it_plain, res, r0 in rows:
        print(f"  {it_plain} | {res['warm']} {res['coarse']} {res['both']} | {r0:.3e}")
    assert all(r0 < 1.0 for _, _, r0 in rows)


def test_trained_warm_start_saves_iterations():
    """The warm start pays where the fields it learns are resolved by the grid: on
    refinement 5 x 32 levels with right-hand sides of degree <= 4, a network trained
    on 200 solves of the method saves at least one of plain mixed TPMG-PCG's
    iterations on every held-out field, at the same ||r|| <= 1e-5 ||f|| (checked on
    the true residual).  (On the smaller grid of the test above, whose fields vary
    on the scale of the 1-ring, the per-column network saves nothing.)"""
    kw = dict(refinement=5, n_levels=6, n_r=32, grading=1.05, courant_c=8.0, **MIXED)
    data_solver = binding.Solver(graphs=0, **kw)
    fields = learned.SmoothFields(data_solver, l_max=4)
    data = learned.generate(data_solver, fields, n_pairs=200, seed=inputs.SEED_LEARNED + 1000, cells_per_pair=256,
                            coarse_per_pair=2)
    warm = binding.Net(data_solver.n_r, 64)
    warm.set_params(learned.init_params(warm.sizes, inputs.SEED_LEARNED + 70))
    tw = learned.train(warm, data["xw"], data["tw"], steps=800, seed=inputs.SEED_LEARNED + 71, batch=1024)
    assert tw["final"] < 1e-2 * tw["history"][0][1]
    s = binding.Solver(**kw)
    rows = []
    for j in range(6):
        f = fields.field(inputs.SEED_LEARNED + 5000 + j)   # held out
        u = torch.zeros_like(f)
        st, it_plain, rel_plain, _ = s.solve(f, u, rtol=1e-5, max_iter=100)
        assert st == binding.TPMG_OK
        s.attach_net(binding.TPMG_NET_WARM, warm)
        u = torch.zeros_like(f)
        st, it, rel, info, fb, _ = s.solve_learned(f, u, rtol=1e-5, max_iter=100)
        s.attach_net(binding.TPMG_NET_WARM, None)
        assert st == binding.TPMG_OK and rel <= 1e-5
        assert info & binding.TPMG_LEARNED_WARM_USED and fb == 0   # the judge kept the guess, no fallback
        r = torch.zeros_like(f)
        s.apply_operator(u, r)
        assert float(torch.linalg.norm(f - r) / torch.linalg.norm(f)) <= 2e-5
        rows.append((it_plain, it))
    print(f"\nwarm start on refinement 5 x 32 (l <= 4): iterations plain -> learned {rows}")
    assert all(it <= it_plain - 1 for it_plain, it in rows), rows
