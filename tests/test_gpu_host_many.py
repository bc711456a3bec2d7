"""Pipelined solves with host buffers (tpmg_solve_host_many) through the C ABI (needs a GPU).

Each system is tpmg_solve's PCG (Sec. 5) on one of two staging slots, so its
solution, iteration count and residual must equal those of tpmg_solve on the
same right-hand side and guess bit for bit; one system is also compared with
the oracle's PCG at the path's 1e-10 relative solution error.
"""
import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64 = dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1)
MIXED = dict(refinement=4, n_levels=4, n_r=32, grading=1.05, courant_c=80.0, precision=1, coeff_storage=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def pinned(a):
    t = torch.empty(a.size, dtype=torch.float64, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def device_solve(s, f, u0, rtol, max_iter):
    u = torch.from_numpy(np.ascontiguousarray(u0)).to("cuda")
    st, it, rel, _ = s.solve(torch.from_numpy(np.ascontiguousarray(f)).to("cuda"), u, rtol=rtol, max_iter=max_iter,
                             raise_on_fail=False)
    torch.cuda.synchronize()
    return st, it, rel, u.cpu().numpy()


def rhs(s, j):
    return inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 40 + j, s.N)


@pytest.mark.parametrize("kw", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n", [1, 2, 5])
def test_zero_guess_matches_device_solves(kw, n):
    s = binding.Solver(**kw)
    fs_np = [rhs(s, j % 3) for j in range(n)]   # repeated right-hand sides are allowed
    fs = [pinned(f) for f in fs_np]
    us = [pinned(np.full(s.N, 7.0)) for _ in range(n)]   # overwritten: the guess is zero
    st, it, rel, sts = s.solve_host_many([t.numpy() for t in fs], [t.numpy() for t in us], guess=False, rtol=1e-8)
    assert st == binding.TPMG_OK and list(sts) == [binding.TPMG_OK] * n
    for j in range(n):
        st2, it2, rel2, u2 = device_solve(s, fs_np[j], np.zeros(s.N), 1e-8, 100)
        assert (st2, it2, rel2) == (binding.TPMG_OK, it[j], rel[j])
        np.testing.assert_array_equal(us[j].numpy(), u2)


@pytest.mark.parametrize("pin", [True, False], ids=["pinned", "pageable"])
def test_initial_guesses_are_copied_in(pin):
    s = binding.Solver(**FP64)
    n = 4
    fs = [rhs(s, j) for j in range(n)]
    g = [inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 60 + j, s.N) * 0.1 for j in range(n)]
    us = [pinned(x).numpy() if pin else x.copy() for x in g]
    st, it, rel, sts = s.solve_host_many(fs, us, guess=True, rtol=1e-7)
    assert st == binding.TPMG_OK
    for j in range(n):
        st2, it2, rel2, u2 = device_solve(s, fs[j], g[j], 1e-7, 100)
        assert (st2, it2, rel2) == (binding.TPMG_OK, it[j], rel[j])
        np.testing.assert_array_equal(us[j], u2)


def test_one_system_against_the_oracle():
    s, o = binding.Solver(**FP64), oracle.Oracle(**FP64)
    fs = [rhs(s, 0), rhs(s, 1), rhs(s, 2)]
    us = [np.zeros(s.N) for _ in fs]
    st, it, rel, _ = s.solve_host_many(fs, us, rtol=0.0, max_iter=6, raise_on_fail=False)
    # rtol 0 with a fixed count: every system runs exactly 6 iterations, as the oracle does
    assert st == binding.TPMG_ERR_NOT_CONVERGED and list(it) == [6, 6, 6]
    ro = o.pcg(fs[1], rtol=0.0, max_iter=6)
    assert ro["iters"] == 6
    err = np.linalg.norm(us[1] - ro["u"]) / np.linalg.norm(ro["u"])
    assert err <= 1e-10, err


def test_failed_systems_do_not_stop_the_others():
    s = binding.Solver(**FP64)
    f_ok = rhs(s, 0)
    f_nan = np.ones(s.N)
    f_nan[5] = np.nan
    fs = [f_ok, np.zeros(s.N), f_nan, f_ok]
    us = [np.zeros(s.N) for _ in fs]
    st, it, rel, sts = s.solve_host_many(fs, us, rtol=1e-8, raise_on_fail=False)
    assert st == binding.TPMG_ERR_BREAKDOWN
    assert list(sts) == [binding.TPMG_OK, binding.TPMG_OK, binding.TPMG_ERR_BREAKDOWN, binding.TPMG_OK]
    assert it[1] == 0 and rel[1] == 0.0 and not np.any(us[1])
    _, it2, _, u2 = device_solve(s, f_ok, np.zeros(s.N), 1e-8, 100)
    assert it[0] == it[3] == it2
    np.testing.assert_array_equal(us[0], u2)
    np.testing.assert_array_equal(us[3], u2)


def test_rejected_arguments_launch_nothing():
    s = binding.Solver(**FP64)
    f = rhs(s, 0)
    u = np.zeros(s.N)
    with pytest.raises(binding.TPMGError):
        s.solve_host_many([f, f], [u, u])          # one solution array for two systems
    v = np.zeros(s.N)
    with pytest.raises(binding.TPMGError):
        s.solve_host_many([f, v], [v, u])          # a solution array that is another system's input
    assert not np.any(u) and not np.any(v)
    st, it, rel, sts = s.solve_host_many([], [])
    assert st == binding.TPMG_OK and len(it) == 0


def test_device_solves_in_between_keep_their_graphs():
    """Host solves alternate two staging slots; a device solve on other vectors in
    between captures a graph of its own, and every result stays the same."""
    s = binding.Solver(**FP64)
    fs = [rhs(s, j) for j in range(3)]
    ref = []
    for f in fs:
        ref.append(device_solve(s, f, np.zeros(s.N), 1e-8, 100))
    for _ in range(2):
        us = [np.zeros(s.N) for _ in fs]
        s.solve_host_many(fs, us, rtol=1e-8)
        for j in range(3):
            np.testing.assert_array_equal(us[j], ref[j][3])
        st, it, rel, u = device_solve(s, fs[1], np.zeros(s.N), 1e-8, 100)
        np.testing.assert_array_equal(u, ref[1][3])


def test_host_driven_loop_gives_the_same_results():
    """Without graphs each system's solve returns before the next is enqueued; the
    results are those of the same context's device solves."""
    s = binding.Solver(graphs=0, **FP64)
    fs = [rhs(s, j) for j in range(3)]
    us = [np.zeros(s.N) for _ in fs]
    st, it, rel, sts = s.solve_host_many(fs, us, rtol=1e-8)
    assert st == binding.TPMG_OK
    for j in range(3):
        st2, it2, rel2, u2 = device_solve(s, fs[j], np.zeros(s.N), 1e-8, 100)
        assert (it2, rel2) == (it[j], rel[j])
        np.testing.assert_array_equal(us[j], u2)
