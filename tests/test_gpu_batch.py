"""Batched form: many independent solves in one graph launch (tpmg_batch_*),
through the C ABI (needs a GPU).

A batched solve runs the same kernels in the same order as tpmg_solve, with
its loop on the device, so every problem's solution and iteration count must
equal those of its own solve bit for bit (the solve itself is checked against
the oracle by the parity tests).
"""
import numpy as np
import pytest

from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)

PROBLEMS = [
    dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1),
    dict(refinement=4, n_levels=5, n_r=32, grading=1.05, courant_c=80.0),
    dict(refinement=2, n_levels=3, n_r=7, grading=1.1, courant_c=20.0, smoother=1, relax=0.6),
    dict(refinement=4, n_levels=4, n_r=64, grading=1.05, courant_c=150.0, **MIXED),
    dict(refinement=3, n_levels=2, n_r=128, grading=1.02, courant_c=4.0, **MIXED),
    dict(refinement=1, n_levels=2, n_r=33, courant_c=30.0),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rhs(s, j):
    return torch.from_numpy(inputs.uniform_pm1(inputs.SEED_BATCH + j, s.N)).cuda()


def test_batch_matches_individual_solves():
    solvers = [binding.Solver(**kw) for kw in PROBLEMS]
    fs = [rhs(s, j) for j, s in enumerate(solvers)]
    us = [torch.zeros_like(f) for f in fs]
    b = binding.Batch(solvers, fs, us, rtol=1e-6, max_iter=100)
    for rep in range(2):   # a second run from zero guesses repeats the first
        for u in us:
            u.zero_()
        st, it, rel, sts, launches = b.run()
        torch.cuda.synchronize()
        assert st == binding.TPMG_OK and np.all(sts == binding.TPMG_OK) and launches > 0
        for j, (kw, f, u) in enumerate(zip(PROBLEMS, fs, us)):
            ref = binding.Solver(graphs=0, **kw)
            u_ref = torch.zeros_like(f)
            st_r, it_r, rel_r, _ = ref.solve(f, u_ref, rtol=1e-6, max_iter=100)
            assert (st_r, it_r) == (binding.TPMG_OK, it[j]), (j, it_r, it[j])
            assert rel_r == rel[j]
            assert torch.equal(u, u_ref), j


def test_batch_problems_match_the_oracle():
    """Batched solves against the CPU oracle directly (not only against the
    library's own solves): an FP64 problem reaches the oracle's PCG solution to
    the 1e-10 relative solution error of the FP64 parity tests, and a
    mixed-precision problem takes the oracle's flexible-CG iterations with the
    BF16 V-cycle (up to one at the stopping boundary) and, solved tightly,
    reaches the FP64 oracle solution to 1e-9 in the energy norm."""
    import oracle

    oracle.build()
    kw64, kwmx = PROBLEMS[1], PROBLEMS[3]
    o64 = oracle.Oracle(**kw64)
    omx = oracle.Oracle(**{k: v for k, v in kwmx.items() if k not in ("precision", "coeff_storage")})

    def run(rtol):
        solvers = [binding.Solver(**kw64), binding.Solver(**kwmx)]
        fs = [rhs(s, 20 + j) for j, s in enumerate(solvers)]
        us = [torch.zeros_like(f) for f in fs]
        st, it, rel, sts, _ = binding.Batch(solvers, fs, us, rtol=rtol, max_iter=300).run()
        torch.cuda.synchronize()
        assert st == binding.TPMG_OK and np.all(sts == binding.TPMG_OK)
        return [f.cpu().numpy() for f in fs], [u.cpu().numpy() for u in us], it

    fs, us, it = run(1e-11)
    r64 = o64.pcg(fs[0], rtol=1e-11, max_iter=300)
    err64 = np.linalg.norm(us[0] - r64["u"]) / np.linalg.norm(r64["u"])
    rmx = omx.pcg(fs[1], rtol=1e-11, max_iter=300)
    e = us[1] - rmx["u"]
    errmx = np.sqrt(max(e @ omx.apply(e), 0.0)) / np.sqrt(rmx["u"] @ omx.apply(rmx["u"]))
    print(f"FP64 member: {it[0]} iterations (oracle {r64['iters']}), rel. solution error {err64:.2e}; "
          f"mixed member: {it[1]} iterations (FP64 oracle {rmx['iters']}), energy-norm rel. error {errmx:.2e}")
    assert err64 <= 1e-10, err64
    assert errmx <= 1e-9, errmx

    fs, us, it = run(1e-5)
    omx.set_vcycle_bf16(True)
    flex = omx.pcg(fs[1], rtol=1e-5, max_iter=100, flexible=True)
    print(f"mixed member at 1e-5: {it[1]} iterations, oracle flexible CG with the BF16 V-cycle {flex['iters']}")
    assert abs(int(it[1]) - flex["iters"]) <= 1


def test_batch_reports_each_problem():
    solvers = [binding.Solver(**kw) for kw in PROBLEMS[:3]]
    fs = [rhs(s, j) for j, s in enumerate(solvers)]
    fs[1] = torch.zeros_like(fs[1])          # zero right-hand side: done in 0 iterations
    us = [torch.zeros_like(f) for f in fs]
    b = binding.Batch(solvers, fs, us, rtol=1e-12, max_iter=3)
    st, it, rel, sts, _ = b.run()
    assert sts[1] == binding.TPMG_OK and it[1] == 0 and rel[1] == 0.0
    assert sts[0] == binding.TPMG_ERR_NOT_CONVERGED and it[0] == 3 and rel[0] > 1e-12
    assert st == binding.TPMG_ERR_NOT_CONVERGED


def test_batch_rejects_a_repeated_context():
    s = binding.Solver(**PROBLEMS[0])
    f = rhs(s, 0)
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    with pytest.raises(binding.TPMGError) as exc:
        binding.Batch([s, s], [f, f], [u1, u2])
    assert exc.value.status == binding.TPMG_ERR_INVALID_ARG


def test_device_loop_solve_matches_host_loop():
    """tpmg_solve with graphs on runs its loop on the device; with graphs off the
    host drives it: same kernels, same order, same bits."""
    for kw in PROBLEMS:
        outs = []
        for graphs in (0, 1):
            s = binding.Solver(graphs=graphs, **kw)
            f = rhs(s, 9)
            u = torch.zeros_like(f)
            st, it, rel, hist = s.solve(f, u, rtol=1e-8, max_iter=200, history=True)
            torch.cuda.synchronize()
            outs.append((st, it, rel, hist, u.cpu().numpy()))
        (a, b) = outs
        assert a[:3] == b[:3]
        np.testing.assert_array_equal(a[3], b[3])
        np.testing.assert_array_equal(a[4], b[4])


def test_autotuned_kernels_give_identical_results():
    """The autotuner picks among relaxation kernels that do the same arithmetic
    in the same order, so tuned and untuned solves agree bit for bit."""
    for kw in (PROBLEMS[1], PROBLEMS[3], PROBLEMS[4]):
        outs = []
        for tune in (0, 1):
            s = binding.Solver(autotune=tune, **kw)
            tuning = s.tuning()
            assert len(tuning) == s.n_levels
            if tune:
                mixed = kw.get("precision", 0) == binding.TPMG_PREC_MIXED
                for variant, us in tuning:
                    # the warp-scan levels (every FP32 level) have four CTA shapes
                    tried = us[:4] if (mixed or us[4] == 0.0) else us
                    assert variant in range(len(tried)) and all(t > 0 for t in tried)
                    assert us[variant] == min(tried)
                    if mixed:
                        assert us[4] == 0.0
            else:
                assert all(v == -1 for v, _ in tuning)
            f = rhs(s, 11)
            u = torch.zeros_like(f)
            st, it, rel, _ = s.solve(f, u, rtol=1e-8, max_iter=200)
            torch.cuda.synchronize()
            outs.append((st, it, rel, u.cpu().numpy()))
        assert outs[0][:3] == outs[1][:3]
        np.testing.assert_array_equal(outs[0][3], outs[1][3])


# Mixed-precision CG problems: the work-list form.  Different numbers of levels (so the
# schedule aligns members of 1 to 5 levels at the coarsest), column heights in three
# rows-per-lane classes (7 and 32: one row per lane; 33 and 64: two; 128: four),
# block-SOR and block Jacobi, a single-level problem and a relaxation weight != 1.
WORKLIST = [
    dict(refinement=4, n_levels=5, n_r=64, grading=1.05, courant_c=150.0, **MIXED),
    dict(refinement=3, n_levels=2, n_r=128, grading=1.02, courant_c=4.0, **MIXED),
    dict(refinement=3, n_levels=4, n_r=32, courant_c=8.0, nu_pre=1, nu_post=1, **MIXED),
    dict(refinement=2, n_levels=3, n_r=7, grading=1.1, courant_c=20.0, smoother=1, relax=0.6, **MIXED),
    dict(refinement=1, n_levels=2, n_r=33, courant_c=30.0, nu_coarse=2, **MIXED),
    dict(refinement=0, n_levels=1, n_r=16, courant_c=8.0, **MIXED),
]


def own_solve(kw, f, rtol, max_iter=100):
    ref = binding.Solver(**kw)
    u = torch.zeros_like(f)
    st, it, rel, _ = ref.solve(f, u, rtol=rtol, max_iter=max_iter, raise_on_fail=False)
    torch.cuda.synchronize()
    return st, it, rel, u


@pytest.mark.parametrize("groups", [1, 0, 6])   # all members in one schedule, the default, one each
def test_worklist_batch_matches_individual_solves(groups):
    solvers = [binding.Solver(**kw) for kw in WORKLIST]
    fs = [rhs(s, 30 + j) for j, s in enumerate(solvers)]
    us = [torch.zeros_like(f) for f in fs]
    b = binding.Batch(solvers, fs, us, rtol=1e-6, max_iter=100, form="worklist", groups=groups)
    assert b.form == "worklist"
    for rep in range(2):   # a second run from zero guesses repeats the first
        for u in us:
            u.zero_()
        st, it, rel, sts, launches = b.run()
        torch.cuda.synchronize()
        assert st == binding.TPMG_OK and np.all(sts == binding.TPMG_OK) and launches > 0
        for j, (kw, f, u) in enumerate(zip(WORKLIST, fs, us)):
            st_r, it_r, rel_r, u_ref = own_solve(kw, f, 1e-6)
            assert (st_r, it_r) == (binding.TPMG_OK, it[j]), (j, it_r, it[j])
            assert rel_r == rel[j], j
            assert torch.equal(u, u_ref), j


def test_worklist_batch_many_right_hand_sides_on_one_operator():
    """Several right-hand sides on one context share its grid, stencil and factors;
    each gets its own work vectors and its own solve's bits, interleaved with a
    second operator's right-hand sides."""
    a, c = binding.Solver(**WORKLIST[0]), binding.Solver(**WORKLIST[2])
    solvers = [a, c, a, a, c]
    fs = [rhs(s, 40 + j) for j, s in enumerate(solvers)]
    us = [torch.zeros_like(f) for f in fs]
    b = binding.Batch(solvers, fs, us, rtol=1e-7, max_iter=100)
    assert b.form == "worklist"   # a repeated context takes the work list automatically
    st, it, rel, sts, _ = b.run()
    torch.cuda.synchronize()
    assert st == binding.TPMG_OK
    kws = [WORKLIST[0], WORKLIST[2], WORKLIST[0], WORKLIST[0], WORKLIST[2]]
    for j, (kw, f, u) in enumerate(zip(kws, fs, us)):
        st_r, it_r, rel_r, u_ref = own_solve(kw, f, 1e-7)
        assert (st_r, it_r, rel_r) == (binding.TPMG_OK, it[j], rel[j]), j
        assert torch.equal(u, u_ref), j


def test_worklist_batch_reports_each_problem():
    solvers = [binding.Solver(**kw) for kw in WORKLIST[:3]]
    fs = [rhs(s, j) for j, s in enumerate(solvers)]
    fs[1] = torch.zeros_like(fs[1])          # zero right-hand side: done in 0 iterations
    us = [torch.zeros_like(f) for f in fs]
    b = binding.Batch(solvers, fs, us, rtol=1e-12, max_iter=3, form="worklist", groups=2)
    assert b.form == "worklist"
    st, it, rel, sts, _ = b.run()
    assert sts[1] == binding.TPMG_OK and it[1] == 0 and rel[1] == 0.0
    assert sts[0] == binding.TPMG_ERR_NOT_CONVERGED and it[0] == 3 and rel[0] > 1e-12
    assert st == binding.TPMG_ERR_NOT_CONVERGED
    # a member stopped early keeps its own solve's iterate: the solve with max_iter = 3
    for j in (0, 2):
        st_r, it_r, rel_r, u_ref = own_solve(WORKLIST[j], fs[j], 1e-12, max_iter=3)
        assert it_r == it[j] and rel_r == rel[j] and torch.equal(us[j], u_ref), j


def test_worklist_batch_member_matches_the_oracle():
    """A work-list member against the CPU oracle directly: the flexible-CG
    iterations with the BF16 V-cycle at 1e-5 (up to one at the stopping
    boundary), and the FP64 oracle solution to 1e-9 in the energy norm when
    solved tightly."""
    import oracle

    oracle.build()
    kw = WORKLIST[0]
    o = oracle.Oracle(**{k: v for k, v in kw.items() if k not in ("precision", "coeff_storage")})
    a, c = binding.Solver(**kw), binding.Solver(**WORKLIST[1])
    for rtol in (1e-11, 1e-5):
        fs = [rhs(a, 50), rhs(c, 51)]
        us = [torch.zeros_like(f) for f in fs]
        st, it, rel, sts, _ = binding.Batch([a, c], fs, us, rtol=rtol, max_iter=300, form="worklist").run()
        torch.cuda.synchronize()
        assert sts[0] == binding.TPMG_OK
        f0, u0 = fs[0].cpu().numpy(), us[0].cpu().numpy()
        if rtol < 1e-6:
            o.set_vcycle_bf16(False)
            ro = o.pcg(f0, rtol=1e-11, max_iter=300)
            e = u0 - ro["u"]
            err = np.sqrt(max(e @ o.apply(e), 0.0)) / np.sqrt(ro["u"] @ o.apply(ro["u"]))
            print(f"work-list member: {it[0]} iterations, FP64 oracle {ro['iters']}, energy-norm rel. error {err:.2e}")
            assert err <= 1e-9, err
        else:
            o.set_vcycle_bf16(True)
            flex = o.pcg(f0, rtol=1e-5, max_iter=100, flexible=True)
            print(f"work-list member at 1e-5: {it[0]} iterations, oracle flexible CG (BF16 V-cycle) {flex['iters']}")
            assert abs(int(it[0]) - flex["iters"]) <= 1


def test_batch_form_follows_the_members():
    mixed, mixed2 = binding.Solver(**WORKLIST[2]), binding.Solver(**WORKLIST[1])
    fp64 = binding.Solver(**PROBLEMS[0])
    f1, f2, f3 = rhs(mixed, 0), rhs(fp64, 0), rhs(mixed2, 0)
    z = torch.zeros_like
    assert binding.Batch([mixed, fp64], [f1, f2], [z(f1), z(f2)]).form == "branches"
    assert binding.Batch([mixed, mixed2], [f1, f3], [z(f1), z(f3)]).form == "branches"   # distinct contexts
    assert binding.Batch([mixed, mixed2], [f1, f3], [z(f1), z(f3)], form="worklist").form == "worklist"
    with pytest.raises(binding.TPMGError):   # an FP64 member cannot join the work list
        binding.Batch([mixed, fp64], [f1, f2], [z(f1), z(f2)], form="worklist")
    u1, u2 = torch.zeros_like(f1), torch.zeros_like(f1)
    with pytest.raises(binding.TPMGError) as exc:   # two members writing one solution vector
        binding.Batch([mixed, mixed], [f1, f1.clone()], [u1, u1])
    assert exc.value.status == binding.TPMG_ERR_INVALID_ARG
