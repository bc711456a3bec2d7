"""Mixed-precision form (FP32 V-cycle on a BF16 stencil, FP64 outer flexible CG)
against the CPU oracle, through the C ABI (needs a GPU).

Two oracle references separate the two sources of difference:
* the oracle's V-cycle with the same BF16-rounded coefficients in FP64
  arithmetic: the GPU differs from it only by FP32 rounding (unit 2^-24);
* the oracle's FP64 solve: the mixed solve reaches it because the outer
  residual and update are FP64 with the exact operator.
Measured errors are printed so the stated bounds can be checked against them.
"""
import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)

CASES = {
    "ref3_nr16_uniform_c8_nu1": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1),
    "ref2_nr7_graded_c80_nu2": dict(refinement=2, n_levels=3, n_r=7, grading=1.1, courant_c=80.0),
    "ref0_nr1_single_level": dict(refinement=0, n_levels=1, n_r=1, courant_c=8.0),
    "ref1_nr33_jacobi": dict(refinement=1, n_levels=2, n_r=33, courant_c=20.0, smoother=1, relax=0.6, nu_pre=1,
                             nu_post=1, nu_coarse=2),
    "ref2_nr200_tall": dict(refinement=2, n_levels=3, n_r=200, grading=1.02, courant_c=8.0, nu_pre=1, nu_post=1),
    "ref4_nr64_graded_c80": dict(refinement=4, n_levels=5, n_r=64, grading=1.05, courant_c=80.0),
    # columns of exactly 128 rows: 4 rows per lane with 16-byte accesses; 100 rows: the
    # segmented layout of the same rows-per-lane class
    "ref3_nr128_graded_c80": dict(refinement=3, n_levels=4, n_r=128, grading=1.02, courant_c=80.0),
    "ref3_nr128_graded_c8": dict(refinement=3, n_levels=4, n_r=128, grading=1.02, courant_c=8.0),
    "ref2_nr100_graded_c8": dict(refinement=2, n_levels=3, n_r=100, grading=1.03, courant_c=8.0),
    # weighted block-Jacobi (relax != 1, a second buffer) in the wide-access layouts
    "ref2_nr64_jacobi": dict(refinement=2, n_levels=3, n_r=64, courant_c=20.0, smoother=1, relax=0.6, nu_pre=1,
                             nu_post=1, nu_coarse=2),
    "ref2_nr128_jacobi_relax07": dict(refinement=2, n_levels=3, n_r=128, grading=1.02, courant_c=8.0, smoother=1,
                                      relax=0.7, nu_pre=2, nu_post=2, nu_coarse=2),
    "ref2_nr128_sor_relax08": dict(refinement=2, n_levels=3, n_r=128, courant_c=8.0, relax=0.8, nu_pre=1,
                                   nu_post=1, nu_coarse=1),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def energy(o, e):
    return float(np.sqrt(max(e @ o.apply(e), 0.0)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_vcycle_vs_oracle_bf16(name):
    kw = CASES[name]
    s, o = binding.Solver(**MIXED, **kw), oracle.Oracle(**kw)
    o.set_vcycle_bf16(True)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 8, s.N)
    z = torch.full((s.N,), float("nan"), dtype=torch.float64, device="cuda")
    s.vcycle(cuda(r), z)
    zg, zo = host(z), o.vcycle(r)
    assert np.all(np.isfinite(zg))
    rel = energy(o, zg - zo) / energy(o, zo)
    print(f"{name}: FP32 V-cycle vs BF16-coefficient oracle V-cycle, energy-norm rel. error {rel:.2e}")
    # FP32 rounding of the line solves is amplified by cond(A_T) (1e6-1e9): measured
    # 6.6e-8 (one column of one level) to 1.35e-3 (200 levels); an O(1) mistake is far above
    assert rel <= 5e-3, rel


@pytest.mark.parametrize("name", ["ref3_nr16_uniform_c8_nu1", "ref2_nr7_graded_c80_nu2", "ref4_nr64_graded_c80",
                                  "ref3_nr128_graded_c80"])
def test_mixed_solve_reaches_fp64_solution(name):
    kw = CASES[name]
    s, o = binding.Solver(**MIXED, **kw), oracle.Oracle(**kw)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 1, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(cuda(f), u, rtol=1e-11, max_iter=300)
    ro = o.pcg(f, rtol=1e-11, max_iter=300)
    assert st == binding.TPMG_OK and ro["status"] == 0
    ug = host(u)
    err_a = energy(o, ug - ro["u"]) / energy(o, ro["u"])
    print(f"{name}: mixed {it} iterations, FP64 oracle {ro['iters']}; energy-norm rel. error {err_a:.2e}")
    assert err_a <= 1e-9, err_a


@pytest.mark.parametrize("name", ["ref3_nr16_uniform_c8_nu1", "ref2_nr7_graded_c80_nu2", "ref4_nr64_graded_c80",
                                  "ref3_nr128_graded_c8"])
def test_mixed_iterations_match_oracle_flexible_bf16(name):
    """At the paper's 1e-5 reduction the mixed solve takes the oracle's flexible
    CG iterations with the BF16 V-cycle (up to one at the stopping boundary) and
    no more than one iteration beyond plain FP64 PCG.  Not asserted where the
    FP32 rounding of the line solves dominates the first iterations: at 128 rows
    and omega^2/h^2 = 80 on refinement 3 the mixed solve takes 7 iterations to the
    oracle's 5, with either row layout of the FP32 pass (measured), since the
    rounding noise of the column solves carries the large vertical couplings into
    the residual; that case is held to the FP64 solution instead."""
    kw = CASES[name]
    s, o = binding.Solver(**MIXED, **kw), oracle.Oracle(**kw)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, hist = s.solve(cuda(f), u, rtol=1e-5, max_iter=100, history=True)
    fp64 = o.pcg(f, rtol=1e-5, max_iter=100)
    o.set_vcycle_bf16(True)
    flex = o.pcg(f, rtol=1e-5, max_iter=100, flexible=True)
    ug = host(u)
    err = np.linalg.norm(ug - flex["u"]) / np.linalg.norm(flex["u"])
    err64 = np.linalg.norm(ug - fp64["u"]) / np.linalg.norm(fp64["u"])
    print(f"{name}: iterations mixed {it}, oracle flexible BF16 {flex['iters']}, oracle FP64 {fp64['iters']}; "
          f"rel. error vs flexible BF16 oracle {err:.2e}, vs FP64 oracle {err64:.2e}")
    assert st == binding.TPMG_OK and abs(it - flex["iters"]) <= 1 and it <= fp64["iters"] + 1
    assert rel <= 1e-5 and hist[-1] == rel
    # reported, not bounded: the FP32 V-cycle changes the residual of the last
    # iterations by up to a few times (measured 0.3-3.8x) while the stop agrees
    n = min(len(hist), len(flex["hist"]))
    dev = np.max(np.abs(hist[:n] / flex["hist"][:n] - 1.0))
    print(f"  max relative deviation of the residual history from the oracle's: {dev:.2e}")


# Grids whose finest level has 81,920 columns (refinement 6): the size at which the
# FP32 relaxation runs the finest level's passes in CTAs of several warps (as the
# autotuner chooses there; 4 warps without it) on the FP64 right-hand side, one
# column per warp.  n_r = 32 takes the one-row-per-lane layout, n_r = 64 the
# two-rows-per-lane one.
LARGE = {
    "ref6_nr32_graded_c80": dict(refinement=6, n_levels=6, n_r=32, grading=1.05, courant_c=80.0),
    "ref6_nr64_graded_c80": dict(refinement=6, n_levels=6, n_r=64, grading=1.05, courant_c=80.0),
}
_large_oracle = {}


def large_oracle(name):
    """The oracle and its BF16-coefficient V-cycle of the seeded residual (computed once)."""
    if name not in _large_oracle:
        o = oracle.Oracle(**LARGE[name])
        o.set_vcycle_bf16(True)
        r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 8, o.size())
        _large_oracle[name] = (o, r, o.vcycle(r))
    return _large_oracle[name]


@pytest.mark.parametrize("autotune", [0, 1])
@pytest.mark.parametrize("name", sorted(LARGE))
def test_mixed_vcycle_vs_oracle_bf16_81920_columns(name, autotune):
    o, r, zo = large_oracle(name)
    s = binding.Solver(autotune=autotune, **MIXED, **LARGE[name])
    assert s.N == r.size
    z = torch.full((s.N,), float("nan"), dtype=torch.float64, device="cuda")
    s.vcycle(cuda(r), z)
    zg = host(z)
    assert np.all(np.isfinite(zg))
    rel = energy(o, zg - zo) / energy(o, zo)
    finest = s.tuning()[-1][0]
    print(f"{name} autotune={autotune} (finest-level variant {finest}): FP32 V-cycle vs BF16-coefficient oracle "
          f"V-cycle, energy-norm rel. error {rel:.2e}")
    assert rel <= 5e-3, rel


def test_mixed_solve_reaches_fp64_solution_81920_columns():
    """The mixed solve on the refinement-6 grid reaches the FP64 oracle's PCG
    solution (1e-9 in the energy norm, as on the small grids)."""
    name = "ref6_nr32_graded_c80"
    o, _, _ = large_oracle(name)
    o.set_vcycle_bf16(False)
    try:
        s = binding.Solver(**MIXED, **LARGE[name])
        f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 1, s.N)
        u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        st, it, rel, _ = s.solve(cuda(f), u, rtol=1e-11, max_iter=300)
        ro = o.pcg(f, rtol=1e-11, max_iter=300)
    finally:
        o.set_vcycle_bf16(True)
    assert st == binding.TPMG_OK and ro["status"] == 0
    ug = host(u)
    err_a = energy(o, ug - ro["u"]) / energy(o, ro["u"])
    print(f"{name}: mixed {it} iterations, FP64 oracle {ro['iters']}; energy-norm rel. error {err_a:.2e}")
    assert err_a <= 1e-9, err_a


def test_mixed_rejects_factorised_storage():
    with pytest.raises(binding.TPMGError):
        binding.Solver(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FACTORISED, **CASES["ref0_nr1_single_level"])


def test_mixed_graph_replay_matches_direct():
    kw = CASES["ref4_nr64_graded_c80"]
    f = cuda(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 5, binding.Solver(**MIXED, **kw).N))
    outs = []
    for graphs in (0, 1):
        s = binding.Solver(graphs=graphs, **MIXED, **kw)
        for _ in range(2):
            u = torch.zeros_like(f)
            s.solve(f, u, rtol=1e-8)
            outs.append(host(u))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
