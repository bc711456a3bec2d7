"""Vertical advection (the -omega^2 xi_r d_r u term of Sec. 2, eq. HelmholtzVector,
centred as in Appendix A) on the GPU against the oracle, through the C ABI (needs a
GPU): the operator, the V-cycle of every coefficient storage and precision, and
Richardson / BiCGStab solves; CG is refused, and so are profiles whose column blocks
would not be M-matrices."""
import math

import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(refinement=4, n_levels=4, n_r=24, grading=1.05, courant_c=20.0)
MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)
STORAGE = {"fac": dict(), "partial": dict(coeff_storage=binding.TPMG_COEFF_PARTIAL),
           "full": dict(coeff_storage=binding.TPMG_COEFF_FULL)}
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def snorm(A_apply, e):
    """sqrt(e^T A e): a norm while the symmetric part of A is positive definite (the
    advection is small against the diffusion)."""
    return math.sqrt(max(float(e @ A_apply(e)), 0.0))


def flow(n_freq, storage, general, **extra):
    """The balanced flow with advection: factorised profiles at set-up, the exact ones
    as the outer operator when `general`; the oracle's V-cycle in the storage's mode."""
    o = oracle.Oracle(**KW)
    outer, fac, eps = inputs.balanced_flow(o.grid(o.refinement)["centre"], o.vertical()["r"], n_freq, advection=True)
    o.set_profiles(**fac)
    s = binding.Solver(profiles=fac, **KW, **STORAGE.get(storage, {}), **extra)
    if general:
        o.set_outer_profiles(**outer)
        s.set_outer_profiles(**outer)
        if storage == "full" or extra.get("precision") == binding.TPMG_PREC_MIXED:
            o.set_vcycle_full(True)
        elif storage == "partial":
            o.set_vcycle_partial(True)
    return s, o


def gpu(s, fn, x):
    y = torch.empty(s.N, dtype=torch.float64, device="cuda")
    fn(torch.from_numpy(x).cuda(), y)
    return y.cpu().numpy()


@pytest.mark.parametrize("general", [False, True], ids=["factorised", "general"])
def test_operator_parity(general):
    """A x with advection against the oracle: 64 ulp of 2 |A| |x| (|A| from the
    factorised operator's M-matrix form, within a factor 2 of the profiled one)."""
    s, o = flow(0.028, "fac", general)
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 80, s.N)
    y = gpu(s, s.apply_operator, x)
    yo = o.apply_outer(x) if general else o.apply(x)
    _, diag, _ = o.column_blocks()
    bound = 2.0 * (2.0 * diag.reshape(-1) * np.abs(x) - o.apply(np.abs(x)))
    assert np.all(np.abs(y - yo) <= 64 * EPS * np.abs(bound))
    outer, fac, _ = inputs.balanced_flow(o.grid(o.refinement)["centre"], o.vertical()["r"], 0.028)
    if general:
        o.set_outer_profiles(**outer)
    else:
        o.set_profiles(**fac)
    plain = o.apply_outer(x) if general else o.apply(x)
    assert np.max(np.abs(yo - plain)) > 1e-9 * np.max(np.abs(yo))   # the advection is there


@pytest.mark.parametrize("scan", [0, 5120], ids=["twisted", "scan"])
@pytest.mark.parametrize("general", [False, True], ids=["factorised", "general"])
@pytest.mark.parametrize("storage", STORAGE.keys())
def test_vcycle_parity(storage, general, scan):
    """The FP64 V-cycle with the non-symmetric column blocks against the oracle's."""
    s, o = flow(0.028, storage, general, scan_max_cells=scan)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 81, s.N)
    z, zo = gpu(s, s.vcycle, r), o.vcycle(r)
    A = o.apply_outer if general else o.apply
    assert snorm(A, z - zo) <= 1e-11 * snorm(A, zo)


def test_mixed_vcycle_parity():
    """Mixed precision: the BF16 stencil with the advection X in BF16 and the FP32 V-cycle
    against the oracle's V-cycle on BF16-rounded coefficients (TPMG^full)."""
    s, o = flow(0.028, "mixed", True, **MIXED)
    o.set_vcycle_bf16(True)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 82, s.N)
    z, zo = gpu(s, s.vcycle, r), o.vcycle(r)
    assert snorm(o.apply_outer, z - zo) <= 5e-3 * snorm(o.apply_outer, zo)


@pytest.mark.parametrize("outer", [binding.TPMG_OUTER_RICHARDSON, binding.TPMG_OUTER_BICGSTAB],
                         ids=["richardson", "bicgstab"])
@pytest.mark.parametrize("storage", STORAGE.keys())
def test_solves_match_the_oracle(storage, outer):
    """Richardson and BiCGStab on the non-symmetric problem: the oracle's iteration count
    (within one) and solution."""
    s, o = flow(0.025, storage, True, outer=outer)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 83, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-10, max_iter=300)
    assert st == binding.TPMG_OK
    if outer == binding.TPMG_OUTER_RICHARDSON:
        uo, hist = o.richardson(f, np.zeros(s.N), it)
        assert hist[-1] <= 1e-10 * hist[0] * 1.01
        if it > 1:
            _, h1 = o.richardson(f, np.zeros(s.N), it - 1)
            assert h1[-1] > 1e-10 * h1[0] * 0.99
    else:
        ref = o.bicgstab(f, rtol=1e-10, max_iter=300)
        assert ref["status"] == 0 and abs(it - ref["iters"]) <= 1, (it, ref["iters"])
        uo = ref["u"]
    e = u.cpu().numpy() - uo
    assert snorm(o.apply_outer, e) <= 1e-8 * snorm(o.apply_outer, uo)
    print(f"\n{storage} outer {outer}: {it} iterations")


@pytest.mark.parametrize("outer", [binding.TPMG_OUTER_RICHARDSON, binding.TPMG_OUTER_BICGSTAB],
                         ids=["richardson", "bicgstab"])
def test_mixed_solves_reach_the_true_residual(outer):
    """The mixed-precision V-cycle (TPMG^full in BF16 / FP32) with the FP64 outer
    iteration: the true residual of the non-symmetric problem to 1e-7, in at most one
    more iteration than TPMG^full in FP64."""
    its = []
    for storage, extra in (("full", {}), ("mixed", MIXED)):
        s, o = flow(0.025, storage, True, outer=outer, **extra)
        f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 86, s.N)).cuda()
        u = torch.zeros_like(f)
        st, it, rel, _ = s.solve(f, u, rtol=1e-8, max_iter=300)
        assert st == binding.TPMG_OK
        r = torch.empty_like(u)
        s.apply_operator(u, r)
        assert float(torch.linalg.norm(f - r) / torch.linalg.norm(f)) <= 1e-7
        its.append(it)
    assert its[1] <= its[0] + 1, its


def test_cg_is_refused_with_advection():
    s, _ = flow(0.025, "fac", False)
    f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 84, s.N)).cuda()
    u = torch.zeros_like(f)
    st, _, _, _ = s.solve(f, u, rtol=1e-5, max_iter=10, raise_on_fail=False)
    assert st == binding.TPMG_ERR_INVALID_ARG


def test_too_strong_advection_is_rejected():
    """Column blocks that are no M-matrices are refused: at set-up (factorised xi), and by
    tpmg_set_outer_profiles (general xi, TPMG^full), which then leaves the V-cycle as it was."""
    o = oracle.Oracle(**KW)
    outer, fac, _ = inputs.balanced_flow(o.grid(o.refinement)["centre"], o.vertical()["r"], 0.028, advection=True)
    strong = dict(fac, xi_r=fac["xi_r"] * 1e6)
    with pytest.raises(binding.TPMGError) as ei:
        binding.Solver(profiles=strong, **KW)
    assert ei.value.status == binding.TPMG_ERR_INVALID_ARG
    s = binding.Solver(profiles=fac, coeff_storage=binding.TPMG_COEFF_FULL, **KW)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 85, s.N)
    z0 = gpu(s, s.vcycle, r)
    with pytest.raises(binding.TPMGError) as ei:
        s.set_outer_profiles(**dict(outer, xi=outer["xi"] * 1e6))
    assert ei.value.status == binding.TPMG_ERR_INVALID_ARG
    assert np.array_equal(gpu(s, s.vcycle, r), z0)


def test_batch_refuses_advection():
    s, _ = flow(0.025, "fac", False)
    f = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    with pytest.raises(binding.TPMGError) as exc:
        binding.Batch([s], [f], [u])
    assert exc.value.status == binding.TPMG_ERR_INVALID_ARG
