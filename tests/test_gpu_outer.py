"""The outer iterations Richardson and BiCGStab (params.outer, Sec. 5) on the GPU
against the oracle's, through the C ABI (needs a GPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1),
         dict(refinement=4, n_levels=5, n_r=32, grading=1.05, courant_c=80.0)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def energy(o, e):
    return math.sqrt(max(float(e @ o.apply(e)), 0.0))


@pytest.mark.parametrize("kw", CASES)
def test_richardson_matches_the_oracle(kw):
    """Six steps u <- u + B(f - A u) from zero: the same iterates and residual history."""
    s = binding.Solver(outer=binding.TPMG_OUTER_RICHARDSON, **kw)
    o = oracle.Oracle(**kw)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 40, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, hist = s.solve(torch.from_numpy(f).cuda(), u, rtol=0.0, max_iter=6, history=True,
                                raise_on_fail=False)
    assert st == binding.TPMG_ERR_NOT_CONVERGED and it == 6
    u_or, h_or = o.richardson(f, np.zeros(s.N), 6)
    ug = u.cpu().numpy()
    assert energy(o, ug - u_or) <= 1e-10 * energy(o, u_or)
    np.testing.assert_allclose(hist, h_or / h_or[0], rtol=1e-8)
    print(f"Richardson factor per step: {(h_or[-1] / h_or[-4]) ** (1 / 3):.3f}")


@pytest.mark.parametrize("kw", CASES)
def test_bicgstab_matches_the_oracle(kw):
    s = binding.Solver(outer=binding.TPMG_OUTER_BICGSTAB, **kw)
    o = oracle.Oracle(**kw)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 41, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, hist = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-10, max_iter=60, history=True)
    ref = o.bicgstab(f, rtol=1e-10, max_iter=60)
    assert st == binding.TPMG_OK and ref["status"] == 0
    assert abs(it - ref["iters"]) <= 1, (it, ref["iters"])
    k = min(it, ref["iters"], 4)
    np.testing.assert_allclose(hist[:k + 1], ref["hist"][:k + 1], rtol=1e-6)
    ug = u.cpu().numpy()
    assert energy(o, ug - ref["u"]) <= 1e-8 * energy(o, ref["u"])
    pcg = o.pcg(f, rtol=1e-10, max_iter=100)
    print(f"BiCGStab {it} iterations (2 V-cycles each), CG {pcg['iters']}")


def test_outer_iterations_in_mixed_precision():
    """Richardson and BiCGStab with the FP32/BF16 V-cycle reach the tolerance on the
    true residual, in at most one more iteration than with the FP64 V-cycle."""
    kw = CASES[1]
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 42, 20 * 4 ** kw["refinement"] * kw["n_r"])
    for outer in (binding.TPMG_OUTER_RICHARDSON, binding.TPMG_OUTER_BICGSTAB):
        its = []
        for prec in ((binding.TPMG_PREC_FP64, binding.TPMG_COEFF_FACTORISED),
                     (binding.TPMG_PREC_MIXED, binding.TPMG_COEFF_FULL)):
            s = binding.Solver(outer=outer, precision=prec[0], coeff_storage=prec[1], **kw)
            fg = torch.from_numpy(f).cuda()
            u = torch.zeros_like(fg)
            st, it, rel, _ = s.solve(fg, u, rtol=1e-8, max_iter=100)
            r = torch.empty_like(u)
            s.apply_operator(u, r)
            assert float(torch.linalg.norm(fg - r) / torch.linalg.norm(fg)) <= 1e-7
            its.append(it)
        assert its[1] <= its[0] + 1, (outer, its)


def test_batch_rejects_non_cg_outer():
    s = binding.Solver(outer=binding.TPMG_OUTER_BICGSTAB, **CASES[0])
    f = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    with pytest.raises(binding.TPMGError) as exc:
        binding.Batch([s], [f], [u])
    assert exc.value.status == binding.TPMG_ERR_INVALID_ARG
