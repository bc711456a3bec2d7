"""Linear prolongation (params.prolongation = TPMG_PROLONG_LINEAR; Sec. 5) on the GPU
against the oracle's, through the C ABI (needs a GPU): the V-cycle in FP64 (block-SOR
and block-Jacobi, twisted and warp-scan relaxation, with and without post-smoothing)
and in mixed precision, and Richardson / BiCGStab solves; CG is refused."""
import math

import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(refinement=4, n_levels=4, n_r=24, grading=1.05, courant_c=20.0)
LIN = dict(prolongation=binding.TPMG_PROLONG_LINEAR)
MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def energy(o, e):
    return math.sqrt(max(float(e @ o.apply(e)), 0.0))


def pair(**kw):
    okw = {k: v for k, v in kw.items() if k not in ("scan_max_cells", "outer", "precision", "coeff_storage")}
    o = oracle.Oracle(**okw)
    o.set_prolongation(True)
    s = binding.Solver(**kw, **LIN)
    return s, o


def vcycle(s, r):
    z = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.vcycle(torch.from_numpy(r).cuda(), z)
    return z.cpu().numpy()


@pytest.mark.parametrize("case", [
    dict(scan_max_cells=0), dict(scan_max_cells=5120), dict(smoother=1, relax=0.5, scan_max_cells=0),
    dict(nu_post=0), dict(nu_coarse=0)], ids=["twisted", "scan", "jacobi", "no_post", "no_coarse"])
def test_vcycle_parity(case):
    s, o = pair(**KW, **case)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 100, s.N)
    z, zo = vcycle(s, r), o.vcycle(r)
    assert energy(o, z - zo) <= 1e-11 * energy(o, zo)
    o.set_prolongation(False)
    assert energy(o, zo - o.vcycle(r)) > 1e-4 * energy(o, zo)   # not the piecewise-constant P


def test_mixed_vcycle_parity():
    s, o = pair(**KW, **MIXED)
    o.set_vcycle_bf16(True)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 101, s.N)
    z, zo = vcycle(s, r), o.vcycle(r)
    assert energy(o, z - zo) <= 5e-3 * energy(o, zo)


@pytest.mark.parametrize("outer", [binding.TPMG_OUTER_RICHARDSON, binding.TPMG_OUTER_BICGSTAB],
                         ids=["richardson", "bicgstab"])
def test_solves_match_the_oracle(outer):
    s, o = pair(**KW, outer=outer)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 102, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-10, max_iter=200)
    assert st == binding.TPMG_OK
    if outer == binding.TPMG_OUTER_RICHARDSON:
        uo, hist = o.richardson(f, np.zeros(s.N), it)
        assert hist[-1] <= 1e-10 * hist[0] * 1.01
        _, h1 = o.richardson(f, np.zeros(s.N), it - 1)
        assert h1[-1] > 1e-10 * h1[0] * 0.99
    else:
        ref = o.bicgstab(f, rtol=1e-10, max_iter=200)
        assert ref["status"] == 0 and abs(it - ref["iters"]) <= 1, (it, ref["iters"])
        uo = ref["u"]
    assert energy(o, u.cpu().numpy() - uo) <= 1e-8 * energy(o, uo)


def test_iterations_against_piecewise_constant():
    """Richardson to 1e-8 on the same problem: linear prolongation needs no more
    iterations than P = R^T (it is the more accurate transfer)."""
    f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 103, 20 * 4 ** 5 * 32)).cuda()
    its = {}
    for name, extra in (("constant", {}), ("linear", LIN)):
        s = binding.Solver(refinement=5, n_levels=5, n_r=32, grading=1.05, courant_c=20.0,
                           outer=binding.TPMG_OUTER_RICHARDSON, **extra)
        u = torch.zeros_like(f)
        st, it, _, _ = s.solve(f, u, rtol=1e-8, max_iter=200)
        assert st == binding.TPMG_OK
        its[name] = it
    print("\n", its)
    assert its["linear"] <= its["constant"]


def test_cg_is_refused():
    s = binding.Solver(**KW, **LIN)
    f = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    st, _, _, _ = s.solve(f, u, rtol=1e-5, max_iter=10, raise_on_fail=False)
    assert st == binding.TPMG_ERR_INVALID_ARG
