"""Factorised profiles (tpmg_setup_profiles; Sec. 2 eq. profiles, the TPMG^otimes form)
on the GPU against the oracle with the same profiles (needs a GPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
KW = dict(refinement=4, n_levels=4, n_r=24, grading=1.05, courant_c=20.0)
MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def random_profiles(o, seed):
    n = o.level_cells(o.n_levels - 1)
    u = lambda k, m: 1.0 + 0.6 * inputs.uniform_pm1(seed + k, m)
    return dict(beta_r=u(1, o.n_r), alphaS_r=u(2, o.n_r), alphar_r=u(3, o.n_r + 1),
                beta_s=u(4, n), alphar_s=u(5, n), alphaS_s=u(6, n))


def flow_profiles(o):
    return inputs.balanced_flow_profiles(o.grid(o.refinement)["centre"], o.vertical()["r"])


def pair(prof_fn, **extra):
    o = oracle.Oracle(**KW)
    prof = prof_fn(o)
    o.set_profiles(**prof)
    s = binding.Solver(profiles=prof, **KW, **extra)
    return s, o


def energy(o, e):
    return math.sqrt(max(float(e @ o.apply(e)), 0.0))


@pytest.mark.parametrize("prof_fn", [lambda o: random_profiles(o, 500), flow_profiles], ids=["random", "balanced_flow"])
def test_apply_and_vcycle_parity(prof_fn):
    s, o = pair(prof_fn)
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 50, s.N)
    y = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.apply_operator(torch.from_numpy(x).cuda(), y)
    yo = o.apply(x)
    _, diag, _ = o.column_blocks()
    bound = 2.0 * diag.reshape(-1) * np.abs(x) - o.apply(np.abs(x))   # |A| |x| of the M-matrix
    assert np.all(np.abs(y.cpu().numpy() - yo) <= 64 * EPS * bound)
    z = torch.empty_like(y)
    s.vcycle(torch.from_numpy(x).cuda(), z)
    zo = o.vcycle(x)
    assert energy(o, z.cpu().numpy() - zo) <= 1e-11 * energy(o, zo)


def test_unit_profiles_change_nothing():
    o = oracle.Oracle(**KW)
    ones = {k: np.ones_like(v) for k, v in random_profiles(o, 501).items()}
    a = binding.Solver(profiles=ones, **KW)
    b = binding.Solver(**KW)
    f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 51, a.N)).cuda()
    ua, ub = torch.zeros_like(f), torch.zeros_like(f)
    ra, rb = a.solve(f, ua, rtol=1e-8), b.solve(f, ub, rtol=1e-8)
    assert ra[:3] == rb[:3] and torch.equal(ua, ub)


@pytest.mark.parametrize("outer", [binding.TPMG_OUTER_CG, binding.TPMG_OUTER_BICGSTAB])
def test_balanced_flow_solve_matches_the_oracle(outer):
    s, o = pair(flow_profiles, outer=outer)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 52, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-10, max_iter=100)
    ref = o.pcg(f, rtol=1e-12, max_iter=200)
    assert st == binding.TPMG_OK and ref["status"] == 0
    assert energy(o, u.cpu().numpy() - ref["u"]) <= 1e-8 * energy(o, ref["u"])
    plain = binding.Solver(**KW, outer=outer)
    u2 = torch.zeros_like(u)
    _, it_plain, _, _ = plain.solve(torch.from_numpy(f).cuda(), u2, rtol=1e-10, max_iter=100)
    print(f"\nouter {outer}: {it} iterations with the balanced-flow profiles, {it_plain} with unit profiles")
    assert it <= it_plain + 2


def test_mixed_precision_with_profiles():
    """The BF16 stencil built from the profiled coefficients: the FP32 V-cycle against
    the oracle's BF16 V-cycle, and flexible CG to the FP64 solution."""
    s, o = pair(flow_profiles, **MIXED)
    o.set_vcycle_bf16(True)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 53, s.N)
    z = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.vcycle(torch.from_numpy(r).cuda(), z)
    zo = o.vcycle(r)
    assert energy(o, z.cpu().numpy() - zo) <= 5e-3 * energy(o, zo)
    o.set_vcycle_bf16(False)
    u = torch.zeros_like(z)
    st, it, rel, _ = s.solve(torch.from_numpy(r).cuda(), u, rtol=1e-10, max_iter=100)
    ref = o.pcg(r, rtol=1e-12, max_iter=200)
    assert st == binding.TPMG_OK
    assert energy(o, u.cpu().numpy() - ref["u"]) <= 1e-8 * energy(o, ref["u"])
