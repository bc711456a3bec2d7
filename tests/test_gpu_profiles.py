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


@pytest.mark.parametrize("scan", [5120, 0], ids=["scan", "twisted"])
@pytest.mark.parametrize("prof_fn", [lambda o: random_profiles(o, 500), flow_profiles], ids=["random", "balanced_flow"])
def test_apply_and_vcycle_parity(prof_fn, scan):
    # scan 0: twisted tasks on every level, whose right-hand side comes from the couplings
    # scaled by the pivots of the profiles' column blocks
    s, o = pair(prof_fn, scan_max_cells=scan)
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


# ---- general (non-factorising) profiles: the balanced flow at N > N* ---------------

N_STAR = 9.81 / math.sqrt(1005.0 * 273.0)


def flow_pair(n_freq, **extra):
    o = oracle.Oracle(**KW)
    outer, fac, eps = inputs.balanced_flow(o.grid(o.refinement)["centre"], o.vertical()["r"], n_freq)
    o.set_profiles(**fac)
    o.set_outer_profiles(**outer)
    s = binding.Solver(profiles=fac, **KW, **extra)
    s.set_outer_profiles(**outer)
    return s, o, eps


def test_full_operator_parity():
    """The problem's operator from per-unknown coefficients (TPMG^full storage) against
    the oracle's.  Bound: 64 ulp of |A||x|, with |A| from the factorised operator (the
    general profiles differ from it by less than a factor 2 here) times 2."""
    s, o, eps = flow_pair(0.028)
    assert eps > 1.0
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 60, s.N)
    y = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.apply_operator(torch.from_numpy(x).cuda(), y)
    yo = o.apply_outer(x)
    _, diag, _ = o.column_blocks()
    bound = 2.0 * (2.0 * diag.reshape(-1) * np.abs(x) - o.apply(np.abs(x)))
    assert np.all(np.abs(y.cpu().numpy() - yo) <= 64 * EPS * bound)
    assert np.max(np.abs(yo - o.apply(x))) > 1e-3 * np.max(np.abs(yo))   # not the factorised operator


@pytest.mark.parametrize("outer", [binding.TPMG_OUTER_CG, binding.TPMG_OUTER_BICGSTAB])
def test_tpmg_fac_preconditions_the_full_operator(outer):
    """FP64: the V-cycle of the factorised approximation preconditions the full operator
    (Sec. 3.2.2); the solve matches the oracle's."""
    s, o, _ = flow_pair(0.025, outer=outer)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 61, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-10, max_iter=200)
    ref = o.pcg(f, rtol=1e-10, max_iter=200) if outer == binding.TPMG_OUTER_CG else o.bicgstab(f, rtol=1e-10, max_iter=200)
    assert st == binding.TPMG_OK and ref["status"] == 0 and abs(it - ref["iters"]) <= 1, (it, ref["iters"])
    e = u.cpu().numpy() - ref["u"]
    assert math.sqrt(e @ o.apply_outer(e)) <= 1e-8 * math.sqrt(ref["u"] @ o.apply_outer(ref["u"]))


def test_mixed_vcycle_on_general_profiles_matches_the_oracle():
    """Mixed precision: the BF16 stencil rebuilt from the general profiles on every level
    (TPMG^full) against the oracle's V-cycle on the same profiles (BF16-rounded
    coefficients, FP64 arithmetic)."""
    s, o, _ = flow_pair(0.028, **MIXED)
    o.set_vcycle_full(True)
    o.set_vcycle_bf16(True)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 62, s.N)
    z = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.vcycle(torch.from_numpy(r).cuda(), z)
    zo = o.vcycle(r)
    e = z.cpu().numpy() - zo
    assert math.sqrt(e @ o.apply_outer(e)) <= 5e-3 * math.sqrt(zo @ o.apply_outer(zo))
    s.set_outer_profiles(None)   # back to the factorised stencil and operator
    o.set_outer_profiles(None)
    o.set_vcycle_full(False)
    s.vcycle(torch.from_numpy(r).cuda(), z)
    zf = o.vcycle(r)
    assert math.sqrt((z.cpu().numpy() - zf) @ o.apply(z.cpu().numpy() - zf)) <= 5e-3 * math.sqrt(zf @ o.apply(zf))


def test_factorisation_sweep_reports_iterations():
    """Iterations to ||r|| <= 1e-5 ||r_0|| against the buoyancy frequency (eps = 0 ... 1.24),
    the experiment of Sec. 5 (Fig. 3, right): the FP64 V-cycle on the factorised
    approximation (TPMG^fac) and the mixed V-cycle on the full profiles (TPMG^full), each
    preconditioning the full operator with Richardson, CG and BiCGStab."""
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 63, 20 * 4 ** KW["refinement"] * KW["n_r"])
    rows = []
    for n_freq in (N_STAR, 0.022, 0.025, 0.028):
        row = []
        for extra in ({}, MIXED):
            for outer in (binding.TPMG_OUTER_RICHARDSON, binding.TPMG_OUTER_CG, binding.TPMG_OUTER_BICGSTAB):
                s, _, eps = flow_pair(n_freq, outer=outer, **extra)
                fg = torch.from_numpy(f).cuda()
                u = torch.zeros_like(fg)
                st, it, rel, _ = s.solve(fg, u, rtol=1e-5, max_iter=300)
                assert st == binding.TPMG_OK
                row.append(it)
        rows.append((eps, row))
    print("\neps    | TPMG^fac (FP64): Richardson CG BiCGStab | TPMG^full (mixed): Richardson CG BiCGStab")
    for eps, row in rows:
        print(f"{eps:5.2f}  | {row[0]:4d} {row[1]:4d} {row[2]:4d} | {row[3]:4d} {row[4]:4d} {row[5]:4d}")
    fac0, fac1 = rows[0][1][:3], rows[-1][1][:3]
    full0, full1 = rows[0][1][3:], rows[-1][1][3:]
    assert all(b >= a for a, b in zip(fac0, fac1))        # the factorised preconditioner degrades
    assert all(b <= a + 2 for a, b in zip(full0, full1))  # the full one is robust
