"""The FP64 V-cycle with its stencil stored per unknown: coeff_storage FULL (TPMG^full)
and PARTIAL (alpha_r per face and column, beta and alpha_S factorised: TPMG^partial),
Sec. 4.2 and Sec. 5.3, against the oracle's V-cycle on the same profiles, through the
C ABI (needs a GPU).  scan_max_cells 0 relaxes every level with the twisted
factorisation, 5120 every level of these grids with the warp-scan kernel."""
import math

import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(refinement=4, n_levels=4, n_r=24, grading=1.05, courant_c=20.0)
STORAGE = {"full": binding.TPMG_COEFF_FULL, "partial": binding.TPMG_COEFF_PARTIAL}
SCAN = {"twisted": 0, "scan": 5120}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def oracle_mode(o, storage):
    if storage == "full":
        o.set_vcycle_full(True)
    else:
        o.set_vcycle_partial(True)


def outer_energy(o, e):
    return math.sqrt(max(float(e @ o.apply_outer(e)), 0.0))


def energy(o, e):
    return math.sqrt(max(float(e @ o.apply(e)), 0.0))


def flow_pair(n_freq, storage, **extra):
    o = oracle.Oracle(**KW)
    outer, fac, eps = inputs.balanced_flow(o.grid(o.refinement)["centre"], o.vertical()["r"], n_freq)
    o.set_profiles(**fac)
    o.set_outer_profiles(**outer)
    oracle_mode(o, storage)
    s = binding.Solver(profiles=fac, coeff_storage=STORAGE[storage], **KW, **extra)
    s.set_outer_profiles(**outer)
    return s, o, eps


def vcycle(s, r):
    z = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.vcycle(torch.from_numpy(r).cuda(), z)
    return z.cpu().numpy()


@pytest.mark.parametrize("scan", SCAN.values(), ids=SCAN.keys())
@pytest.mark.parametrize("storage", STORAGE.keys())
def test_stored_factorised_coefficients_give_the_factorised_vcycle(storage, scan):
    """Before general profiles are given the stored stencil holds the factorised
    coefficients: the V-cycle is TPMG^fac up to rounding, on the GPU and in the oracle."""
    o = oracle.Oracle(**KW)
    prof = inputs.balanced_flow_profiles(o.grid(o.refinement)["centre"], o.vertical()["r"])
    o.set_profiles(**prof)
    s = binding.Solver(profiles=prof, coeff_storage=STORAGE[storage], scan_max_cells=scan, **KW)
    fac = binding.Solver(profiles=prof, scan_max_cells=scan, **KW)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 70, s.N)
    z, zf, zo = vcycle(s, r), vcycle(fac, r), o.vcycle(r)
    assert energy(o, z - zf) <= 1e-12 * energy(o, zf)
    assert energy(o, z - zo) <= 1e-11 * energy(o, zo)


@pytest.mark.parametrize("scan", SCAN.values(), ids=SCAN.keys())
@pytest.mark.parametrize("storage", STORAGE.keys())
def test_vcycle_on_general_profiles_matches_the_oracle(storage, scan):
    """The balanced flow at N = 0.028 (eps = 1.24): the stencil rebuilt on every level
    from the general profiles (FULL: all three; PARTIAL: alpha_r) against the oracle's
    V-cycle in the same mode; clearing the profiles restores TPMG^fac."""
    s, o, eps = flow_pair(0.028, storage, scan_max_cells=scan)
    assert eps > 1.0
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 71, s.N)
    z, zo = vcycle(s, r), o.vcycle(r)
    assert outer_energy(o, z - zo) <= 1e-11 * outer_energy(o, zo)
    o.set_vcycle_full(False)
    zfac = o.vcycle(r)
    assert outer_energy(o, zo - zfac) > 1e-4 * outer_energy(o, zo)   # not the factorised V-cycle
    s.set_outer_profiles(None)
    o.set_outer_profiles(None)
    z = vcycle(s, r)
    assert energy(o, z - zfac) <= 1e-11 * energy(o, zfac)


@pytest.mark.parametrize("outer", [binding.TPMG_OUTER_RICHARDSON, binding.TPMG_OUTER_CG, binding.TPMG_OUTER_BICGSTAB],
                         ids=["richardson", "cg", "bicgstab"])
@pytest.mark.parametrize("storage", STORAGE.keys())
def test_solves_match_the_oracle(storage, outer):
    """Solves of the full operator preconditioned by TPMG^full / TPMG^partial in FP64: the
    iteration count of the oracle's solve (within one) and its solution."""
    s, o, _ = flow_pair(0.025, storage, outer=outer)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 72, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-10, max_iter=300)
    assert st == binding.TPMG_OK
    ug = u.cpu().numpy()
    if outer == binding.TPMG_OUTER_RICHARDSON:
        uo, hist = o.richardson(f, np.zeros(s.N), it)
        assert hist[-1] <= 1e-10 * hist[0] * 1.01
        if it > 1:
            _, h1 = o.richardson(f, np.zeros(s.N), it - 1)
            assert h1[-1] > 1e-10 * h1[0] * 0.99   # the oracle needs the same number of steps
    else:
        ref = o.pcg(f, rtol=1e-10, max_iter=300) if outer == binding.TPMG_OUTER_CG else \
            o.bicgstab(f, rtol=1e-10, max_iter=300)
        assert ref["status"] == 0 and abs(it - ref["iters"]) <= 1, (it, ref["iters"])
        uo = ref["u"]
    assert outer_energy(o, ug - uo) <= 1e-8 * outer_energy(o, uo)
    print(f"\n{storage} outer {outer}: {it} iterations")


def test_partial_and_full_iterations_on_the_balanced_flow():
    """Iterations to 1e-5 at eps = 1.24 with Richardson: TPMG^full in FP64 stays near its
    eps = 0 count (robust, Sec. 5); TPMG^partial, whose beta and alpha_S are factorised,
    needs no fewer than TPMG^full."""
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 73, 20 * 4 ** KW["refinement"] * KW["n_r"])
    its = {}
    for storage in ("full", "partial"):
        for n_freq in (9.81 / math.sqrt(1005.0 * 273.0), 0.028):
            s, _, eps = flow_pair(n_freq, storage, outer=binding.TPMG_OUTER_RICHARDSON)
            u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
            st, it, _, _ = s.solve(torch.from_numpy(f).cuda(), u, rtol=1e-5, max_iter=300)
            assert st == binding.TPMG_OK
            its[(storage, round(eps, 2))] = it
    print("\n", its)
    assert its[("full", 1.24)] <= its[("full", 0.0)] + 2
    assert its[("partial", 1.24)] >= its[("full", 1.24)]
