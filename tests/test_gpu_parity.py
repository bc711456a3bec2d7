"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Tolerances (derivations in the design notes):
* grid: cell order, neighbours and colours bit-exact; centres to a few ulp;
  areas / flux factors to 1e-12 relative (different but equivalent formulas).
* operator: 64 eps times |A| |x| per element (9 rounded operations per row).
* V-cycle: 1e-11 relative in the energy norm ||.||_A (and 1e-7 in the
  2-norm).  The column blocks have condition numbers 1e6-1e9 (vertical
  coupling over the mass term), so two equivalent orderings of the line solve
  differ by ~eps * cond in the 2-norm, but that difference lies in the nearly
  null vertically constant mode, whose energy is ~1/cond of a typical mode.
* PCG: 1e-10 relative solution error (the accuracy target of the path).
"""
import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps

CASES = {
    "ref3_nr16_uniform_c8_nu1": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1),
    "ref2_nr7_graded_c80_nu2": dict(refinement=2, n_levels=3, n_r=7, grading=1.1, courant_c=80.0),
    "ref0_nr1_single_level": dict(refinement=0, n_levels=1, n_r=1, courant_c=8.0),
    "ref1_nr33_jacobi": dict(refinement=1, n_levels=2, n_r=33, courant_c=20.0, smoother=1, relax=0.6, nu_pre=1,
                             nu_post=1, nu_coarse=2),
    "ref3_nr5_relax08_vertexmean": dict(refinement=3, n_levels=2, n_r=5, courant_c=8.0, relax=0.8, centre=1),
    "ref2_nr200_tall": dict(refinement=2, n_levels=3, n_r=200, grading=1.02, courant_c=8.0, nu_pre=1, nu_post=1),
    "ref4_nr24_graded_deep": dict(refinement=4, n_levels=5, n_r=24, grading=1.05, courant_c=30.0),
    # 5120- and 1280-cell levels relaxed in twisted tasks except their small third colours
    # (140 and 66 cells), which take the warp scans; the 320- and 80-cell levels all scans
    "ref4_nr24_small_colours_scanned": dict(refinement=4, n_levels=4, n_r=24, grading=1.05, courant_c=30.0,
                                            scan_max_cells=640),
    # every level in twisted tasks: the right-hand side from the scaled couplings (f / pivot
    # written by each colour's first pass in a visit), and the factorised form beside it
    "ref3_nr16_twisted_scaled": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1,
                                     nu_coarse=1, scan_max_cells=0),
    "ref3_nr16_twisted_factorised": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1,
                                         nu_coarse=1, scan_max_cells=0, scaled_rhs=0),
    # no pre-smoothing: each colour's first pass of a visit is a post-smoothing pass
    "ref2_nr7_twisted_no_presmoothing": dict(refinement=2, n_levels=3, n_r=7, grading=1.1, courant_c=80.0, nu_pre=0,
                                             nu_post=2, scan_max_cells=0),
    "ref1_nr33_twisted_jacobi": dict(refinement=1, n_levels=2, n_r=33, courant_c=20.0, smoother=1, relax=0.6,
                                     nu_pre=1, nu_post=1, nu_coarse=2, scan_max_cells=0),
}


def oracle_for(kw):
    # kernel choices, not part of the method
    kw = {k: v for k, v in kw.items() if k not in ("scan_max_cells", "scaled_rhs")}
    if "centre" in kw:
        kw["centre_kind"] = kw.pop("centre")
    return oracle.Oracle(**kw)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def pair(name):
    kw = CASES[name]
    return binding.Solver(**kw), oracle_for(kw)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", sorted(CASES))
def test_mesh_parity(name):
    s, o = pair(name)
    for level in range(s.n_levels):
        m = s.export_mesh(level)
        g = o.grid(o.level_ref(level))
        np.testing.assert_array_equal(m["nbrs"], g["nbr"])
        np.testing.assert_array_equal(m["colour"], g["colour"])
        np.testing.assert_allclose(m["centres"], g["centre"], rtol=0, atol=8 * EPS)
        np.testing.assert_allclose(m["areas"], g["area"], rtol=1e-12)
        np.testing.assert_allclose(m["g"], g["g"], rtol=1e-11)
        assert s.query(level)[3] == o.grid_sizes(o.level_ref(level))["n_colours"]
    np.testing.assert_array_equal(s.export_mesh()["r_faces"], o.vertical()["r"])
    assert abs(s.omega2 - o.omega2) <= 1e-13 * o.omega2


def abs_bound(o, x):
    """|A| |x| per element for the M-matrix A: 2 diag |x| - A |x|."""
    _, diag, _ = o.column_blocks()
    ax = np.abs(x)
    return 2.0 * diag.reshape(-1) * ax - o.apply(ax)


@pytest.mark.parametrize("name", sorted(CASES))
def test_apply_parity(name):
    s, o = pair(name)
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 7, s.N)
    y = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.apply_operator(cuda(x), y)
    yg, yo = host(y), o.apply(x)
    assert np.all(np.abs(yg - yo) <= 64 * EPS * abs_bound(o, x))


@pytest.mark.parametrize("name", sorted(CASES))
def test_vcycle_parity(name):
    s, o = pair(name)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 8, s.N)
    z = torch.full((s.N,), float("nan"), dtype=torch.float64, device="cuda")
    s.vcycle(cuda(r), z)
    zg, zo = host(z), o.vcycle(r)
    assert np.all(np.isfinite(zg))
    e = zg - zo
    rel_a = np.sqrt(e @ o.apply(e)) / np.sqrt(zo @ o.apply(zo))
    assert rel_a <= 1e-11, rel_a
    assert np.linalg.norm(e) <= 1e-7 * np.linalg.norm(zo), np.linalg.norm(e) / np.linalg.norm(zo)


def solve_pair(s, o, f, rtol, max_iter=200):
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, hist = s.solve(cuda(f), u, rtol=rtol, max_iter=max_iter, history=True, raise_on_fail=False)
    ro = o.pcg(f, rtol=rtol, max_iter=max_iter)
    return st, it, rel, hist, host(u), ro


def check_solve(s, o, f, rtol, max_iter=200, tol=1e-10):
    st, it, rel, hist, ug, ro = solve_pair(s, o, f, rtol, max_iter)
    assert ro["status"] == 0 and st == binding.TPMG_OK
    if it != ro["iters"]:
        # stop-boundary tie: both rerun for exactly the oracle's iteration count
        assert abs(it - ro["iters"]) == 1
        st, it, rel, hist, ug, ro = solve_pair(s, o, f, 0.0, ro["iters"])
    err = np.linalg.norm(ug - ro["u"]) / np.linalg.norm(ro["u"])
    assert err <= tol, err
    np.testing.assert_allclose(hist, ro["hist"], rtol=1e-6)
    return it, err


SYMMETRIC = [n for n in sorted(CASES) if CASES[n].get("nu_pre", 2) == CASES[n].get("nu_post", 2)]


@pytest.mark.parametrize("name", SYMMETRIC)
def test_solve_parity(name):
    s, o = pair(name)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, s.N)
    check_solve(s, o, f, 1e-5)


@pytest.mark.parametrize("name", ["ref3_nr16_uniform_c8_nu1", "ref2_nr7_graded_c80_nu2"])
def test_solve_parity_tight(name):
    s, o = pair(name)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 1, s.N)
    check_solve(s, o, f, 1e-11)


def test_small_workload_1280x16():
    """Icosahedron refined 3 times x 16 uniform levels, omega^2/h^2 = 8, nu 1/1, RHS uniform[-1,1]."""
    kw = dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1)
    s, o = binding.Solver(**kw), oracle.Oracle(**kw)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, s.N)
    it, err = check_solve(s, o, f, 1e-5)
    assert it <= 10


@pytest.mark.slow
def test_full_workload_81920x64_manufactured():
    """Refinement 6 x 64 levels graded 1.05, omega^2/h^2 = 80, manufactured solution, rtol 1e-5."""
    kw = dict(refinement=6, n_levels=6, n_r=64, grading=1.05, courant_c=80.0)
    s, o = binding.Solver(**kw), oracle.Oracle(**kw)
    m = s.export_mesh()
    ustar = inputs.manufactured_solution(m["centres"], m["r_faces"], inputs.SEED_MANUFACTURED)
    # the right-hand side is built by the oracle so both solvers see identical bytes
    f = o.apply(ustar)
    fg = torch.empty(s.N, dtype=torch.float64, device="cuda")
    s.apply_operator(cuda(ustar), fg)
    assert np.all(np.abs(host(fg) - f) <= 64 * EPS * abs_bound(o, ustar))
    it, err = check_solve(s, o, f, 1e-5)
    assert it <= 10


def test_zero_rhs_returns_immediately():
    s, _ = pair("ref2_nr7_graded_c80_nu2")
    f = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    st, it, rel, _ = s.solve(f, u)
    assert st == binding.TPMG_OK and it == 0 and rel == 0.0
    assert torch.count_nonzero(u).item() == 0


def test_nan_rhs_is_breakdown():
    s, _ = pair("ref2_nr7_graded_c80_nu2")
    f = torch.ones(s.N, dtype=torch.float64, device="cuda")
    f[5] = float("nan")
    u = torch.zeros_like(f)
    st, it, rel, _ = s.solve(f, u, raise_on_fail=False)
    assert st == binding.TPMG_ERR_BREAKDOWN


def test_max_iter_is_not_converged():
    s, o = pair("ref3_nr16_uniform_c8_nu1")
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, s.N)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, it, rel, _ = s.solve(cuda(f), u, rtol=1e-12, max_iter=2, raise_on_fail=False)
    assert st == binding.TPMG_ERR_NOT_CONVERGED and it == 2 and rel > 1e-12


def test_initial_guess_resume():
    """A solve resumed from its own iterate continues from the reached residual."""
    s, o = pair("ref3_nr16_uniform_c8_nu1")
    f = cuda(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, s.N))
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.solve(f, u, rtol=1e-3)
    u1 = u.clone()
    st, it, rel, _ = s.solve(f, u, rtol=1e-4)
    assert st == binding.TPMG_OK and it >= 1
    r = torch.empty_like(f)
    s.apply_operator(u, r)
    rfin = torch.linalg.norm(f - r).item()
    s.apply_operator(u1, r)
    assert rfin <= 1e-4 * torch.linalg.norm(f - r).item() * 1.0001


def test_solve_is_deterministic():
    s, _ = pair("ref4_nr24_graded_deep")
    f = cuda(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, s.N))
    outs = []
    for _ in range(2):
        u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        s.solve(f, u, rtol=1e-8)
        outs.append(host(u))
    np.testing.assert_array_equal(outs[0], outs[1])


def test_solve_host_matches_device_solve():
    s, _ = pair("ref2_nr7_graded_c80_nu2")
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 3, s.N)
    u_host = np.zeros(s.N)
    st, it, rel = s.solve_host(f, u_host, rtol=1e-6)
    u = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st2, it2, rel2, _ = s.solve(cuda(f), u, rtol=1e-6)
    assert (st, it) == (st2, it2)
    np.testing.assert_array_equal(u_host, host(u))


def test_overlapping_buffers_rejected():
    s, _ = pair("ref0_nr1_single_level")
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TPMGError):
        s.apply_operator(x, x)
    with pytest.raises(binding.TPMGError):
        s.vcycle(x, x)


def test_graph_replay_matches_direct_launches():
    """The captured V-cycle graph replays exactly the kernels launched one by one."""
    kw = CASES["ref4_nr24_graded_deep"]
    f = cuda(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 5, binding.Solver(**kw).N))
    outs, its = [], []
    for graphs in (0, 1):
        s = binding.Solver(graphs=graphs, **kw)
        for _ in range(2):   # with graphs: the first solve captures, the second replays
            u = torch.zeros_like(f)
            st, it, rel, _ = s.solve(f, u, rtol=1e-9)
            outs.append(host(u))
            its.append(it)
    assert len(set(its)) == 1
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


# The FP64 relaxation kernels of the twisted 16-column tasks (tpmg_query_tuning's
# variants 0-4, forced with relax_variant) perform the same arithmetic per column, so
# whole solves agree bit for bit.  The cases put each kernel through its paths: a
# finest level of 2548 tasks per colour; twisted tasks on every level
# (scan_max_cells = 0), so the fused prolongation and the small coarse passes run
# through each variant; block Jacobi with a relaxation weight; the stencil stored per
# unknown (TPMG^full); a column of 160 levels.
VARIANT_CASES = {
    "ref6_nr16_many_tasks": dict(refinement=6, n_levels=2, n_r=16, grading=1.05, courant_c=80.0),
    "ref4_nr24_twisted_everywhere_jacobi": dict(refinement=4, n_levels=5, n_r=24, grading=1.05, courant_c=30.0,
                                                smoother=1, relax=0.7, scan_max_cells=0),
    "ref5_nr40_full_storage": dict(refinement=5, n_levels=3, n_r=40, courant_c=20.0, coeff_storage=1,
                                   scan_max_cells=0),
    "ref3_nr160_tall": dict(refinement=3, n_levels=3, n_r=160, grading=1.02, courant_c=8.0, scan_max_cells=0),
}


@pytest.mark.parametrize("name", sorted(VARIANT_CASES))
def test_relaxation_variants_give_identical_results(name):
    kw = VARIANT_CASES[name]
    outs = []
    for variant in range(5):
        s = binding.Solver(relax_variant=variant, **kw)
        assert all(v == variant for v, _ in s.tuning())
        f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 60, s.N)).cuda()
        u = torch.zeros_like(f)
        st, it, rel, _ = s.solve(f, u, rtol=1e-8, max_iter=200)
        z = torch.empty_like(f)
        s.vcycle(f, z)
        torch.cuda.synchronize()
        outs.append((st, it, rel, u.cpu().numpy(), z.cpu().numpy()))
        s.close()
    for v in range(1, 5):
        assert outs[v][:3] == outs[0][:3], (v, outs[v][:3], outs[0][:3])
        np.testing.assert_array_equal(outs[v][3], outs[0][3])
        np.testing.assert_array_equal(outs[v][4], outs[0][4])


def test_deep_warp_relaxation_vs_oracle():
    """The V-cycle with the wide-gather one-warp twisted passes (variant 4) on every
    level against the oracle's V-cycle (the V-cycle bound of this file)."""
    kw = VARIANT_CASES["ref4_nr24_twisted_everywhere_jacobi"]
    s, o = binding.Solver(relax_variant=4, **kw), oracle_for(kw)
    r = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 61, s.N)
    z = torch.full((s.N,), float("nan"), dtype=torch.float64, device="cuda")
    s.vcycle(cuda(r), z)
    zg, zo = host(z), o.vcycle(r)
    e = zg - zo
    rel_a = np.sqrt(e @ o.apply(e)) / np.sqrt(zo @ o.apply(zo))
    assert rel_a <= 1e-11, rel_a
