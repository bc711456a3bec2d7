"""Programmatic dependent launch against plain launches, through the C ABI
(needs a GPU).

With params.pdl = 1 each kernel of the V-cycle and of the outer loop may be
scheduled while its predecessor in the stream finishes, but it waits for the
predecessor's results before it reads or writes any vector.  The arithmetic
and its order are unchanged, so every result must equal the plain launches'
bit for bit: solves kernel by kernel and as one graph, block-SOR and
block-Jacobi, the mixed-precision form, the non-symmetric outer iterations,
the batched form, and the operator and V-cycle calls on their own.
"""
import numpy as np
import pytest

from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = dict(precision=binding.TPMG_PREC_MIXED, coeff_storage=binding.TPMG_COEFF_FULL)

CASES = {
    "fp64_graph": dict(refinement=4, n_levels=5, n_r=24, grading=1.05, courant_c=30.0),
    "fp64_host_loop": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1, graphs=0),
    "fp64_twisted_coarse": dict(refinement=4, n_levels=3, n_r=40, grading=1.05, courant_c=80.0, scan_max_cells=0),
    "jacobi": dict(refinement=2, n_levels=3, n_r=33, courant_c=20.0, smoother=1, relax=0.6, nu_pre=1, nu_post=1,
                   nu_coarse=2),
    "full_storage": dict(refinement=3, n_levels=3, n_r=20, grading=1.1, courant_c=50.0, coeff_storage=1),
    "mixed": dict(refinement=4, n_levels=4, n_r=64, grading=1.05, courant_c=150.0, **MIXED),
    "linear_bicgstab": dict(refinement=3, n_levels=3, n_r=16, courant_c=8.0, prolongation=1, outer=2),
    "linear_richardson": dict(refinement=3, n_levels=3, n_r=16, courant_c=8.0, prolongation=1, outer=1),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rhs(n, j):
    return torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 70 + j, n)).cuda()


@pytest.mark.parametrize("name", sorted(CASES))
def test_pdl_solve_is_bit_identical(name):
    kw = CASES[name]
    a = binding.Solver(pdl=1, **kw)
    b = binding.Solver(pdl=0, **kw)
    assert a.params.pdl == 1 and b.params.pdl == 0
    f = rhs(a.N, 0)
    for rep in range(2):   # the second solve replays a captured graph where graphs are on
        ua = torch.zeros_like(f)
        ub = torch.zeros_like(f)
        sa, ita, ra, _ = a.solve(f, ua, rtol=1e-8, max_iter=40, raise_on_fail=False)
        sb, itb, rb, _ = b.solve(f, ub, rtol=1e-8, max_iter=40, raise_on_fail=False)
        torch.cuda.synchronize()
        assert sa == sb and sa in (binding.TPMG_OK, binding.TPMG_ERR_NOT_CONVERGED)
        assert ita == itb > 0 and ra == rb
        assert torch.equal(ua, ub)


def test_pdl_operator_and_vcycle_are_bit_identical():
    kw = CASES["fp64_graph"]
    a = binding.Solver(pdl=1, **kw)
    b = binding.Solver(pdl=0, **kw)
    x = rhs(a.N, 1)
    ya, yb, za, zb = (torch.full_like(x, float("nan")) for _ in range(4))
    a.apply_operator(x, ya)
    b.apply_operator(x, yb)
    a.vcycle(x, za)
    b.vcycle(x, zb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb) and torch.equal(za, zb)


def test_pdl_batch_is_bit_identical():
    probs = [CASES["fp64_graph"], CASES["jacobi"], CASES["mixed"]]
    out = {}
    for pdl in (1, 0):
        solvers = [binding.Solver(pdl=pdl, **kw) for kw in probs]
        fs = [rhs(s.N, 2 + j) for j, s in enumerate(solvers)]
        us = [torch.zeros_like(f) for f in fs]
        bt = binding.Batch(solvers, fs, us, rtol=1e-6, max_iter=100)
        st, it, rel, sts, _ = bt.run()
        torch.cuda.synchronize()
        assert st == binding.TPMG_OK and np.all(sts == binding.TPMG_OK)
        out[pdl] = (it.copy(), rel.copy(), [u.clone() for u in us])
        bt.close()
    assert np.array_equal(out[1][0], out[0][0]) and np.array_equal(out[1][1], out[0][1])
    assert all(torch.equal(x, y) for x, y in zip(out[1][2], out[0][2]))


def test_pdl_rejects_other_values():
    with pytest.raises(binding.TPMGError) as exc:
        binding.Solver(refinement=1, n_levels=2, n_r=4, pdl=2)
    assert exc.value.status == binding.TPMG_ERR_INVALID_ARG
