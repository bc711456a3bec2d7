"""tpmg_vcycle_noalloc against tpmg_vcycle, through the C ABI (needs a GPU).

tpmg_vcycle_noalloc serves callers that may not let the library allocate
device memory once their own run has started: a host model that owns the
device through its own memory pool, or code that cannot afford the device
synchronisation a cudaMalloc / cudaFree may cause.  It takes the coarse-level
work vectors from a fixed device array built into the library instead.  Its
result must be the V-cycle of tpmg_vcycle bit for bit: both launch the same
kernels in the same order on the same data, and only the addresses of the
work vectors differ, so any difference would be a wrong offset into the
array or a value left over from an earlier call.  Two calls in a row, with
different right-hand sides and a second context sharing the array, show that
values left in the array by a previous call do not leak into the next result.

This file is collected last on purpose, so a run that stops at its first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "mcsor_ref3_nr16": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1),
    "mcsor_ref4_nr24_graded": dict(refinement=4, n_levels=5, n_r=24, grading=1.05, courant_c=30.0),
    "jacobi_ref1_nr33": dict(refinement=1, n_levels=2, n_r=33, courant_c=20.0, smoother=1, relax=0.6, nu_pre=1,
                             nu_post=1, nu_coarse=2),
    # twisted tasks on every level: the f / pivot work vectors come from the array too
    "mcsor_ref3_nr16_twisted": dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1,
                                    nu_coarse=1, scan_max_cells=0),
    "jacobi_ref2_nr16_twisted": dict(refinement=2, n_levels=3, n_r=16, courant_c=8.0, smoother=1, relax=0.7,
                                     scan_max_cells=0),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def energy_rel(s, e, z):
    ae = torch.empty_like(e)
    az = torch.empty_like(z)
    s.apply_operator(e, ae)
    s.apply_operator(z, az)
    return (torch.dot(e, ae).abs().sqrt() / torch.dot(z, az).sqrt()).item()


def check_equal(s, z_new, z_ref):
    assert torch.isfinite(z_new).all()
    if not torch.equal(z_new, z_ref):
        e = z_new - z_ref
        pytest.fail(f"fixed-scratch V-cycle differs from tpmg_vcycle: energy-norm rel. {energy_rel(s, e, z_ref):.3e}, "
                    f"2-norm rel. {(torch.linalg.norm(e) / torch.linalg.norm(z_ref)).item():.3e}")


@pytest.mark.parametrize("name", sorted(CASES))
def test_vcycle_noalloc_matches_vcycle_twice(name):
    s = binding.Solver(**CASES[name])
    other = binding.Solver(**CASES["mcsor_ref3_nr16"])
    rs = [torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 40 + j, s.N)).cuda() for j in range(2)]
    r_other = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 50, other.N)).cuda()
    for r in rs:
        r_copy = r.clone()
        z_ref = torch.full_like(r, float("nan"))
        s.vcycle(r, z_ref)
        z_new = torch.full_like(r, float("nan"))
        s.vcycle_noalloc(r, z_new)
        # a call of another context in between leaves its own values in the shared array
        z_other = torch.empty_like(r_other)
        other.vcycle_noalloc(r_other, z_other)
        torch.cuda.synchronize()
        check_equal(s, z_new, z_ref)
        assert torch.equal(r, r_copy)   # the input is not modified
    z_o_ref = torch.empty_like(r_other)
    other.vcycle(r_other, z_o_ref)
    torch.cuda.synchronize()
    check_equal(other, z_other, z_o_ref)


def test_vcycle_noalloc_rejects_problems_beyond_the_array():
    # 2 coarse vectors of 5120 cells x 256 levels = 2.6M doubles > 2^21
    s = binding.Solver(refinement=5, n_levels=2, n_r=256, courant_c=8.0)
    r = torch.ones(s.N, dtype=torch.float64, device="cuda")
    z = torch.full_like(r, float("nan"))
    with pytest.raises(binding.TPMGError) as exc:
        s.vcycle_noalloc(r, z)
    assert exc.value.status == binding.TPMG_ERR_INVALID_ARG
    assert "scratch" in str(exc.value)
    torch.cuda.synchronize()
    assert torch.isnan(z).all()   # nothing was launched


def test_vcycle_noalloc_rejects_overlap():
    s = binding.Solver(**CASES["mcsor_ref3_nr16"])
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TPMGError):
        s.vcycle_noalloc(x, x)
