"""Per-class kernel timing (tpmg_profile / tpmg_profile_read) through the C ABI
(needs a GPU).

Launches made one by one each get an event pair; inside a captured graph one
pair spans each run of consecutive launches of the timed class.  Either way
the timing must not change a result, every launch of the class must lie in
some pair (timed counts them), and a replayed graph's pairs hold its latest
replay.
"""
import pytest

from paper_1408_2981_gb300 import binding, build, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(refinement=4, n_levels=5, n_r=24, grading=1.05, courant_c=30.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("pdl", [1, 0])
def test_timed_solve_is_bit_identical_and_counts_every_launch(graphs, pdl):
    s = binding.Solver(graphs=graphs, pdl=pdl, **KW)
    ref = binding.Solver(graphs=graphs, pdl=pdl, **KW)
    f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 90, s.N)).cuda()
    u_ref = torch.zeros_like(f)
    _, it_ref, rel_ref, _ = ref.solve(f, u_ref, rtol=1e-8, max_iter=50)
    s.profile(classes=("relax", "restrict"))
    for rep in range(2):
        u = torch.zeros_like(f)
        _, it, rel, _ = s.solve(f, u, rtol=1e-8, max_iter=50)
        torch.cuda.synchronize()
        assert it == it_ref and rel == rel_ref and torch.equal(u, u_ref)
    pr = s.profile_read()
    for cls in ("relax", "restrict"):
        p = pr[cls]
        assert p["launches"] > 0 and p["ms"] > 0.0
        if graphs:
            # the V-cycle graph's pairs hold its latest replay: one V-cycle's launches
            assert 0 < p["timed"] < p["launches"] and p["launches"] % p["timed"] == 0
        else:
            assert p["timed"] == p["launches"]
    assert pr["apply"]["timed"] == 0 and pr["apply"]["launches"] > 0


def test_device_loop_solve_counts_its_launches():
    """A solve run as one graph with its loop on the device counts its kernels like
    launches made one by one: each iteration applies one V-cycle."""
    s = binding.Solver(graphs=1, **KW)
    f = torch.from_numpy(inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 91, s.N)).cuda()
    z = torch.empty_like(f)
    s.profile(classes=())
    s.vcycle(f, z)
    per_vcycle = s.profile_read()["relax"]
    assert per_vcycle["launches"] > 0
    for rep in range(2):   # the capturing solve, then a replay
        s.profile(classes=())
        u = torch.zeros_like(f)
        st, it, rel, _ = s.solve(f, u, rtol=1e-8, max_iter=50)
        torch.cuda.synchronize()
        pr = s.profile_read()
        assert st == binding.TPMG_OK and it > 0
        assert pr["relax"]["launches"] == it * per_vcycle["launches"]
        assert pr["relax"]["units"] == it * per_vcycle["units"]
        assert pr["apply"]["launches"] == it and pr["residual"]["launches"] >= 1
