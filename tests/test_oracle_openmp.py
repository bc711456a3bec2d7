"""The oracle compiled with OpenMP (the multi-core baseline timing) gives the same
bits as the plain build: its parallel loops share out independent columns and rows,
and its dot products stay sequential."""
import numpy as np
import pytest

import oracle
from paper_1408_2981_gb300 import inputs


@pytest.fixture(scope="module")
def omp_lib():
    lib = oracle.build_openmp()
    if lib is None:
        pytest.skip("no OpenMP compiler")
    oracle.threads(4, lib_path=lib)
    return lib


@pytest.mark.parametrize("case", [
    dict(), dict(smoother=1, relax=0.5), dict(prolong=True), dict(advection=True)],
    ids=["mcsor", "jacobi", "linear_prolongation", "advection"])
def test_same_bits_as_the_plain_build(omp_lib, case):
    kw = dict(refinement=4, n_levels=4, n_r=24, grading=1.05, courant_c=20.0)
    kw.update({k: v for k, v in case.items() if k in ("smoother", "relax")})
    a, b = oracle.Oracle(**kw), oracle.Oracle(**kw, lib_path=omp_lib)
    for o in (a, b):
        if case.get("prolong"):
            o.set_prolongation(True)
        if case.get("advection"):
            outer, fac, _ = inputs.balanced_flow(o.grid(o.refinement)["centre"], o.vertical()["r"], 0.025,
                                                 advection=True)
            o.set_profiles(**fac)
            o.set_outer_profiles(**outer)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 110, a.size())
    assert np.array_equal(a.vcycle(f), b.vcycle(f))
    if case.get("prolong") or case.get("advection"):
        ra, rb = a.bicgstab(f, rtol=1e-8, max_iter=60), b.bicgstab(f, rtol=1e-8, max_iter=60)
    else:
        ra, rb = a.pcg(f, rtol=1e-8, max_iter=60), b.pcg(f, rtol=1e-8, max_iter=60)
    assert ra["iters"] == rb["iters"] and np.array_equal(ra["u"], rb["u"])
