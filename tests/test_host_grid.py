"""The library's host grid (grid.cpp, built without a GPU) against the oracle's grid.

The two are independent implementations (sorted half-edge matching vs
hierarchical neighbour derivation; Van Oosterom-Strackee vs L'Huilier areas;
atan2 vs chord arcs); they must agree on the cell order, the neighbour slots
and the colours exactly, and on the geometry to rounding.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1408_2981_gb300", "csrc")


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("grid") / "grid_dump")
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I", cuda_inc,
                    os.path.join(CSRC, "grid.cpp"), os.path.join(ROOT, "tests", "native", "grid_dump.cpp"),
                    "-o", exe], check=True)
    return exe


def library_grid(exe, tmp_path, refinement, n_levels, n_r, H=10.0 / 6371.0, grading=1.0, omega2=0.0,
                 courant_c=8.0, centre=0):
    out = str(tmp_path / "grid.bin")
    subprocess.run([exe, str(refinement), str(n_levels), str(n_r), repr(H), repr(grading), repr(omega2),
                    repr(courant_c), str(centre), out], check=True)
    buf = open(out, "rb").read()
    pos = 0

    def take(dtype, count):
        nonlocal pos
        a = np.frombuffer(buf, dtype=dtype, count=count, offset=pos)
        pos += a.nbytes
        return a.copy()

    omega2_, hmin = take(np.float64, 2)
    res = dict(omega2=omega2_, h_min=hmin, r=take(np.float64, n_r + 1), dr=take(np.float64, n_r),
               vol=take(np.float64, n_r), levels=[])
    for _ in range(n_levels):
        n, nc = take(np.int32, 2)
        lev = dict(n=int(n), n_colours=int(nc), centre=take(np.float64, 3 * n).reshape(n, 3),
                   area=take(np.float64, n), g=take(np.float64, 3 * n).reshape(n, 3),
                   nbr=take(np.int32, 3 * n).reshape(n, 3), colour=take(np.int32, n),
                   corner=take(np.float64, 9 * n).reshape(n, 3, 3))
        res["levels"].append(lev)
    assert pos == len(buf)
    return res


CASES = [dict(refinement=0, n_levels=1, n_r=1), dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0),
         dict(refinement=5, n_levels=3, n_r=64, grading=1.05, courant_c=80.0),
         dict(refinement=4, n_levels=2, n_r=7, grading=1.3, H=0.5, centre=1),
         dict(refinement=6, n_levels=2, n_r=64, grading=1.05, courant_c=80.0)]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()))
def test_host_grid_matches_oracle(dump_exe, tmp_path, kw):
    lib = library_grid(dump_exe, tmp_path, **kw)
    okw = dict(kw)
    if "centre" in okw:
        okw["centre_kind"] = okw.pop("centre")
    o = oracle.Oracle(**okw)
    v = o.vertical()
    np.testing.assert_array_equal(lib["r"], v["r"])
    np.testing.assert_array_equal(lib["dr"], v["dr"])
    np.testing.assert_allclose(lib["vol"], v["vol"], rtol=4e-16, atol=0)
    assert abs(lib["h_min"] - o.h_min) <= 1e-15 * o.h_min
    assert abs(lib["omega2"] - o.omega2) <= 1e-15 * o.omega2
    for level in range(o.n_levels):
        L, g = lib["levels"][level], o.grid(o.level_ref(level))
        assert L["n"] == g["area"].shape[0]
        np.testing.assert_array_equal(L["corner"], g["corners"])   # same arithmetic: bit-identical vertices
        np.testing.assert_array_equal(L["nbr"], g["nbr"])
        np.testing.assert_array_equal(L["colour"], g["colour"])
        np.testing.assert_array_equal(L["centre"], g["centre"])
        np.testing.assert_allclose(L["area"], g["area"], rtol=1e-13 * 2 ** o.level_ref(level), atol=0)
        np.testing.assert_allclose(L["g"], g["g"], rtol=1e-13 * 2 ** o.level_ref(level), atol=0)
