"""The C-ABI library builds, loads and exports every entry point of include/tpmg.h (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1408_2981_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "tpmg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tpmg_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(binding.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_struct_layout_matches_header():
    # the ctypes mirror must have one field per member of tpmg_params, in order
    txt = open(os.path.join(ROOT, "include", "tpmg.h")).read()
    body = txt[txt.index("typedef struct {", txt.index("TPMG_PREC_MIXED")):txt.index("} tpmg_params;")]
    names = re.findall(r"(?:int|double)\s+(\w+)\s*;", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert names == [f[0] for f in binding.tpmg_params._fields_]


def test_default_params_on_host(lib):
    p = binding.default_params()
    assert (p.refinement, p.n_levels, p.n_r) == (3, 4, 16)
    assert abs(p.H - 10.0 / 6371.0) < 1e-18 and p.courant_c == 8.0
    assert lib.tpmg_default_params(None) == binding.TPMG_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [dict(refinement=-1), dict(refinement=10), dict(n_levels=0), dict(n_levels=5),
                                 dict(n_r=0), dict(n_r=2000), dict(H=0.0), dict(grading=-1.0),
                                 dict(omega2=0.0, courant_c=0.0), dict(nu_pre=-1), dict(smoother=7),
                                 dict(relax=0.0), dict(relax=2.0), dict(centre=3), dict(coeff_storage=9),
                                 dict(precision=9), dict(precision=1, coeff_storage=0), dict(precision=1, coeff_storage=2), dict(prolongation=2),
                                 dict(refinement=9, n_levels=3, n_r=1024), dict(scan_max_cells=-1), dict(outer=3),
                                 dict(relax_variant=-2), dict(relax_variant=5), dict(relax_variant=4, precision=1, coeff_storage=1),
                                 dict(scaled_rhs=2), dict(scaled_rhs=-1), dict(net_tcgen05=2)])
def test_setup_rejects_bad_params_before_touching_cuda(lib, bad):
    p = binding.default_params(**bad)
    h = ctypes.c_void_p()
    assert lib.tpmg_setup(ctypes.byref(p), None, ctypes.byref(h)) == binding.TPMG_ERR_INVALID_ARG
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.tpmg_setup(None, None, None) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_apply_operator(None, None, None) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_vcycle(None, None, None) == binding.TPMG_ERR_INVALID_ARG
    it, rel = ctypes.c_int(), ctypes.c_double()
    assert lib.tpmg_solve(None, None, None, 1e-5, 10, ctypes.byref(it), ctypes.byref(rel), None) == \
        binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_query(None, 0, None, None, None, None) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_solve_host(None, None, None, 1e-5, 10, ctypes.byref(it), ctypes.byref(rel), None) == \
        binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_solve_host_many(None, 0, None, None, 0, 1e-5, 10, None, None, None) == \
        binding.TPMG_ERR_INVALID_ARG
    lib.tpmg_destroy(None)


def test_status_strings(lib):
    assert lib.tpmg_status_string(0) == b"TPMG_OK"
    assert lib.tpmg_status_string(5) == b"TPMG_ERR_BREAKDOWN"
    assert lib.tpmg_status_string(99) == b"TPMG_UNKNOWN_STATUS"


def declared_learned_functions():
    txt = open(os.path.join(ROOT, "include", "tpmg_learned.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tpmg_[a-z0-9_]+)\s*\(", txt)))


def test_learned_header_and_binding_agree(lib):
    assert declared_learned_functions() == sorted(binding.EXPORTS_LEARNED)
    for name in declared_learned_functions():
        assert hasattr(lib, name), name


def test_kernel_classes_follow_the_header_enum():
    txt = open(os.path.join(ROOT, "include", "tpmg.h")).read()
    names = re.findall(r"TPMG_K_([A-Z]+) = (\d+)", txt)
    order = [n.lower() for n, v in sorted(((n, int(v)) for n, v in names if n != "COUNT"), key=lambda t: t[1])]
    assert order == binding.KERNEL_CLASSES


def test_learned_entry_points_reject_bad_arguments_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.tpmg_net_create(0, 64, None, ctypes.byref(h)) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_net_create(16, 0, None, ctypes.byref(h)) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_net_create(16, 64, None, None) == binding.TPMG_ERR_INVALID_ARG
    assert not h.value
    assert lib.tpmg_net_n_params(None) == 0
    assert lib.tpmg_net_forward(None, None, 1, None) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_net_train_step(None, None, None, 1, 1e-3, None) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_attach_net(None, 0, None) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_record_coarse(None, None, 0) == binding.TPMG_ERR_INVALID_ARG
    assert lib.tpmg_coarse_solve(None, None, None, 1) == binding.TPMG_ERR_INVALID_ARG
    it, rel = ctypes.c_int(), ctypes.c_double()
    assert lib.tpmg_solve_learned(None, None, None, 1e-5, 10, ctypes.byref(it), ctypes.byref(rel), None, None,
                                  None) == binding.TPMG_ERR_INVALID_ARG
    lib.tpmg_net_destroy(None)


def test_setup_profiles_rejects_non_positive_profiles_before_touching_cuda(lib):
    import numpy as np
    p = binding.default_params(refinement=1, n_levels=2, n_r=4)
    for field, n in (("beta_r", 4), ("alphar_r", 5), ("alphaS_s", 80)):
        bad = np.ones(n)
        bad[n // 2] = -1.0 if field != "alphar_r" else 0.0
        prof = binding.tpmg_profiles(**{field: bad.ctypes.data})
        h = ctypes.c_void_p()
        assert lib.tpmg_setup_profiles(ctypes.byref(p), ctypes.byref(prof), None, ctypes.byref(h)) == \
            binding.TPMG_ERR_INVALID_ARG
        assert not h.value
    # the vertical advection may take either sign but must be finite
    for field, n in (("xi_r", 5), ("xi_s", 80)):
        bad = np.ones(n)
        bad[n // 2] = np.nan
        prof = binding.tpmg_profiles(**{field: bad.ctypes.data})
        h = ctypes.c_void_p()
        assert lib.tpmg_setup_profiles(ctypes.byref(p), ctypes.byref(prof), None, ctypes.byref(h)) == \
            binding.TPMG_ERR_INVALID_ARG
        assert not h.value
