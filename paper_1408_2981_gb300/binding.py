"""Thin ctypes binding of ``libtpmg.so`` (C ABI declared in ``include/tpmg.h``).

Functions keep the C names (``tpmg_setup``, ``tpmg_apply_operator``,
``tpmg_vcycle``, ``tpmg_solve``, ...).  ``Solver`` wraps a context for torch
float64 CUDA tensors: it only checks shapes/dtypes and passes data pointers
and the current CUDA stream.  Every step of the solve runs in the library's
CUDA kernels; there is no CPU fallback -- if the library is missing or fails
to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtpmg.so")

TPMG_OK = 0
TPMG_ERR_INVALID_ARG = 1
TPMG_ERR_CUDA = 2
TPMG_ERR_OOM = 3
TPMG_ERR_NOT_CONVERGED = 4
TPMG_ERR_BREAKDOWN = 5

TPMG_SMOOTH_MCSOR = 0
TPMG_SMOOTH_JACOBI = 1
TPMG_COEFF_FACTORISED = 0
TPMG_COEFF_FULL = 1
TPMG_COEFF_PARTIAL = 2
TPMG_PROLONG_CONSTANT = 0
TPMG_PROLONG_LINEAR = 1
TPMG_CENTRE_CIRCUM = 0
TPMG_CENTRE_VERTEX_MEAN = 1
TPMG_PREC_FP64 = 0
TPMG_PREC_MIXED = 1
TPMG_OUTER_CG = 0
TPMG_OUTER_RICHARDSON = 1
TPMG_OUTER_BICGSTAB = 2

# every entry point declared in include/tpmg.h
EXPORTS = ["tpmg_default_params", "tpmg_setup", "tpmg_setup_profiles", "tpmg_set_outer_profiles",
           "tpmg_apply_operator", "tpmg_vcycle", "tpmg_vcycle_noalloc",
           "tpmg_solve",
           "tpmg_solve_host", "tpmg_solve_host_many", "tpmg_query", "tpmg_query_tuning", "tpmg_export_mesh", "tpmg_profile", "tpmg_profile_read",
           "tpmg_profile_work", "tpmg_fp64_peak",
           "tpmg_status_string", "tpmg_last_error", "tpmg_destroy", "tpmg_batch_create", "tpmg_batch_run",
           "tpmg_batch_create_ex", "tpmg_batch_form", "tpmg_batch_destroy"]

TPMG_BATCH_AUTO = -1
TPMG_BATCH_BRANCHES = 0
TPMG_BATCH_WORKLIST = 1

# every entry point declared in include/tpmg_learned.h
EXPORTS_LEARNED = ["tpmg_net_create", "tpmg_net_n_params", "tpmg_net_set_params", "tpmg_net_get_params",
                   "tpmg_net_forward", "tpmg_net_gradients", "tpmg_net_train_step", "tpmg_net_last_error",
                   "tpmg_net_destroy", "tpmg_net_features", "tpmg_net_targets", "tpmg_record_coarse",
                   "tpmg_record_count", "tpmg_coarse_solve", "tpmg_attach_net", "tpmg_net_predict", "tpmg_net_fault",
                   "tpmg_vcycle_learned",
                   "tpmg_solve_learned"]

TPMG_NET_COARSE = 0
TPMG_NET_WARM = 1
TPMG_LEARNED_WARM_USED = 1
TPMG_LEARNED_WARM_REJECTED = 2
TPMG_LEARNED_FALLBACK = 4

KERNEL_CLASSES = ["apply", "residual", "restrict", "relax", "prolong", "dot", "axpy", "xpby", "finish", "copy",
                  "net"]


class tpmg_params(ctypes.Structure):
    _fields_ = [("refinement", ctypes.c_int), ("n_levels", ctypes.c_int), ("n_r", ctypes.c_int),
                ("H", ctypes.c_double), ("grading", ctypes.c_double), ("omega2", ctypes.c_double),
                ("courant_c", ctypes.c_double), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("nu_coarse", ctypes.c_int), ("smoother", ctypes.c_int), ("relax", ctypes.c_double),
                ("coeff_storage", ctypes.c_int), ("centre", ctypes.c_int), ("precision", ctypes.c_int),
                ("graphs", ctypes.c_int), ("autotune", ctypes.c_int), ("scan_max_cells", ctypes.c_int),
                ("outer", ctypes.c_int), ("prolongation", ctypes.c_int), ("pdl", ctypes.c_int),
                ("relax_variant", ctypes.c_int), ("scaled_rhs", ctypes.c_int),
                ("net_tcgen05", ctypes.c_int)]


class tpmg_profiles(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("beta_r", "alphaS_r", "alphar_r", "beta_s", "alphar_s", "alphaS_s", "xi_r", "xi_s")]


class TPMGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libtpmg.so and declare its prototypes.  Raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built: run paper_1408_2981_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.tpmg_default_params.argtypes = [ctypes.POINTER(tpmg_params)]
    lib.tpmg_setup.argtypes = [ctypes.POINTER(tpmg_params), P, ctypes.POINTER(P)]
    lib.tpmg_setup_profiles.argtypes = [ctypes.POINTER(tpmg_params), ctypes.POINTER(tpmg_profiles), P,
                                        ctypes.POINTER(P)]
    lib.tpmg_apply_operator.argtypes = [P, P, P]
    lib.tpmg_set_outer_profiles.argtypes = [P, P, P, P, P]
    lib.tpmg_vcycle.argtypes = [P, P, P]
    lib.tpmg_vcycle_noalloc.argtypes = [P, P, P]
    lib.tpmg_solve.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.tpmg_solve_host.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    lib.tpmg_solve_host_many.argtypes = [P, I, P, P, I, D, I, P, P, P]
    lib.tpmg_query.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.tpmg_export_mesh.argtypes = [P, I, P, P, P, P, P, P]
    lib.tpmg_query_tuning.argtypes = [P, I, ctypes.POINTER(I), P]
    lib.tpmg_profile.argtypes = [P, ctypes.c_uint]
    lib.tpmg_profile_read.argtypes = [P, I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D), ctypes.POINTER(D),
                                      ctypes.POINTER(ctypes.c_longlong)]
    lib.tpmg_profile_work.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.tpmg_fp64_peak.argtypes = [P, ctypes.POINTER(D)]
    lib.tpmg_status_string.argtypes = [I]
    lib.tpmg_status_string.restype = ctypes.c_char_p
    lib.tpmg_last_error.argtypes = [P]
    lib.tpmg_last_error.restype = ctypes.c_char_p
    lib.tpmg_destroy.argtypes = [P]
    lib.tpmg_destroy.restype = None
    lib.tpmg_batch_create.argtypes = [P, I, P, P, D, I, ctypes.POINTER(P)]
    lib.tpmg_batch_run.argtypes = [P, P, P, P, P, ctypes.POINTER(ctypes.c_longlong)]
    lib.tpmg_batch_create_ex.argtypes = [P, I, P, P, D, I, I, I, ctypes.POINTER(P)]
    lib.tpmg_batch_form.argtypes = [P]
    lib.tpmg_batch_form.restype = I
    lib.tpmg_batch_destroy.argtypes = [P]
    lib.tpmg_batch_destroy.restype = None
    L, F, LL = ctypes.c_long, ctypes.c_float, ctypes.c_longlong
    lib.tpmg_net_create.argtypes = [I, I, P, ctypes.POINTER(P)]
    lib.tpmg_net_n_params.argtypes = [P]
    lib.tpmg_net_n_params.restype = ctypes.c_size_t
    lib.tpmg_net_set_params.argtypes = [P, P]
    lib.tpmg_net_get_params.argtypes = [P, P]
    lib.tpmg_net_forward.argtypes = [P, P, L, P]
    lib.tpmg_net_gradients.argtypes = [P, P, P, L, P, P]
    lib.tpmg_net_train_step.argtypes = [P, P, P, L, F, P]
    lib.tpmg_net_last_error.argtypes = [P]
    lib.tpmg_net_last_error.restype = ctypes.c_char_p
    lib.tpmg_net_destroy.argtypes = [P]
    lib.tpmg_net_destroy.restype = None
    lib.tpmg_net_features.argtypes = [P, I, P, P, L, P, P]
    lib.tpmg_net_targets.argtypes = [P, I, P, P, P, L, P]
    lib.tpmg_record_coarse.argtypes = [P, P, I]
    lib.tpmg_record_count.argtypes = [P, ctypes.POINTER(I)]
    lib.tpmg_coarse_solve.argtypes = [P, P, P, I]
    lib.tpmg_attach_net.argtypes = [P, I, P]
    lib.tpmg_vcycle_learned.argtypes = [P, P, P]
    lib.tpmg_net_predict.argtypes = [P, I, P, P]
    lib.tpmg_net_fault.argtypes = [P, ctypes.POINTER(I)]
    lib.tpmg_solve_learned.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I),
                                       ctypes.POINTER(I), ctypes.POINTER(LL)]
    no_status = ("tpmg_destroy", "tpmg_status_string", "tpmg_last_error", "tpmg_batch_destroy", "tpmg_net_n_params",
                 "tpmg_net_last_error", "tpmg_net_destroy")
    for name in EXPORTS + EXPORTS_LEARNED:
        if name not in no_status:
            getattr(lib, name).restype = I
    if path is None:
        _lib = lib
    return lib


def fp64_peak_tflops(stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s (tpmg_fp64_peak)."""
    import torch

    lib = load()
    stream = stream or torch.cuda.current_stream()
    t = ctypes.c_double()
    st = lib.tpmg_fp64_peak(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(t))
    if st != TPMG_OK:
        raise TPMGError(st, "tpmg_fp64_peak")
    return t.value


def status_name(status: int) -> str:
    try:
        return load().tpmg_status_string(status).decode()
    except Exception:
        return f"status {status}"


def default_params(**overrides) -> tpmg_params:
    p = tpmg_params()
    st = load().tpmg_default_params(ctypes.byref(p))
    if st != TPMG_OK:
        raise TPMGError(st, "tpmg_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t) -> int:
    return t.data_ptr()


class Solver:
    """A tpmg context bound to the current CUDA device and stream.

    Keyword arguments are the fields of ``tpmg_params``.  Vectors are torch
    float64 CUDA tensors with ``n_cells * n_r`` elements ([cell][k], k fastest).
    ``profiles``: optional dict of factorised profiles (the fields of
    ``tpmg_profiles``, numpy float64 arrays; absent = 1, except the vertical
    advection xi_r, xi_s: both absent = none).
    """

    def __init__(self, stream=None, profiles=None, **params):
        import torch

        self._torch = torch
        self._lib = load()
        self.params = default_params(**params)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        if profiles:
            arrs = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in profiles.items()}
            unknown = set(arrs) - {f[0] for f in tpmg_profiles._fields_}
            if unknown:
                raise KeyError(sorted(unknown))
            prof = tpmg_profiles(**{k: a.ctypes.data for k, a in arrs.items()})
            st = self._lib.tpmg_setup_profiles(ctypes.byref(self.params), ctypes.byref(prof),
                                               ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        else:
            st = self._lib.tpmg_setup(ctypes.byref(self.params), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != TPMG_OK:
            raise TPMGError(st, "tpmg_setup rejected the parameters or failed")
        self._h = h
        self.n_levels = self.params.n_levels
        self.n_r = self.params.n_r
        self.n_cells, _, self.omega2, self.n_colours = self.query(self.n_levels - 1)
        self.N = self.n_cells * self.n_r

    # --------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.tpmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != TPMG_OK:
            raise TPMGError(st, f"{what}: {self._lib.tpmg_last_error(self._h).decode()}")

    def _vec(self, t, name: str):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError(f"{name} must be a float64 CUDA tensor")
        if t.numel() != self.N or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with {self.N} elements")
        return _ptr(t)

    # --------------------------------------------------------------- queries
    def query(self, level: int):
        n, nr, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        w = ctypes.c_double()
        st = self._lib.tpmg_query(self._h, level, ctypes.byref(n), ctypes.byref(nr), ctypes.byref(w), ctypes.byref(c))
        if st != TPMG_OK:
            raise TPMGError(st, "tpmg_query")
        return n.value, nr.value, w.value, c.value

    def tuning(self) -> list:
        """Per level (coarsest first): (chosen relaxation variant, microseconds of each variant)."""
        out = []
        for level in range(self.n_levels):
            v = ctypes.c_int()
            us = np.zeros(5, dtype=np.float32)
            st = self._lib.tpmg_query_tuning(self._h, level, ctypes.byref(v), us.ctypes.data)
            if st != TPMG_OK:
                raise TPMGError(st, "tpmg_query_tuning")
            out.append((v.value, us.tolist()))
        return out

    def export_mesh(self, level: int | None = None) -> dict:
        level = self.n_levels - 1 if level is None else level
        n = self.query(level)[0]
        out = dict(centres=np.zeros((n, 3)), areas=np.zeros(n), nbrs=np.zeros((n, 3), dtype=np.int32),
                   g=np.zeros((n, 3)), colour=np.zeros(n, dtype=np.int32), r_faces=np.zeros(self.n_r + 1))
        st = self._lib.tpmg_export_mesh(self._h, level, *(out[k].ctypes.data for k in
                                                           ("centres", "areas", "nbrs", "g", "colour", "r_faces")))
        if st != TPMG_OK:
            raise TPMGError(st, "tpmg_export_mesh")
        return out

    # --------------------------------------------------------------- tracing
    def profile(self, classes=()):
        """Reset the counters; time the named kernel classes (see KERNEL_CLASSES)."""
        mask = 0
        for c in classes:
            mask |= 1 << KERNEL_CLASSES.index(c)
        self._check(self._lib.tpmg_profile(self._h, mask), "tpmg_profile")

    def profile_read(self) -> dict:
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            n, ms, units, timed = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
            self._check(self._lib.tpmg_profile_read(self._h, i, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(units),
                                                    ctypes.byref(timed)), "tpmg_profile_read")
            b, tb, fl, tfl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            self._check(self._lib.tpmg_profile_work(self._h, i, ctypes.byref(b), ctypes.byref(tb), ctypes.byref(fl),
                                                    ctypes.byref(tfl)), "tpmg_profile_work")
            out[name] = dict(launches=n.value, ms=ms.value, units=units.value, timed=timed.value, bytes=b.value,
                             timed_bytes=tb.value, flops=fl.value, timed_flops=tfl.value)
        return out

    def set_outer_profiles(self, beta=None, alphar=None, alphaS=None, xi=None):
        """The problem's operator with general profiles on the finest level (numpy
        arrays: beta, alphaS [n_cells, n_r], alphar and the vertical advection xi
        [n_cells, n_r + 1]; xi None = no advection); None restores the factorised
        operator.  The V-cycle follows its coefficient storage: FACTORISED keeps the
        profiles of the set-up (TPMG^fac), FULL adopts all of them (TPMG^full), PARTIAL
        adopts alpha_r (TPMG^partial)."""
        if beta is None:
            self._check(self._lib.tpmg_set_outer_profiles(self._h, None, None, None, None), "tpmg_set_outer_profiles")
            return
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (beta, alphar, alphaS)]
        xa = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64).reshape(-1)
        self._check(self._lib.tpmg_set_outer_profiles(self._h, *(a.ctypes.data for a in arrs),
                                                      None if xa is None else xa.ctypes.data),
                    "tpmg_set_outer_profiles")

    # --------------------------------------------------------------- compute
    def apply_operator(self, x, y):
        self._check(self._lib.tpmg_apply_operator(self._h, self._vec(x, "x"), self._vec(y, "y")), "tpmg_apply_operator")

    def vcycle(self, r, z):
        self._check(self._lib.tpmg_vcycle(self._h, self._vec(r, "r"), self._vec(z, "z")), "tpmg_vcycle")

    def vcycle_noalloc(self, r, z):
        """z = B r like vcycle(), with the coarse-level work vectors in the
        library's fixed device array instead of the context's (no allocation)."""
        self._check(self._lib.tpmg_vcycle_noalloc(self._h, self._vec(r, "r"), self._vec(z, "z")),
                    "tpmg_vcycle_noalloc")

    def solve(self, f, u, rtol: float = 1e-5, max_iter: int = 100, history: bool = False, raise_on_fail: bool = True):
        """PCG; u holds the initial guess and receives the solution.
        Returns (status, iters, rel_resid, hist)."""
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        hist = np.zeros(max_iter + 1) if history else None
        st = self._lib.tpmg_solve(self._h, self._vec(f, "f"), self._vec(u, "u"), rtol, max_iter, ctypes.byref(it),
                                  ctypes.byref(rel), hist.ctypes.data if history else None)
        if raise_on_fail and st not in (TPMG_OK,):
            self._check(st, "tpmg_solve")
        return st, it.value, rel.value, (hist[:it.value + 1] if history else None)

    def solve_host(self, f: np.ndarray, u: np.ndarray, rtol: float = 1e-5, max_iter: int = 100,
                   raise_on_fail: bool = True):
        """PCG on host buffers (copies inside the call).  u is updated in place."""
        for a, name in ((f, "f"), (u, "u")):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
                    and a.size == self.N):
                raise ValueError(f"{name} must be a contiguous float64 array of {self.N} elements")
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = self._lib.tpmg_solve_host(self._h, f.ctypes.data, u.ctypes.data, rtol, max_iter, ctypes.byref(it),
                                       ctypes.byref(rel), None)
        if raise_on_fail and st != TPMG_OK:
            self._check(st, "tpmg_solve_host")
        return st, it.value, rel.value

    def solve_host_many(self, fs, us, guess: bool = False, rtol: float = 1e-5, max_iter: int = 100,
                        raise_on_fail: bool = True):
        """Solves A u_j = f_j for host arrays fs[j], us[j] (us[j] receives the solution, and
        holds the initial guess when guess is true), with the copies of the neighbouring
        systems overlapping each solve.  Returns (status, iters[n], rel_resid[n], status[n])."""
        n = len(fs)
        if len(us) != n:
            raise ValueError("fs and us must have the same length")
        for j in range(n):
            for a, name in ((fs[j], f"fs[{j}]"), (us[j], f"us[{j}]")):
                if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
                        and a.size == self.N):
                    raise ValueError(f"{name} must be a contiguous float64 array of {self.N} elements")
        pf = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in fs])
        pu = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in us])
        it = np.zeros(max(n, 1), dtype=np.int32)
        rel = np.zeros(max(n, 1))
        sts = np.zeros(max(n, 1), dtype=np.int32)
        st = self._lib.tpmg_solve_host_many(self._h, n, pf, pu, 1 if guess else 0, rtol, max_iter, it.ctypes.data,
                                            rel.ctypes.data, sts.ctypes.data)
        if raise_on_fail and st != TPMG_OK:
            self._check(st, "tpmg_solve_host_many")
        return st, it[:n].copy(), rel[:n].copy(), sts[:n].copy()


    # --------------------------------------------------------------- learned form
    def _level_vec(self, t, level: int, name: str, dtype=None):
        torch = self._torch
        dtype = dtype or torch.float64
        n = self.query(level)[0] * self.n_r
        if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
        if t.numel() != n:
            raise ValueError(f"{name} must have {n} elements (level {level})")
        return _ptr(t)

    @staticmethod
    def _rows(cells, rows):
        if cells is None:
            return None, rows
        import torch
        if cells.dtype != torch.int32 or not cells.is_cuda or not cells.is_contiguous():
            raise TypeError("cells must be a contiguous int32 CUDA tensor")
        return _ptr(cells), cells.numel()

    def net_features(self, level: int, f, x, cells=None) -> float:
        """x [rows, 2 n_r] float32 <- the network inputs of the columns `cells`
        (int32 CUDA tensor; None = every column) of f on `level`.  Returns s."""
        cp, rows = self._rows(cells, self.query(level)[0])
        if x.dtype != self._torch.float32 or not x.is_cuda or x.numel() != rows * 2 * self.n_r or not x.is_contiguous():
            raise ValueError("x must be a contiguous float32 CUDA tensor of rows x 2 n_r")
        s = ctypes.c_double()
        self._check(self._lib.tpmg_net_features(self._h, level, self._level_vec(f, level, "f"), cp, rows, _ptr(x),
                                                ctypes.byref(s)), "tpmg_net_features")
        return s.value

    def net_targets(self, level: int, f, u, t, cells=None):
        """t [rows, n_r] float32 <- u / s (s of f) on the columns `cells`."""
        cp, rows = self._rows(cells, self.query(level)[0])
        if t.dtype != self._torch.float32 or not t.is_cuda or t.numel() != rows * self.n_r or not t.is_contiguous():
            raise ValueError("t must be a contiguous float32 CUDA tensor of rows x n_r")
        self._check(self._lib.tpmg_net_targets(self._h, level, self._level_vec(f, level, "f"),
                                               self._level_vec(u, level, "u"), cp, rows, _ptr(t)), "tpmg_net_targets")

    def record_coarse(self, buf=None, capacity: int = 0):
        """Record the coarsest-level right-hand side of every V-cycle into buf
        (float64 CUDA tensor of capacity x n_cells(0) x n_r); None stops."""
        if buf is None:
            self._check(self._lib.tpmg_record_coarse(self._h, None, 0), "tpmg_record_coarse")
            return
        n0 = self.query(0)[0] * self.n_r
        if buf.dtype != self._torch.float64 or not buf.is_cuda or buf.numel() < capacity * n0:
            raise ValueError("buf must be a float64 CUDA tensor of at least capacity x n_cells(0) x n_r")
        self._rec = buf
        self._check(self._lib.tpmg_record_coarse(self._h, _ptr(buf), capacity), "tpmg_record_coarse")

    def record_count(self) -> int:
        c = ctypes.c_int()
        self._check(self._lib.tpmg_record_count(self._h, ctypes.byref(c)), "tpmg_record_count")
        return c.value

    def coarse_solve(self, f0, u0, sweeps: int):
        """u0 <- coarsest-level solution of f0 by `sweeps` symmetric line-relaxation sweeps."""
        self._check(self._lib.tpmg_coarse_solve(self._h, self._level_vec(f0, 0, "f0"), self._level_vec(u0, 0, "u0"),
                                                sweeps), "tpmg_coarse_solve")

    def attach_net(self, role: int, net):
        if not hasattr(self, "_nets"):
            self._nets = {}
        self._check(self._lib.tpmg_attach_net(self._h, role, net._h if net is not None else None), "tpmg_attach_net")
        self._nets[role] = net   # keep the network alive while attached

    def net_predict(self, role: int, f, u):
        """u = s network(features(f)) of the network attached in `role` on its level."""
        level = 0 if role == TPMG_NET_COARSE else self.n_levels - 1
        self._check(self._lib.tpmg_net_predict(self._h, role, self._level_vec(f, level, "f"),
                                               self._level_vec(u, level, "u")), "tpmg_net_predict")

    def net_fault(self) -> bool:
        """True if a tcgen05 network kernel of this context gave up waiting (outputs NaN)."""
        flag = ctypes.c_int()
        self._check(self._lib.tpmg_net_fault(self._h, ctypes.byref(flag)), "tpmg_net_fault")
        return bool(flag.value)

    def vcycle_learned(self, r, z):
        """z = B r with the attached COARSE network as the coarsest-level solve."""
        self._check(self._lib.tpmg_vcycle_learned(self._h, self._vec(r, "r"), self._vec(z, "z")), "tpmg_vcycle_learned")

    def solve_learned(self, f, u, rtol: float = 1e-5, max_iter: int = 100, raise_on_fail: bool = True):
        """Flexible CG with the attached networks, stop at ||r|| <= rtol ||f||.
        Returns (status, iters, rel_resid, info bits, fallback_iters, kernel_launches)."""
        it, fb, info = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        launches = ctypes.c_longlong(0)
        st = self._lib.tpmg_solve_learned(self._h, self._vec(f, "f"), self._vec(u, "u"), rtol, max_iter,
                                          ctypes.byref(it), ctypes.byref(rel), ctypes.byref(info), ctypes.byref(fb),
                                          ctypes.byref(launches))
        if raise_on_fail and st != TPMG_OK:
            self._check(st, "tpmg_solve_learned")
        return st, it.value, rel.value, info.value, fb.value, launches.value


class Net:
    """tpmg_net: the learned form's per-column network (include/tpmg_learned.h).

    Tensors are float32 CUDA tensors; ``x`` [rows, 2 n_r], ``t``/``y`` [rows, n_r].
    """

    def __init__(self, n_r: int, hidden: int = 64, stream=None):
        import torch

        self._torch = torch
        self._lib = load()
        stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self._lib.tpmg_net_create(n_r, hidden, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != TPMG_OK:
            raise TPMGError(st, "tpmg_net_create")
        self._h = h
        self.n_r, self.hidden = n_r, hidden
        self.sizes = [2 * n_r, hidden, hidden, hidden, n_r]
        self.n_params = int(self._lib.tpmg_net_n_params(h))

    def _check(self, st: int, what: str):
        if st != TPMG_OK:
            raise TPMGError(st, f"{what}: {self._lib.tpmg_net_last_error(self._h).decode()}")

    def _f32(self, t, cols: int, name: str) -> int:
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if t.numel() % cols:
            raise ValueError(f"{name} must have a multiple of {cols} elements")
        return _ptr(t)

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        self._check(self._lib.tpmg_net_set_params(self._h, a.ctypes.data), "tpmg_net_set_params")

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        self._check(self._lib.tpmg_net_get_params(self._h, a.ctypes.data), "tpmg_net_get_params")
        return a

    def unflatten(self, flat: np.ndarray) -> list:
        """[(W_l [out, in], b_l [out])] of a flat parameter vector."""
        out, off = [], 0
        for i, o in zip(self.sizes[:-1], self.sizes[1:]):
            W = flat[off:off + o * i].reshape(o, i)
            off += o * i
            b = flat[off:off + o]
            off += o
            out.append((W, b))
        return out

    def forward(self, x, y):
        rows = x.numel() // (2 * self.n_r)
        self._check(self._lib.tpmg_net_forward(self._h, self._f32(x, 2 * self.n_r, "x"), rows,
                                               self._f32(y, self.n_r, "y")), "tpmg_net_forward")

    def gradients(self, x, t, grad) -> float:
        rows = x.numel() // (2 * self.n_r)
        loss = ctypes.c_double()
        self._check(self._lib.tpmg_net_gradients(self._h, self._f32(x, 2 * self.n_r, "x"), self._f32(t, self.n_r, "t"),
                                                 rows, self._f32(grad, 1, "grad"), ctypes.byref(loss)),
                    "tpmg_net_gradients")
        return loss.value

    def train_step(self, x, t, lr: float, want_loss: bool = False):
        rows = x.numel() // (2 * self.n_r)
        loss = ctypes.c_double()
        self._check(self._lib.tpmg_net_train_step(self._h, self._f32(x, 2 * self.n_r, "x"),
                                                  self._f32(t, self.n_r, "t"), rows, float(lr),
                                                  ctypes.byref(loss) if want_loss else None), "tpmg_net_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tpmg_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """tpmg_batch: one PCG solve per (Solver, right-hand side) in one graph launch.

    ``solvers``, ``fs``, ``us``: equal-length lists; fs[i], us[i] are float64 CUDA
    tensors of solvers[i] (us[i] = initial guess, overwritten by the solution).
    A Solver may appear several times (several right-hand sides on one operator)
    when the batch takes the work-list form (``form == "worklist"``: every Solver
    mixed precision with the defaults of the CG path).  The tensors must stay
    alive while the batch is used.
    """

    def __init__(self, solvers, fs, us, rtol: float = 1e-5, max_iter: int = 100, form: str = "auto", groups: int = 0):
        if not (len(solvers) == len(fs) == len(us)) or not solvers:
            raise ValueError("solvers, fs and us must be non-empty lists of equal length")
        self._lib = load()
        self.solvers, self.fs, self.us = list(solvers), list(fs), list(us)
        n = len(solvers)
        self.n = n
        ctxs = (ctypes.c_void_p * n)(*[s._h.value for s in solvers])
        fp = (ctypes.c_void_p * n)(*[s._vec(f, "f") for s, f in zip(solvers, fs)])
        up = (ctypes.c_void_p * n)(*[s._vec(u, "u") for s, u in zip(solvers, us)])
        h = ctypes.c_void_p()
        fcode = {"auto": TPMG_BATCH_AUTO, "branches": TPMG_BATCH_BRANCHES, "worklist": TPMG_BATCH_WORKLIST}[form]
        st = self._lib.tpmg_batch_create_ex(ctxs, n, fp, up, rtol, max_iter, fcode, groups, ctypes.byref(h))
        if st != TPMG_OK:
            raise TPMGError(st, "tpmg_batch_create")
        self._h = h
        self.form = {TPMG_BATCH_BRANCHES: "branches", TPMG_BATCH_WORKLIST: "worklist"}[self._lib.tpmg_batch_form(h)]

    def run(self, stream=None):
        """Returns (status, iters[n], rel_resid[n], status[n], kernel_launches)."""
        import torch

        stream = stream if stream is not None else torch.cuda.current_stream()
        it = np.zeros(self.n, dtype=np.int32)
        rel = np.zeros(self.n)
        sts = np.zeros(self.n, dtype=np.int32)
        launches = ctypes.c_longlong(0)
        st = self._lib.tpmg_batch_run(self._h, ctypes.c_void_p(stream.cuda_stream), it.ctypes.data, rel.ctypes.data,
                                      sts.ctypes.data, ctypes.byref(launches))
        return st, it, rel, sts, launches.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tpmg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
