"""CPU oracle for the tensor-product multigrid preconditioned-CG path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never imports it, and this
package imports nothing from the product path.

The arithmetic lives in ``tpmg_oracle.c`` (plain single-threaded FP64 C,
compiled with ``-ffp-contract=off``); this module only compiles it and marshals
numpy arrays through ctypes.  Every function of the C file cites the passage of
Dedner, Mueller & Scheichl (arXiv:1408.2981) it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpmg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_tpmg.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle_tpmg.so`` (gcc, C99, -O2)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


_LIB_OMP_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle_tpmg_omp.so")


def build_openmp(force: bool = False) -> str | None:
    """The same source compiled with OpenMP (``oracle/liboracle_tpmg_omp.so``): the
    columns of a colour pass, the operator's rows and the transfers are shared out over
    threads, with the same results bit for bit.  Only a baseline timing uses it.
    None where the compiler has no OpenMP."""
    if (not force and os.path.exists(_LIB_OMP_PATH)
            and os.path.getmtime(_LIB_OMP_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_OMP_PATH
    try:
        return compile_source(_SRC, _LIB_OMP_PATH, openmp=True)
    except (subprocess.CalledProcessError, OSError):
        return None


_libs: dict = {}


def compile_source(src: str, out_path: str, openmp: bool = False) -> str:
    """Compile one oracle C source into a shared library at ``out_path``."""
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           src, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True, stderr=subprocess.DEVNULL if openmp else None)
    os.replace(tmp, out_path)
    return out_path


def threads(n: int = 0, lib_path: str | None = None) -> int:
    """Threads of the parallel loops of a library built with OpenMP (1 without):
    sets n when n > 0, returns the number in use."""
    return int(_load(lib_path).oracle_threads(int(n)))


def _load(path: str | None = None):
    """ctypes handle of the oracle library (the built default, or ``path``)."""
    global _lib
    with _lock:
        key = path or _LIB_PATH
        if key in _libs:
            return _libs[key]
        lib = ctypes.CDLL(path if path else build())
        lib.oracle_create.restype = _P
        lib.oracle_threads.argtypes = [_I]
        lib.oracle_threads.restype = _I
        lib.oracle_create.argtypes = [_I, _I, _I, _D, _D, _D, _D, _I, _I, _I, _I, _D, _I]
        lib.oracle_destroy.argtypes = [_P]
        lib.oracle_info.argtypes = [_P, _P, _P]
        lib.oracle_grid_sizes.argtypes = [_P, _I, _P]
        lib.oracle_export_grid.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P]
        lib.oracle_export_vertical.argtypes = [_P, _P, _P, _P]
        lib.oracle_level_cells.argtypes = [_P, _I]
        lib.oracle_apply.argtypes = [_P, _I, _P, _P]
        lib.oracle_column_blocks.argtypes = [_P, _I, _P, _P, _P]
        lib.oracle_smooth.argtypes = [_P, _I, _P, _P, _I, _I]
        lib.oracle_restrict.argtypes = [_P, _I, _P, _P]
        lib.oracle_prolong_add.argtypes = [_P, _I, _P, _P]
        lib.oracle_vcycle.argtypes = [_P, _P, _P]
        lib.oracle_pcg.argtypes = [_P, _P, _P, _D, _I, _P, _P, _P, _P]
        lib.oracle_fcg.argtypes = [_P, _P, _P, _D, _I, _P, _P, _P, _P]
        lib.oracle_set_vcycle_bf16.argtypes = [_P, _I]
        lib.oracle_set_vcycle_bf16.restype = None
        lib.oracle_set_profiles.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P]
        lib.oracle_set_profiles.restype = None
        lib.oracle_set_outer_profiles.argtypes = [_P, _P, _P, _P, _P]
        lib.oracle_set_outer_profiles.restype = None
        lib.oracle_apply_outer.argtypes = [_P, _P, _P]
        lib.oracle_set_vcycle_full.argtypes = [_P, _I]
        lib.oracle_set_vcycle_full.restype = None
        lib.oracle_set_vcycle_partial.argtypes = [_P, _I]
        lib.oracle_set_vcycle_partial.restype = None
        lib.oracle_set_prolongation.argtypes = [_P, _I]
        lib.oracle_set_prolongation.restype = None
        lib.oracle_set_coarse_solve.argtypes = [_P, COARSE_SOLVE_FN]
        lib.oracle_set_coarse_solve.restype = None
        lib.oracle_bf16.argtypes = [_D]
        lib.oracle_bf16.restype = _D
        lib.oracle_richardson.argtypes = [_P, _P, _P, _I, _P]
        lib.oracle_bicgstab.argtypes = [_P, _P, _P, _D, _I, _P, _P, _P]
        lib.oracle_thomas.argtypes = [_I, _P, _P, _P, _P, _P]
        lib.oracle_column_solve.argtypes = [_I, _P, _P, _P, _P]
        lib.oracle_column_solve2.argtypes = [_I, _P, _P, _P, _P, _P]
        lib.oracle_column_couplings.argtypes = [_P, _I, _P, _P]
        lib.oracle_column_couplings2.argtypes = [_P, _I, _P, _P, _P]
        _libs[key] = lib
        if path is None:
            _lib = lib
        return lib


# coarsest-level solve callback of the V-cycle: (n_cells, n_r, f, u)
COARSE_SOLVE_FN = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def thomas(a, b, c, d, lib_path: str | None = None) -> np.ndarray:
    """Solve tridiag(a, b, c) x = d (a[0], c[-1] unused) with the oracle's Thomas algorithm."""
    a, b, c, d = (_f64(v) for v in (a, b, c, d))
    n = d.shape[0]
    x = np.empty(n)
    if _load(lib_path).oracle_thomas(n, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x)) != 0:
        raise ValueError("oracle_thomas failed")
    return x


def bf16(x: float, lib_path: str | None = None) -> float:
    """x rounded to the nearest bfloat16 value (ties to even), as the oracle rounds coefficients."""
    return _load(lib_path).oracle_bf16(float(x))


def column_solve(c, m, d, lib_path: str | None = None) -> np.ndarray:
    """Solve the column block with couplings c[1..n-1] (c[0] unused) and diagonal
    excess m (diagonal = m_k + c_k + c_{k+1}) for right-hand side d."""
    c, m, d = (_f64(v) for v in (c, m, d))
    n = d.shape[0]
    x = np.empty(n)
    if _load(lib_path).oracle_column_solve(n, _ptr(c), _ptr(m), _ptr(d), _ptr(x)) != 0:
        raise ValueError("oracle_column_solve failed")
    return x


def column_solve2(cd, cu, m, d, lib_path: str | None = None) -> np.ndarray:
    """Solve the non-symmetric column block tridiag(-cd, m + cd + cu, -cu): couplings
    of each row to the row below, cd[1..n-1], and above, cu[0..n-2]."""
    cd, cu, m, d = (_f64(v) for v in (cd, cu, m, d))
    n = d.shape[0]
    x = np.empty(n)
    if _load(lib_path).oracle_column_solve2(n, _ptr(cd), _ptr(cu), _ptr(m), _ptr(d), _ptr(x)) != 0:
        raise ValueError("oracle_column_solve2 failed")
    return x


class Oracle:
    """One oracle problem instance: icosahedral grid hierarchy, vertical grid,
    operator, smoother, V-cycle and PCG, all in FP64 on the host.

    Multigrid level 0 is the coarsest; level ``n_levels - 1`` is the finest
    (refinement ``refinement``).  Field vectors are ``[n_cells * n_r]`` with
    the vertical index fastest.
    """

    SMOOTH_MCSOR = 0
    SMOOTH_JACOBI = 1
    CENTRE_CIRCUM = 0
    CENTRE_VERTEX_MEAN = 1

    def __init__(self, refinement: int, n_levels: int, n_r: int, H: float = 10.0 / 6371.0,
                 grading: float = 1.0, omega2: float = 0.0, courant_c: float = 8.0,
                 nu_pre: int = 2, nu_post: int = 2, nu_coarse: int = 1,
                 smoother: int = 0, relax: float = 1.0, centre_kind: int = 0,
                 lib_path: str | None = None):
        lib = _load(lib_path)
        self._lib = lib
        self._h = lib.oracle_create(refinement, n_levels, n_r, H, grading, omega2, courant_c,
                                    nu_pre, nu_post, nu_coarse, smoother, relax, centre_kind)
        if not self._h:
            raise ValueError("oracle_create rejected the parameters")
        sc = np.zeros(4)
        it = np.zeros(3, dtype=np.int32)
        lib.oracle_info(self._h, _ptr(sc), _ptr(it))
        self.omega2, self.h_min, self.H, self.grading = (float(v) for v in sc)
        self.refinement, self.n_levels, self.n_r = (int(v) for v in it)
        self.nu_pre, self.nu_post, self.nu_coarse = nu_pre, nu_post, nu_coarse
        self.smoother, self.relax, self.centre_kind = smoother, relax, centre_kind

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    # ------------------------------------------------------------- geometry
    def grid_sizes(self, ref: int) -> dict:
        out = np.zeros(4, dtype=np.int32)
        if self._lib.oracle_grid_sizes(self._h, ref, _ptr(out)) != 0:
            raise ValueError("bad refinement level")
        return dict(n_cells=int(out[0]), n_verts=int(out[1]), n_edges=int(out[2]), n_colours=int(out[3]))

    def grid(self, ref: int) -> dict:
        n = self.grid_sizes(ref)["n_cells"]
        out = dict(centre=np.zeros((n, 3)), area=np.zeros(n), nbr=np.zeros((n, 3), dtype=np.int32),
                   g=np.zeros((n, 3)), colour=np.zeros(n, dtype=np.int32), corners=np.zeros((n, 3, 3)))
        self._lib.oracle_export_grid(self._h, ref, _ptr(out["centre"]), _ptr(out["area"]), _ptr(out["nbr"]),
                                     _ptr(out["g"]), _ptr(out["colour"]), _ptr(out["corners"]))
        return out

    def level_ref(self, level: int) -> int:
        return self.refinement - (self.n_levels - 1 - level)

    def level_cells(self, level: int) -> int:
        n = self._lib.oracle_level_cells(self._h, level)
        if n < 0:
            raise ValueError("bad multigrid level")
        return n

    def vertical(self) -> dict:
        r = np.zeros(self.n_r + 1)
        dr = np.zeros(self.n_r)
        vol = np.zeros(self.n_r)
        self._lib.oracle_export_vertical(self._h, _ptr(r), _ptr(dr), _ptr(vol))
        return dict(r=r, dr=dr, vol=vol)

    def size(self, level: int | None = None) -> int:
        level = self.n_levels - 1 if level is None else level
        return self.level_cells(level) * self.n_r

    # ------------------------------------------------------------- operators
    def apply(self, x, level: int | None = None) -> np.ndarray:
        level = self.n_levels - 1 if level is None else level
        x = _f64(x).reshape(-1)
        assert x.shape[0] == self.size(level)
        y = np.empty_like(x)
        self._lib.oracle_apply(self._h, level, _ptr(x), _ptr(y))
        return y

    def column_blocks(self, level: int | None = None):
        level = self.n_levels - 1 if level is None else level
        n = self.level_cells(level)
        sub, diag, sup = (np.zeros((n, self.n_r)) for _ in range(3))
        self._lib.oracle_column_blocks(self._h, level, _ptr(sub), _ptr(diag), _ptr(sup))
        return sub, diag, sup

    def column_couplings(self, level: int | None = None):
        """(c, m) [n_cells, n_r]: coupling to the level below and diagonal excess per row."""
        level = self.n_levels - 1 if level is None else level
        n = self.level_cells(level)
        c, m = np.zeros((n, self.n_r)), np.zeros((n, self.n_r))
        self._lib.oracle_column_couplings(self._h, level, _ptr(c), _ptr(m))
        return c, m

    def column_couplings2(self, level: int | None = None):
        """(cd, cu, m) [n_cells, n_r]: each row's coupling to the row below and above
        (they differ with vertical advection) and the diagonal excess."""
        level = self.n_levels - 1 if level is None else level
        n = self.level_cells(level)
        cd, cu, m = (np.empty((n, self.n_r)) for _ in range(3))
        self._lib.oracle_column_couplings2(self._h, level, _ptr(cd), _ptr(cu), _ptr(m))
        return cd, cu, m

    def smooth(self, f, u, sweeps: int = 1, direction: int = 1, level: int | None = None) -> np.ndarray:
        level = self.n_levels - 1 if level is None else level
        f = _f64(f).reshape(-1)
        u = _f64(u).reshape(-1).copy()
        self._lib.oracle_smooth(self._h, level, _ptr(f), _ptr(u), sweeps, direction)
        return u

    def restrict(self, r_fine, level_fine: int) -> np.ndarray:
        r_fine = _f64(r_fine).reshape(-1)
        out = np.zeros(self.size(level_fine - 1))
        if self._lib.oracle_restrict(self._h, level_fine, _ptr(r_fine), _ptr(out)) != 0:
            raise ValueError("bad level")
        return out

    def prolong_add(self, u_coarse, u_fine, level_fine: int) -> np.ndarray:
        u_coarse = _f64(u_coarse).reshape(-1)
        out = _f64(u_fine).reshape(-1).copy()
        if self._lib.oracle_prolong_add(self._h, level_fine, _ptr(u_coarse), _ptr(out)) != 0:
            raise ValueError("bad level")
        return out

    def vcycle(self, r) -> np.ndarray:
        r = _f64(r).reshape(-1)
        z = np.empty_like(r)
        self._lib.oracle_vcycle(self._h, _ptr(r), _ptr(z))
        return z

    def set_vcycle_bf16(self, on: bool = True):
        """Use the V-cycle of the mixed-precision form (BF16-rounded coefficients,
        FP64 arithmetic) in vcycle(), pcg() and fcg()."""
        self._lib.oracle_set_vcycle_bf16(self._h, 1 if on else 0)

    def set_profiles(self, beta_r=None, alphaS_r=None, alphar_r=None, beta_s=None, alphar_s=None, alphaS_s=None,
                     xi_r=None, xi_s=None):
        """Factorised profiles alpha(r, x) = alpha^r(r) alpha^S(x) (None = 1): vertical
        factors of beta and alpha_S at the cell centres [n_r], of alpha_r at the faces
        [n_r + 1]; horizontal factors on the finest level's cells.  The vertical advection
        xi_r = xi^r(r) xi^S(x) (faces, cells) is absent when both factors are None."""
        arrs = [None if a is None else _f64(a).reshape(-1).copy() for a in
                (beta_r, alphaS_r, alphar_r, beta_s, alphar_s, alphaS_s, xi_r, xi_s)]
        self._profiles = arrs
        self._lib.oracle_set_profiles(self._h, *(_ptr(a) for a in arrs))

    def set_outer_profiles(self, beta=None, alphar=None, alphaS=None, xi=None):
        """General profiles of the problem's operator on the finest level (beta,
        alpha_S [n_cells, n_r], alpha_r and the vertical advection xi [n_cells, n_r + 1];
        None clears; xi None = no advection): the outer iterations apply this operator,
        the V-cycle keeps its own profiles unless set_vcycle_full / _partial."""
        if beta is None:
            self._outer = None
            self._lib.oracle_set_outer_profiles(self._h, None, None, None, None)
            return
        self._outer = [_f64(a).reshape(-1).copy() for a in (beta, alphar, alphaS)]
        self._outer.append(None if xi is None else _f64(xi).reshape(-1).copy())
        self._lib.oracle_set_outer_profiles(self._h, *(_ptr(a) for a in self._outer))

    def set_vcycle_full(self, on: bool = True):
        """The V-cycle's operators use the general profiles of set_outer_profiles
        (TPMG^full) instead of the factorised ones (TPMG^fac)."""
        self._lib.oracle_set_vcycle_full(self._h, 1 if on else 0)

    def set_prolongation(self, linear: bool = True):
        """The V-cycle's prolongation: linear interpolation with a least-squares
        tangent-plane gradient from the 3 coarse neighbours (the paper's Sec. 5), or with
        linear=False the piecewise-constant P = R^T.  The restriction stays the sum."""
        self._lib.oracle_set_prolongation(self._h, 1 if linear else 0)

    def set_vcycle_partial(self, on: bool = True):
        """The V-cycle's operators take alpha_r from the general profiles of
        set_outer_profiles and beta, alpha_S from the factorised ones (TPMG^partial,
        Sec. 5.3); off: the factorised profiles throughout (TPMG^fac)."""
        self._lib.oracle_set_vcycle_partial(self._h, 1 if on else 0)

    def apply_outer(self, x) -> np.ndarray:
        """y = A x with the problem's operator (the general profiles where set)."""
        x = _f64(x).reshape(-1)
        y = np.empty_like(x)
        self._lib.oracle_apply_outer(self._h, _ptr(x), _ptr(y))
        return y

    def set_coarse_solve(self, fn=None):
        """Replace the V-cycle's coarsest-level solve by the guess fn(f [n_cells *
        n_r]) -> u (the learned form's network) followed by one block-Jacobi
        line relaxation; None restores Algorithm 1's sweeps."""
        if fn is None:
            self._coarse_cb = None
            self._lib.oracle_set_coarse_solve(self._h, COARSE_SOLVE_FN())
            return

        def cb(n_cells, n_r, f_ptr, u_ptr):
            n = n_cells * n_r
            f = np.ctypeslib.as_array(f_ptr, shape=(n,)).copy()
            u = np.asarray(fn(f), dtype=np.float64).reshape(n)
            np.ctypeslib.as_array(u_ptr, shape=(n,))[:] = u

        self._coarse_cb = COARSE_SOLVE_FN(cb)   # kept alive while installed
        self._lib.oracle_set_coarse_solve(self._h, self._coarse_cb)

    def pcg(self, f, u0=None, rtol: float = 1e-5, max_iter: int = 100, flexible: bool = False) -> dict:
        """Preconditioned CG; flexible=True uses the Polak-Ribiere coefficient."""
        f = _f64(f).reshape(-1)
        u = np.zeros_like(f) if u0 is None else _f64(u0).reshape(-1).copy()
        iters = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        true_rel = ctypes.c_double(0.0)
        hist = np.zeros(max_iter + 1)
        fn = self._lib.oracle_fcg if flexible else self._lib.oracle_pcg
        status = fn(self._h, _ptr(f), _ptr(u), rtol, max_iter, ctypes.byref(iters),
                    ctypes.byref(rel), _ptr(hist), ctypes.byref(true_rel))
        return dict(u=u, iters=iters.value, rel_resid=rel.value, true_rel=true_rel.value,
                    hist=hist[:iters.value + 1].copy(), status=status)

    def richardson(self, f, u0, n_iter: int) -> tuple[np.ndarray, np.ndarray]:
        f = _f64(f).reshape(-1)
        u = _f64(u0).reshape(-1).copy()
        hist = np.zeros(n_iter + 1)
        self._lib.oracle_richardson(self._h, _ptr(f), _ptr(u), n_iter, _ptr(hist))
        return u, hist

    def bicgstab(self, f, u0=None, rtol: float = 1e-5, max_iter: int = 100) -> dict:
        """BiCGStab preconditioned from the right by one V-cycle per application."""
        f = _f64(f).reshape(-1)
        u = np.zeros_like(f) if u0 is None else _f64(u0).reshape(-1).copy()
        it = np.zeros(1, dtype=np.int32)
        rel = np.zeros(1)
        hist = np.zeros(max_iter + 1)
        st = self._lib.oracle_bicgstab(self._h, _ptr(f), _ptr(u), rtol, max_iter, _ptr(it), _ptr(rel), _ptr(hist))
        return dict(u=u, status=int(st), iters=int(it[0]), rel_resid=float(rel[0]), hist=hist[:int(it[0]) + 1])

    def dense_operator(self, level: int | None = None) -> np.ndarray:
        """Assemble A column by column from the matrix-free apply (tiny grids only)."""
        n = self.size(level)
        if n > 6000:
            raise ValueError("dense assembly is for tiny grids")
        A = np.zeros((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[j] = 1.0
            A[:, j] = self.apply(e, level)
            e[j] = 0.0
        return A
