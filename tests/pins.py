"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` function takes a namespace ``ns`` with ``ns.Oracle`` (the oracle
class, or a variant bound to another build of the oracle) and ``ns.thomas``, and
raises ``AssertionError`` when the oracle disagrees with the fixed fact.  The
pins are used twice: on the real oracle (``test_oracle_pins.py``) and on
copies of the oracle with a planted mistake (``test_oracle_mutants.py``), which
must each fail at least one pin.

Citations are to Dedner, Mueller & Scheichl, arXiv:1408.2981.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from paper_1408_2981_gb300 import inputs

EPS = np.finfo(np.float64).eps
FOUR_PI = 4.0 * math.pi


# ----------------------------------------------------------------------------- grid
def pin_mesh_counts(ns, max_ref: int = 4):
    """Sec. 4.1: each coarse triangle holds four fine ones.  A closed triangulated
    sphere refined by bisection has F = 20*4^L, E = 30*4^L, V = 10*4^L + 2 (Euler V-E+F = 2)."""
    o = ns.Oracle(refinement=max_ref, n_levels=1, n_r=1)
    for ref in range(max_ref + 1):
        s = o.grid_sizes(ref)
        assert s["n_cells"] == 20 * 4 ** ref
        assert s["n_edges"] == 30 * 4 ** ref
        assert s["n_verts"] == 10 * 4 ** ref + 2
        assert s["n_verts"] - s["n_edges"] + s["n_cells"] == 2


def pin_mesh_areas(ns, max_ref: int = 5):
    """Spherical areas tile the unit sphere (sum 4 pi); the four children of a cell
    tile it exactly; the 20 faces of the icosahedron are congruent (4 pi / 20)."""
    o = ns.Oracle(refinement=max_ref, n_levels=1, n_r=1)
    prev = None
    for ref in range(max_ref + 1):
        a = o.grid(ref)["area"]
        assert abs(a.sum() - FOUR_PI) <= 64 * EPS * FOUR_PI
        if ref == 0:
            np.testing.assert_allclose(a, FOUR_PI / 20.0, rtol=16 * EPS, atol=0)
        if prev is not None:
            np.testing.assert_allclose(a.reshape(-1, 4).sum(axis=1), prev, rtol=32 * EPS * 2 ** ref, atol=0)
        prev = a


def pin_level0_closed_forms(ns):
    """Regular icosahedron: adjacent vertices subtend arccos(1/sqrt5); adjacent face
    centres subtend pi - dihedral = arccos(sqrt5/3); by symmetry the centre chord is
    normal to the shared edge, so g = |S| / |r_T' - r_T| for every edge (Appendix A)."""
    S = math.acos(1.0 / math.sqrt(5.0))
    theta = math.acos(math.sqrt(5.0) / 3.0)
    d = 2.0 * math.sin(0.5 * theta)
    for ck in (0, 1):
        o = ns.Oracle(refinement=0, n_levels=1, n_r=1, centre_kind=ck)
        g = o.grid(0)
        np.testing.assert_allclose(g["g"], S / d, rtol=64 * EPS, atol=0)
        c = g["centre"]
        for T in range(20):
            for e in range(3):
                Tp = g["nbr"][T, e]
                np.testing.assert_allclose(np.linalg.norm(c[Tp] - c[T]), d, rtol=64 * EPS)
        corners = g["corners"]
        dots = np.einsum("tij,tj->ti", corners, c)
        np.testing.assert_allclose(dots, dots[0, 0], rtol=64 * EPS)


def pin_mesh_topology(ns, max_ref: int = 4):
    """Neighbour relation symmetric, cells counter-clockwise seen from outside,
    the centre child 4T of a refined cell borders exactly its three siblings,
    colouring valid with exactly 3 colours (the 5 cells around an original
    icosahedron vertex form an odd cycle, so 2 never suffice; Brooks' theorem
    guarantees 3 for this cubic planar graph and the saturation-degree order
    finds them), g_TT' > 0 and g_TT' = g_T'T, vertices and centres on the unit
    sphere, circumcentres equidistant from the corners."""
    for ck in (0, 1):
        o = ns.Oracle(refinement=max_ref, n_levels=1, n_r=1, centre_kind=ck)
        for ref in range(max_ref + 1):
            g = o.grid(ref)
            n = g["area"].shape[0]
            nbr, gg, col, cen, cor = g["nbr"], g["g"], g["colour"], g["centre"], g["corners"]
            assert np.all((nbr >= 0) & (nbr < n))
            for T in range(n):
                for e in range(3):
                    Tp = nbr[T, e]
                    assert Tp != T
                    back = np.where(nbr[Tp] == T)[0]
                    assert back.shape[0] == 1
                    assert gg[Tp, back[0]] == gg[T, e]
                    assert col[Tp] != col[T]
                    # the shared edge is (v_e, v_e+1) of T and appears reversed in T'
                    p, q = cor[T, e], cor[T, (e + 1) % 3]
                    ep = back[0]
                    np.testing.assert_array_equal(cor[Tp, ep], q)
                    np.testing.assert_array_equal(cor[Tp, (ep + 1) % 3], p)
            assert col.max() == 2 and col.min() >= 0
            assert np.all(gg > 0)
            np.testing.assert_allclose(np.linalg.norm(cor, axis=2), 1.0, rtol=4 * EPS)
            np.testing.assert_allclose(np.linalg.norm(cen, axis=1), 1.0, rtol=4 * EPS)
            orient = np.einsum("ti,ti->t", np.cross(cor[:, 1] - cor[:, 0], cor[:, 2] - cor[:, 0]), cen)
            assert np.all(orient > 0)
            if ck == 0:
                dd = np.einsum("tij,tj->ti", cor, cen)
                np.testing.assert_allclose(dd, dd[:, :1] * np.ones((1, 3)), rtol=64 * EPS)
            if ref > 0:
                for T in range(n // 4):
                    assert sorted(nbr[4 * T].tolist()) == [4 * T + 1, 4 * T + 2, 4 * T + 3]
                # children lie inside the parent: corners of child j=1..3 include a parent corner
                gp = o.grid(ref - 1)["corners"]
                for T in range(n // 4):
                    np.testing.assert_array_equal(cor[4 * T + 1, 0], gp[T, 0])
                    np.testing.assert_array_equal(cor[4 * T + 2, 1], gp[T, 1])
                    np.testing.assert_array_equal(cor[4 * T + 3, 2], gp[T, 2])


def pin_vertical(ns):
    """Appendix A: 1 = r_0 < ... < r_nr = 1 + H; v_k = (r_{k+1}^3 - r_k^3)/3, so the
    v_k telescope to ((1+H)^3 - 1)/3 and equal dr (r_mid^2 + dr^2/12) exactly;
    geometric grading has a constant ratio dr_{k+1}/dr_k."""
    for n_r, gr, H in [(16, 1.0, 10.0 / 6371.0), (64, 1.05, 10.0 / 6371.0), (7, 1.3, 0.5), (1, 1.0, 0.25)]:
        o = ns.Oracle(refinement=0, n_levels=1, n_r=n_r, H=H, grading=gr)
        v = o.vertical()
        r, dr, vol = v["r"], v["dr"], v["vol"]
        assert r[0] == 1.0 and abs(r[-1] - (1.0 + H)) <= EPS
        assert np.all(dr > 0)
        assert abs(dr.sum() - H) <= 8 * n_r * EPS * H
        exact = H * (3.0 + 3.0 * H + H * H) / 3.0
        assert abs(vol.sum() - exact) <= 8 * n_r * EPS * exact
        rm = 0.5 * (r[:-1] + r[1:])
        np.testing.assert_allclose(vol, dr * (rm * rm + dr * dr / 12.0), rtol=16 * EPS)
        if gr == 1.0:
            np.testing.assert_allclose(dr, H / n_r, rtol=1e-10)
        else:
            np.testing.assert_allclose(dr[1:] / dr[:-1], gr, rtol=1e-9)


# ----------------------------------------------------------------------------- operator
SMALL_CASES = [
    dict(refinement=1, n_levels=2, n_r=5, grading=1.2, H=0.05, courant_c=8.0),
    dict(refinement=2, n_levels=3, n_r=3, grading=1.0, courant_c=80.0),
    dict(refinement=0, n_levels=1, n_r=9, grading=1.05, courant_c=8.0, centre_kind=1),
]


def _vertical_matrix(o):
    """The vertical factor K = diag(v) + omega^2 V^r of the Kronecker form
    (Sec. 3.2.1, A = (omega^2 A^r + B^r) (x) M^S + omega^2 M^r (x) A^S), from the
    exported vertical grid: face coupling 2 r_k^2 / (r_{k+1} - r_{k-1}) (eq. VerticalDiffusion)."""
    v = o.vertical()
    r, vol = v["r"], v["vol"]
    n_r = o.n_r
    z = r - 1.0
    a = np.zeros(n_r + 1)
    if n_r > 1:
        a[1:n_r] = 2.0 * r[1:n_r] ** 2 / (z[2:] - z[:-2])
    Vr = np.diag(a[:-1] + a[1:]) - np.diag(a[1:-1], 1) - np.diag(a[1:-1], -1)
    return np.diag(vol) + o.omega2 * Vr, np.diag(v["dr"])


def _horizontal_laplacian(g):
    n = g["area"].shape[0]
    Lh = np.zeros((n, n))
    for T in range(n):
        for e in range(3):
            Lh[T, T] += g["g"][T, e]
            Lh[T, g["nbr"][T, e]] -= g["g"][T, e]
    return Lh


def pin_constants_in_kernel(ns):
    """The diffusion terms are flux differences that vanish on constants
    (Appendix A), so A 1 = beta_hat = |T| v_k on every level -- exactly, since
    every flux multiplies a difference 1 - 1 = 0."""
    for kw in SMALL_CASES + [dict(refinement=4, n_levels=3, n_r=16, grading=1.05, courant_c=80.0)]:
        o = ns.Oracle(**kw)
        v = o.vertical()
        for level in range(o.n_levels):
            g = o.grid(o.level_ref(level))
            y = o.apply(np.ones(o.size(level)), level)
            np.testing.assert_array_equal(y, np.outer(g["area"], v["vol"]).reshape(-1))


def pin_symmetric_spd(ns):
    """With xi = 0 and constant profiles the operator is symmetric positive
    definite (Sec. 3.2.1); the two-point fluxes also make it an M-matrix: positive
    diagonal, non-positive off-diagonals, strict diagonal dominance (beta_hat > 0)."""
    for kw in SMALL_CASES:
        o = ns.Oracle(**kw)
        for level in range(o.n_levels):
            A = o.dense_operator(level)
            assert np.array_equal(A, A.T)
            np.linalg.cholesky(A)
            off = A - np.diag(np.diag(A))
            assert np.all(off <= 0)
            assert np.all(np.diag(A) > -off.sum(axis=1))


def pin_kronecker(ns):
    """Sec. 3.2.1: for factorising profiles A = diag|T| (x) (diag v + omega^2 V^r)
    + omega^2 L^S (x) diag(dr), assembled here from small matrices and compared
    entry by entry with the matrix-free operator."""
    for kw in SMALL_CASES:
        o = ns.Oracle(**kw)
        K, M = _vertical_matrix(o)
        for level in range(o.n_levels):
            g = o.grid(o.level_ref(level))
            Ak = np.kron(np.diag(g["area"]), K) + o.omega2 * np.kron(_horizontal_laplacian(g), M)
            A = o.dense_operator(level)
            # 1e-11: the heights are rebuilt here as r - 1, which costs ~1e-14 relative
            assert np.all(np.abs(A - Ak) <= 1e-11 * np.abs(Ak) + 1e-300), np.max(np.abs(A - Ak) / np.abs(Ak))


def pin_horizontal_consistency(ns):
    """Spherical harmonics are eigenfunctions of the Laplace-Beltrami operator
    (eigenvalue -l(l+1)).  With n_r = 1 the horizontal part of A divided by
    omega^2 dr is a two-point-flux Laplacian L^S; its Rayleigh quotient on Y_lm
    relative to the area-weighted mass must converge to l(l+1) at second order."""
    o = ns.Oracle(refinement=5, n_levels=1, n_r=1, omega2=1.0)
    v = o.vertical()
    for l, m in [(1, 0), (2, 1), (3, -2), (4, 3)]:
        errs = []
        for ref in (3, 4, 5):
            oo = ns.Oracle(refinement=ref, n_levels=1, n_r=1, omega2=1.0)
            g = oo.grid(ref)
            u = inputs.real_sph_harm(l, m, g["centre"])
            hor = (oo.apply(u) - g["area"] * v["vol"][0] * u) / (oo.omega2 * v["dr"][0])
            rq = (u @ hor) / (u @ (g["area"] * u))
            errs.append(abs(rq - l * (l + 1)))
        assert errs[-1] < 2e-3 * l * (l + 1), errs
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def pin_vertical_consistency(ns):
    """Vertical part: for u = cos(n pi (r - 1)/H), constant on the sphere, the
    horizontal fluxes vanish and (A u)_k / (|T| v_k) must approach the continuous
    u - omega^2 r^-2 d/dr (r^2 du/dr) at the cell centres, at second order on a
    uniform grid (Appendix A, eq. VerticalDiffusion).  H = 0.5 makes the r^2
    metric terms visible."""
    H, n = 0.5, 2
    errs = []
    for n_r in (16, 32, 64):
        o = ns.Oracle(refinement=0, n_levels=1, n_r=n_r, H=H, omega2=0.01)
        g, v = o.grid(0), o.vertical()
        r = v["r"]
        zc = 0.5 * (r[:-1] + r[1:]) - 1.0
        # cell averages of cos(kz) over each cell, weighted by r^2 (finite-volume unknowns)
        kk = n * math.pi / H
        u_col = np.cos(kk * zc)
        u = np.tile(u_col, 20)
        y = o.apply(u).reshape(20, n_r) / np.outer(g["area"], v["vol"])
        rc = 1.0 + zc
        lu = u_col + o.omega2 * (kk * kk * np.cos(kk * zc) + (2.0 / rc) * kk * np.sin(kk * zc))
        interior = slice(1, n_r - 1)
        errs.append(np.max(np.abs(y[0, interior] - lu[interior])) / np.max(np.abs(lu)))
        assert np.allclose(y, y[0:1, :], rtol=1e-12, atol=1e-12 * np.max(np.abs(y)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


# ----------------------------------------------------------------------------- Thomas
def pin_thomas(ns):
    """Thomas algorithm (Sec. 4.1) against dense LU with partial pivoting on random
    diagonally dominant systems, n = 1..16, and on actual column blocks A_T; the
    same for the column solve that takes A_T as couplings + diagonal excess."""
    rng = np.random.default_rng(5)
    for n in range(1, 17):
        for _ in range(5):
            a = rng.uniform(-1, 1, n)
            c = rng.uniform(-1, 1, n)
            b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 2.0, n)
            d = rng.uniform(-1, 1, n)
            Ad = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
            x = ns.thomas(a, b, c, d)
            xd = np.linalg.solve(Ad, d)
            np.testing.assert_allclose(x, xd, rtol=1e-13, atol=1e-13 * np.max(np.abs(xd)))
            cc = rng.uniform(0.0, 2.0, n)
            cc[0] = 0.0
            m = rng.uniform(0.1, 2.0, n)
            nxt = np.append(cc[1:], 0.0)
            Am = np.diag(m + cc + nxt) - np.diag(cc[1:], -1) - np.diag(cc[1:], 1)
            xm = ns.column_solve(cc, m, d)
            xmd = np.linalg.solve(Am, d)
            np.testing.assert_allclose(xm, xmd, rtol=1e-13, atol=1e-13 * np.max(np.abs(xmd)))
    o = ns.Oracle(refinement=2, n_levels=1, n_r=16, grading=1.05, H=0.05, courant_c=80.0)
    sub, diag, sup = o.column_blocks()
    cpl, exc = o.column_couplings()
    A = o.dense_operator()
    for T in (0, 7, 100, 319):
        d = rng.uniform(-1, 1, o.n_r)
        blk = A[T * o.n_r:(T + 1) * o.n_r, T * o.n_r:(T + 1) * o.n_r]
        xd = np.linalg.solve(blk, d)
        np.testing.assert_allclose(ns.thomas(sub[T], diag[T], sup[T], d), xd, rtol=1e-10,
                                   atol=1e-12 * np.max(np.abs(xd)))
        np.testing.assert_allclose(ns.column_solve(cpl[T], exc[T], d), xd, rtol=1e-10,
                                   atol=1e-12 * np.max(np.abs(xd)))


def _exact_column_solve(c, m, d):
    """Gaussian elimination in exact rational arithmetic on the matrix whose
    entries are the given doubles: diagonal m_k + c_k + c_{k+1}, off-diagonal -c."""
    from fractions import Fraction as Fr

    n = len(d)
    c = [Fr(float(v)) for v in c] + [Fr(0)]
    c[0] = Fr(0)
    diag = [Fr(float(m[k])) + c[k] + c[k + 1] for k in range(n)]
    rhs = [Fr(float(v)) for v in d]
    for k in range(1, n):
        f = c[k] / diag[k - 1]
        diag[k] -= f * c[k]
        rhs[k] += f * rhs[k - 1]
    x = [Fr(0)] * n
    x[n - 1] = rhs[n - 1] / diag[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = (rhs[k] + c[k + 1] * x[k + 1]) / diag[k]
    return np.array([float(v) for v in x])


def pin_column_solve_exact(ns):
    """On thin-shell columns (H = 10/6371, omega^2/h^2 = 80, graded: the vertical
    couplings exceed the diagonal excess by ~1e6, cond(A_T) ~ 1e7) the column
    solve equals the exact rational solution of the same matrix to a few ulp:
    no step of the elimination may subtract nearly equal numbers."""
    rng = np.random.default_rng(12)
    o = ns.Oracle(refinement=3, n_levels=1, n_r=24, grading=1.05, courant_c=80.0)
    cpl, exc = o.column_couplings()
    assert cpl[:, 1:].max() / exc.min() > 1e6       # the regime that defeats textbook pivots
    for T in (0, 77, 1279):
        d = rng.uniform(-1, 1, o.n_r)
        x = ns.column_solve(cpl[T], exc[T], d)
        xe = _exact_column_solve(cpl[T], exc[T], d)
        np.testing.assert_allclose(x, xe, rtol=64 * EPS * o.n_r, atol=0)


# ----------------------------------------------------------------------------- transfers
def pin_transfers(ns):
    """Restriction sums the four children (Sec. 5); prolongation is its transpose
    (P = R^T): <R x, y> = <x, P y>.  Restricting the fine cell areas (times any
    vertical profile) gives the coarse areas, because the children tile the parent."""
    o = ns.Oracle(refinement=3, n_levels=3, n_r=4)
    rng = np.random.default_rng(11)
    for lf in (1, 2):
        gf, gc = o.grid(o.level_ref(lf)), o.grid(o.level_ref(lf - 1))
        x = rng.uniform(-1, 1, o.size(lf))
        y = rng.uniform(-1, 1, o.size(lf - 1))
        Rx = o.restrict(x, lf)
        Py = o.prolong_add(y, np.zeros(o.size(lf)), lf)
        assert abs(Rx @ y - x @ Py) <= 1e-13 * (np.abs(Rx) @ np.abs(y))
        prof = np.arange(1.0, o.n_r + 1.0)
        ra = o.restrict(np.outer(gf["area"], prof).reshape(-1), lf)
        np.testing.assert_allclose(ra, np.outer(gc["area"], prof).reshape(-1), rtol=1e-13)
        base = rng.uniform(-1, 1, o.size(lf))
        np.testing.assert_allclose(o.prolong_add(y, base, lf) - base, Py, rtol=1e-14, atol=1e-15)


# ----------------------------------------------------------------------------- smoother / V-cycle
def dense_vcycle(o, r):
    """Algorithm 1 written with dense matrices (tiny grids): smoother
    u <- u + rho A_T^{-1}(f - A u)_T column by column (eq. BlockJacobi) grouped by
    colour (forward colours before, reverse colours after the coarse-grid
    correction, forward-then-reverse on the coarsest level), or all columns at
    once (block Jacobi); R sums children, P = R^T."""
    n_r = o.n_r
    As = [o.dense_operator(l) for l in range(o.n_levels)]
    cols = [o.grid(o.level_ref(l))["colour"] for l in range(o.n_levels)]

    def relax(l, f, u, cells):
        res = f - As[l] @ u
        u = u.copy()
        for T in cells:
            s = slice(T * n_r, (T + 1) * n_r)
            u[s] += o.relax * np.linalg.solve(As[l][s, s], res[s])
        return u

    def sweep(l, f, u, order):
        if o.smoother == 1:
            return relax(l, f, u, range(cols[l].shape[0]))
        for c in order:
            u = relax(l, f, u, np.where(cols[l] == c)[0])
        return u

    def R(l, x):
        return x.reshape(-1, 4, n_r).sum(axis=1).reshape(-1)

    def P(l, x):
        return np.repeat(x.reshape(-1, 1, n_r), 4, axis=1).reshape(-1)

    def cycle(l, f, u):
        nc = int(cols[l].max()) + 1
        fwd, rev = list(range(nc)), list(range(nc - 1, -1, -1))
        if l == 0:
            for _ in range(o.nu_coarse):
                u = sweep(l, f, u, fwd + list(range(nc - 2, -1, -1)))
            return u
        for _ in range(o.nu_pre):
            u = sweep(l, f, u, fwd)
        rc = R(l, f - As[l] @ u)
        uc = cycle(l - 1, rc, np.zeros(rc.shape[0]))
        u = u + P(l, uc)
        for _ in range(o.nu_post):
            u = sweep(l, f, u, rev)
        return u

    return cycle(o.n_levels - 1, r, np.zeros_like(r))


VCYCLE_CASES = [
    dict(refinement=2, n_levels=3, n_r=4, grading=1.1, courant_c=8.0, nu_pre=1, nu_post=1, nu_coarse=1),
    dict(refinement=2, n_levels=2, n_r=3, courant_c=80.0, nu_pre=2, nu_post=2, nu_coarse=2),
    dict(refinement=2, n_levels=3, n_r=4, courant_c=8.0, nu_pre=2, nu_post=2, nu_coarse=1, smoother=1, relax=0.5),
    dict(refinement=1, n_levels=2, n_r=6, courant_c=30.0, nu_pre=1, nu_post=1, nu_coarse=1, relax=0.8),
]


def pin_vcycle_dense(ns):
    """The matrix-free V-cycle equals Algorithm 1 written with dense matrices."""
    rng = np.random.default_rng(3)
    for kw in VCYCLE_CASES:
        o = ns.Oracle(**kw)
        r = rng.uniform(-1, 1, o.size())
        z = o.vcycle(r)
        zd = dense_vcycle(o, r)
        # the column blocks have condition numbers up to ~1e7 (vertical coupling over
        # mass term ~ omega^2/dr^2), so two exact-in-theory solves agree to ~1e-9
        np.testing.assert_allclose(z, zd, rtol=1e-8, atol=1e-10 * np.max(np.abs(zd)))


def pin_preconditioner_symmetric(ns):
    """Symmetric smoothing (reverse colour order after the correction, symmetric
    coarsest sweep, nu_pre = nu_post) and P = R^T make the V-cycle B symmetric;
    positive definite because it converges.  CG needs both."""
    rng = np.random.default_rng(4)
    for kw in VCYCLE_CASES + [dict(refinement=3, n_levels=4, n_r=16, courant_c=8.0, nu_pre=1, nu_post=1)]:
        o = ns.Oracle(**kw)
        for _ in range(3):
            x = rng.uniform(-1, 1, o.size())
            y = rng.uniform(-1, 1, o.size())
            bx, by = o.vcycle(x), o.vcycle(y)
            # rounding in the column solves is amplified by their condition number (~1e7)
            assert abs(bx @ y - x @ by) <= 1e-10 * np.linalg.norm(bx) * np.linalg.norm(y)
            assert bx @ x > 0


def pin_invariant_subspaces(ns):
    """Sec. 3.2.1 (reduction to two dimensions): with (omega^2 A^r + B^r) e_j =
    lambda_j M^r e_j, A maps e_j (x) V^S into M^r e_j (x) V^S, the block smoother
    keeps e_j (x) V^S invariant, and the V-cycle maps M^r e_j (x) V^S into
    e_j (x) V^S; components along the other e_i stay at rounding level."""
    rng = np.random.default_rng(9)
    for kw in [dict(refinement=2, n_levels=3, n_r=6, grading=1.2, H=0.05, courant_c=8.0, nu_pre=1, nu_post=1),
               dict(refinement=2, n_levels=2, n_r=5, H=0.05, courant_c=20.0, smoother=1, relax=0.5)]:
        o = ns.Oracle(**kw)
        K, M = _vertical_matrix(o)
        lam, E = sla.eigh(K, M)           # E^T M E = I
        nc = o.level_cells(o.n_levels - 1)
        for j in (0, o.n_r // 2, o.n_r - 1):
            w = rng.uniform(-1, 1, nc)
            others = [i for i in range(o.n_r) if i != j]
            u = np.outer(w, E[:, j]).reshape(-1)
            Au = o.apply(u).reshape(nc, o.n_r) @ E           # coefficients along M e_i
            assert np.max(np.abs(Au[:, others])) <= 1e-9 * np.max(np.abs(Au[:, j]))
            Su = o.smooth(np.zeros_like(u), u, 1, 1).reshape(nc, o.n_r) @ (M @ E)
            assert np.max(np.abs(Su[:, others])) <= 1e-9 * np.max(np.abs(Su[:, j]))
            x = np.outer(w, M @ E[:, j]).reshape(-1)
            Bx = o.vcycle(x).reshape(nc, o.n_r) @ (M @ E)
            assert np.max(np.abs(Bx[:, others])) <= 1e-9 * np.max(np.abs(Bx[:, j]))


# ----------------------------------------------------------------------------- solver
def pin_pcg_dense(ns):
    """PCG to rtol 1e-13 reproduces the dense direct solution A^{-1} f.

    On shells of moderate aspect ratio (H = 0.1, cond(A) <= ~1e6) the match is
    required to 1e-10 in the 2-norm.  At the atmospheric aspect ratio
    (H = 10/6371) cond(A) reaches ~1e9 through the barely damped vertically
    constant mode, and two backward-stable direct solvers (Cholesky, LU) already
    disagree by ~1e-9; there PCG must agree with Cholesky in the energy norm to
    within 10x that disagreement (floor 1e-12)."""
    cases = [dict(refinement=0, n_levels=1, n_r=8, grading=1.1, H=0.1, courant_c=8.0),
             dict(refinement=1, n_levels=2, n_r=8, H=0.1, courant_c=80.0, nu_pre=1, nu_post=1),
             dict(refinement=2, n_levels=3, n_r=8, grading=1.05, H=0.1, courant_c=8.0),
             dict(refinement=2, n_levels=2, n_r=4, H=0.1, courant_c=20.0, smoother=1, relax=0.5)]
    for kw in cases:
        o = ns.Oracle(**kw)
        f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, o.size())
        res = o.pcg(f, rtol=1e-13, max_iter=300)
        assert res["status"] == 0
        A = o.dense_operator()
        ud = sla.cho_solve(sla.cho_factor(A), f)
        assert np.linalg.norm(res["u"] - ud) <= 1e-10 * np.linalg.norm(ud)
    for kw in [dict(refinement=1, n_levels=2, n_r=8, courant_c=80.0, nu_pre=1, nu_post=1),
               dict(refinement=2, n_levels=3, n_r=8, grading=1.05, courant_c=8.0)]:
        o = ns.Oracle(**kw)
        f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL, o.size())
        res = o.pcg(f, rtol=1e-13, max_iter=300)
        assert res["status"] == 0
        A = o.dense_operator()
        ud = sla.cho_solve(sla.cho_factor(A), f)
        ul = sla.lu_solve(sla.lu_factor(A), f)

        def anorm(e):
            return math.sqrt(max(e @ A @ e, 0.0))

        floor = max(10.0 * anorm(ul - ud), 1e-12 * anorm(ud))
        assert anorm(res["u"] - ud) <= floor, (anorm(res["u"] - ud) / anorm(ud), floor / anorm(ud))


def pin_bf16_rounding(ns):
    """The coefficients of the mixed-precision V-cycle are rounded to bfloat16:
    the nearest number with an 8-bit significand (binary32 exponent range),
    ties to the even significand.  Checked against that definition by brute
    force: the two bfloat16 neighbours of x are built from its exponent, and the
    result must be the nearer one (the even one on a tie)."""
    rng = np.random.default_rng(21)
    xs = list(rng.uniform(-1, 1, 400) * 10.0 ** rng.integers(-30, 30, 400))
    xs += [1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, -(1.0 + 2.0 ** -9), 255.5 / 128, 1.0, 0.0, 3.0e-12, 1.0 / 3.0]
    for x in xs:
        y = ns.bf16(x)
        if x == 0.0:
            assert y == 0.0
            continue
        e = math.floor(math.log2(abs(x)))
        if 2.0 ** e > abs(x):   # guard log2 rounding at powers of two
            e -= 1
        ulp = 2.0 ** (e - 7)
        lo = math.floor(abs(x) / ulp) * ulp
        hi = lo + ulp
        dlo, dhi = abs(x) - lo, hi - abs(x)
        if dlo < dhi:
            want = lo
        elif dhi < dlo:
            want = hi
        else:
            want = lo if round(lo / ulp) % 2 == 0 else hi
        assert y == math.copysign(want, x), (x, y, want)


def pin_flexible_cg(ns):
    """Flexible CG (Polak-Ribiere coefficient) takes the iterates of plain PCG
    when the preconditioner is symmetric, since then <r_{k+1}, z_k> = 0; with the
    mixed-precision V-cycle (BF16 coefficients) it still reaches the dense direct
    solution, because the outer residual uses the exact operator."""
    kw = dict(refinement=2, n_levels=3, n_r=8, grading=1.05, H=0.1, courant_c=8.0)
    o = ns.Oracle(**kw)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 2, o.size())
    a = o.pcg(f, rtol=1e-10, max_iter=200)
    b = o.pcg(f, rtol=1e-10, max_iter=200, flexible=True)
    assert a["status"] == 0 and b["status"] == 0 and a["iters"] == b["iters"]
    assert np.linalg.norm(a["u"] - b["u"]) <= 1e-12 * np.linalg.norm(a["u"])
    o.set_vcycle_bf16(True)
    c = o.pcg(f, rtol=1e-13, max_iter=300, flexible=True)
    assert c["status"] == 0
    A = o.dense_operator()
    ud = sla.cho_solve(sla.cho_factor(A), f)
    assert np.linalg.norm(c["u"] - ud) <= 1e-10 * np.linalg.norm(ud)


def pin_bf16_vcycle(ns):
    """The V-cycle with BF16-rounded coefficients is the V-cycle of a nearby
    operator that is still symmetric (each edge coupling is rounded once and used
    by both of its cells): <B x, y> = <x, B y> to rounding, <B x, x> > 0, and
    B x differs from the plain V-cycle by a few times the BF16 rounding 2^-9."""
    rng = np.random.default_rng(22)
    o = ns.Oracle(refinement=3, n_levels=3, n_r=12, grading=1.05, courant_c=80.0)
    x, y = rng.uniform(-1, 1, o.size()), rng.uniform(-1, 1, o.size())
    bx_plain = o.vcycle(x)
    o.set_vcycle_bf16(True)
    bx, by = o.vcycle(x), o.vcycle(y)
    assert abs(bx @ y - x @ by) <= 1e-12 * np.linalg.norm(bx) * np.linalg.norm(y)
    assert bx @ x > 0
    e = bx - bx_plain
    assert math.sqrt(e @ o.apply(e)) <= 16 * 2.0 ** -9 * math.sqrt(bx_plain @ o.apply(bx_plain))
    assert math.sqrt(e @ o.apply(e)) > 0


def pin_bicgstab(ns):
    """BiCGStab (van der Vorst 1992), right-preconditioned by the V-cycle: to rtol
    1e-13 it reproduces the dense direct solution on moderate-aspect shells, and
    with an exact preconditioner (a single level relaxed by 64 block-SOR sweeps,
    B = A^{-1} to 1e-13) it converges in one iteration."""
    for kw in [dict(refinement=1, n_levels=2, n_r=8, H=0.1, courant_c=80.0, nu_pre=1, nu_post=1),
               dict(refinement=2, n_levels=3, n_r=8, grading=1.05, H=0.1, courant_c=8.0)]:
        o = ns.Oracle(**kw)
        f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 3, o.size())
        res = o.bicgstab(f, rtol=1e-13, max_iter=100)
        assert res["status"] == 0
        ud = sla.cho_solve(sla.cho_factor(o.dense_operator()), f)
        assert np.linalg.norm(res["u"] - ud) <= 1e-10 * np.linalg.norm(ud)
    for kw in [dict(refinement=0, n_levels=1, n_r=4, H=0.1, courant_c=0.5, nu_coarse=64),
               dict(refinement=1, n_levels=1, n_r=6, H=0.1, courant_c=1.0, nu_coarse=64)]:
        o = ns.Oracle(**kw)
        f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 4, o.size())
        res = o.bicgstab(f, rtol=1e-12, max_iter=10)
        assert res["status"] == 0 and res["iters"] == 1, res["hist"]


def _profiles(o, seed):
    """Seeded positive factorised profiles for an oracle instance (all in [0.5, 1.5])."""
    n = o.level_cells(o.n_levels - 1)
    u = lambda k, m: 1.0 + 0.5 * inputs.uniform_pm1(seed + k, m)
    return dict(beta_r=u(1, o.n_r), alphaS_r=u(2, o.n_r), alphar_r=u(3, o.n_r + 1),
                beta_s=u(4, n), alphar_s=u(5, n), alphaS_s=u(6, n))


def pin_profiles(ns):
    """Factorised profiles (Sec. 2, eq. profiles; the TPMG^otimes form):
    unit profiles leave the operator bit for bit; random positive profiles keep it
    symmetric positive definite; a profile of beta alone adds exactly
    (beta - 1) |T| v_k to the diagonal, on the finest level with the given factors
    and on the coarsest with their area-weighted means over the children; and an
    edge couples with the mean of its two cells' alpha_S factors."""
    kw = dict(refinement=2, n_levels=3, n_r=5, grading=1.1, H=0.1, courant_c=8.0)
    o = ns.Oracle(**kw)
    n_f = o.level_cells(2)
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 7, o.size())
    y0 = o.apply(x)
    o.set_profiles(**{k: np.ones_like(v) for k, v in _profiles(o, 11).items()})
    assert np.array_equal(o.apply(x), y0)
    o.set_profiles(**_profiles(o, 12))
    A = o.dense_operator()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0.0
    # beta alone: diagonal shift on the finest and the coarsest level
    bs = 1.0 + 0.5 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 8, n_f)
    br = 1.0 + 0.5 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 9, o.n_r)
    o.set_profiles()
    vol = o.vertical()["vol"]
    for level in (2, 0):
        n = o.level_cells(level)
        xl = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 10 + level, n * o.n_r)
        plain = o.apply(xl, level)
        o.set_profiles(beta_r=br, beta_s=bs)
        prof = o.apply(xl, level)
        o.set_profiles()
        area = o.grid(o.level_ref(level))["area"]
        if level == 2:
            bl = bs
        else:   # area-weighted means over the children, twice
            a1, a2 = o.grid(o.level_ref(1))["area"], o.grid(o.level_ref(2))["area"]
            b1 = (a2 * bs).reshape(-1, 4).sum(1) / a2.reshape(-1, 4).sum(1)
            bl = (a1 * b1).reshape(-1, 4).sum(1) / a1.reshape(-1, 4).sum(1)
        expect = plain + (np.outer(area * bl, vol * br) - np.outer(area, vol)).reshape(-1) * xl
        assert np.max(np.abs(prof - expect)) <= 1e-12 * np.max(np.abs(prof)), level
    # edge coupling: the mean of the two cells' alpha_S^S
    aSs = 1.0 + 0.5 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 13, n_f)
    grid = o.grid(o.level_ref(2))
    A0 = o.dense_operator()
    o.set_profiles(alphaS_s=aSs)
    A1 = o.dense_operator()
    o.set_profiles()
    T, e, k = 7, 1, 2
    Tn = grid["nbr"][T, e]
    i, j = T * o.n_r + k, Tn * o.n_r + k
    assert abs(A1[i, j] - A0[i, j] * 0.5 * (aSs[T] + aSs[Tn])) <= 1e-13 * abs(A0[i, j])


def pin_outer_operator(ns):
    """The problem's operator with general (per-unknown) profiles: for profiles that
    happen to factorise it equals the V-cycle's operator with the factors (two
    independent statements of the same coefficients); it is symmetric positive
    definite; and PCG with the factorised V-cycle as preconditioner reaches its dense
    solution (Sec. 3.2.2: TPMG preconditioning a non-factorising operator)."""
    kw = dict(refinement=2, n_levels=2, n_r=6, grading=1.1, H=0.1, courant_c=8.0)
    o = ns.Oracle(**kw)
    n = o.level_cells(1)
    prof = _profiles(o, 21)
    o.set_profiles(**prof)
    o.set_outer_profiles(beta=np.outer(prof["beta_s"], prof["beta_r"]),
                         alphar=np.outer(prof["alphar_s"], prof["alphar_r"]),
                         alphaS=np.outer(prof["alphaS_s"], prof["alphaS_r"]))
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 21, o.size())
    y_fac, y_out = o.apply(x), o.apply_outer(x)
    assert np.max(np.abs(y_out - y_fac)) <= 1e-13 * np.max(np.abs(y_fac))
    # the V-cycle on the general profiles (TPMG^full; coarse levels averaged per vertical
    # index) equals the factorised one when the profiles are an outer product
    z_fac = o.vcycle(x)
    o.set_vcycle_full(True)
    z_full = o.vcycle(x)
    o.set_vcycle_full(False)
    assert np.max(np.abs(z_full - z_fac)) <= 1e-12 * np.max(np.abs(z_fac))
    # a non-factorising operator: perturb every profile value independently
    pert = lambda k, shape: 1.0 + 0.3 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + k, int(np.prod(shape))).reshape(shape)
    o.set_outer_profiles(beta=np.outer(prof["beta_s"], prof["beta_r"]) * pert(31, (n, o.n_r)),
                         alphar=np.outer(prof["alphar_s"], prof["alphar_r"]) * pert(32, (n, o.n_r + 1)),
                         alphaS=np.outer(prof["alphaS_s"], prof["alphaS_r"]) * pert(33, (n, o.n_r)))
    A = np.stack([o.apply_outer(e) for e in np.eye(o.size())], axis=1)
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0.0
    assert np.abs(A - o.dense_operator()).max() > 1e-3 * np.abs(A).max()   # it is not the V-cycle's operator
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 22, o.size())
    res = o.pcg(f, rtol=1e-13, max_iter=300)
    assert res["status"] == 0
    ud = np.linalg.solve(A, f)
    assert np.linalg.norm(res["u"] - ud) <= 1e-9 * np.linalg.norm(ud)
    # with the V-cycle on the same general profiles (TPMG^full) too
    o.set_vcycle_full(True)
    res2 = o.pcg(f, rtol=1e-13, max_iter=300)
    o.set_vcycle_full(False)
    assert res2["status"] == 0 and np.linalg.norm(res2["u"] - ud) <= 1e-9 * np.linalg.norm(ud)


def pin_partial_profiles(ns):
    """Partial factorisation TPMG^partial (Sec. 5.3): the V-cycle's operators take alpha_r
    from the general profiles and beta, alpha_S from the factorised ones.  On the finest
    level every vertical coupling is the factorised one times alpha_r / (alpha_r^S
    alpha_r^r) and nothing else changes; where only alpha_r departs from a factorisation
    the partial V-cycle is the full one (TPMG^full), and where only beta and alpha_S
    depart it is the factorised one (TPMG^fac), on every level and for the whole cycle."""
    kw = dict(refinement=2, n_levels=2, n_r=5, grading=1.1, H=0.1, courant_c=8.0)
    o = ns.Oracle(**kw)
    n = o.level_cells(1)
    prof = _profiles(o, 41)
    o.set_profiles(**prof)
    pert = lambda k, shape: 1.0 + 0.3 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + k, int(np.prod(shape))).reshape(shape)
    fac = dict(beta=np.outer(prof["beta_s"], prof["beta_r"]), alphar=np.outer(prof["alphar_s"], prof["alphar_r"]),
               alphaS=np.outer(prof["alphaS_s"], prof["alphaS_r"]))
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 42, o.size())

    def modes(**general):
        o.set_outer_profiles(**general)
        out = {}
        for name, sw in (("fac", None), ("full", o.set_vcycle_full), ("partial", o.set_vcycle_partial)):
            if sw:
                sw(True)
            out[name] = ([o.dense_operator(l) for l in range(o.n_levels)], o.vcycle(x))
            if sw:
                sw(False)
        return out

    def same(a, b, tol):
        return all(np.abs(p - q).max() <= tol * np.abs(q).max() for p, q in zip(a[0], b[0])) and \
            np.abs(a[1] - b[1]).max() <= tol * np.abs(b[1]).max()

    # alpha_r alone departs: partial = full, not fac; the finest level's vertical
    # couplings carry exactly the ratio of the profiles
    pr = pert(43, (n, o.n_r + 1))
    m = modes(beta=fac["beta"], alphar=fac["alphar"] * pr, alphaS=fac["alphaS"])
    assert same(m["partial"], m["full"], 1e-12)
    assert not same(m["partial"], m["fac"], 1e-3)
    Ap, Af = m["partial"][0][-1], m["fac"][0][-1]
    for T, k in ((0, 1), (17, 3), (n - 1, 4)):
        i = T * o.n_r + k
        assert abs(Ap[i, i - 1] - Af[i, i - 1] * pr[T, k]) <= 1e-13 * abs(Af[i, i - 1])
        assert abs(Ap[i, i - 1] - Ap[i - 1, i]) <= 1e-13 * abs(Ap[i, i - 1])   # still symmetric
    off_vertical = np.abs(np.subtract.outer(np.arange(o.size()) // o.n_r, np.arange(o.size()) // o.n_r)) > 0
    assert np.abs((Ap - Af)[off_vertical]).max() <= 1e-13 * np.abs(Af).max()
    # beta and alpha_S depart: partial = fac, not full
    m = modes(beta=fac["beta"] * pert(44, (n, o.n_r)), alphar=fac["alphar"],
              alphaS=fac["alphaS"] * pert(45, (n, o.n_r)))
    assert same(m["partial"], m["fac"], 1e-12)
    assert not same(m["partial"], m["full"], 1e-3)
    o.set_outer_profiles()


def pin_advection(ns):
    """Vertical advection -omega^2 xi_r d_r u (Sec. 2, eq. HelmholtzVector; Appendix A;
    reading C24: each row averages the one-sided differences through its two faces,
    weighted by r_face^2 and the row's own thickness).
    * xi = 0 changes nothing, bit for bit, and a constant field has no advection.
    * For u = r at the cell midpoints and constant xi, the discrete term of row k is
      the trapezoid rule for the cell integral of r^2:
      -omega^2 |T| xi (dr_k / 2) (r_k^2 + r_{k+1}^2) = -omega^2 |T| xi (v_k + dr_k^3 / 6)
      on interior rows; the bottom row keeps the upper face's half, the top row the
      lower face's (a closed form on a graded grid).
    * The non-symmetric column solve equals the dense solve of the assembled block.
    * A general xi that factorises gives the factorised operator; BiCGStab reaches the
      dense solution of the non-symmetric operator."""
    kw = dict(refinement=2, n_levels=2, n_r=6, grading=1.2, H=0.1, courant_c=8.0)
    o = ns.Oracle(**kw)
    n, N, n_r = o.level_cells(1), o.size(), o.n_r
    vert = o.vertical()
    r, dr, vol = vert["r"], vert["dr"], vert["vol"]
    area = o.grid(o.refinement)["area"]
    x = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 90, N)
    y0, ones = o.apply(x), np.ones(N)
    o.set_profiles(xi_r=np.zeros(n_r + 1), xi_s=np.ones(n))
    assert np.array_equal(o.apply(x), y0)
    c = 20.0
    o.set_profiles(xi_r=np.full(n_r + 1, c))
    assert np.array_equal(o.apply(ones), (o.set_profiles(), o.apply(ones))[1])
    o.set_profiles(xi_r=np.full(n_r + 1, c))
    u = np.tile(0.5 * (r[:-1] + r[1:]), n)
    with_xi = o.apply(u)
    o.set_profiles()
    D = (with_xi - o.apply(u)).reshape(n, n_r)
    w = o.omega2 * area[:, None] * c
    expect = -w * (vol + dr ** 3 / 6.0)[None, :]
    expect[:, 0] = -w[:, 0] * dr[0] * r[1] ** 2 / 2.0
    expect[:, -1] = -w[:, 0] * dr[-1] * r[-2] ** 2 / 2.0
    scale = np.abs(o.apply(u)).reshape(n, n_r)
    assert np.all(np.abs(D - expect) <= 1e-12 * scale), np.max(np.abs(D - expect) / scale)
    # the column blocks and their solve
    o.set_profiles(xi_r=1.0 + 0.5 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 91, n_r + 1),
                   xi_s=c * (1.0 + 0.5 * inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 92, n)))
    cd, cu, m = o.column_couplings2()
    sub, diag, sup = o.column_blocks()
    assert cd[:, 1:].min() > 0.0 and cu[:, :-1].min() > 0.0
    assert np.abs(cu[:, :-1] - cd[:, 1:]).max() > 1e-6 * cd[:, 1:].max()   # not symmetric
    for T in (0, 11, n - 1):
        Ad = np.diag(m[T] + cd[T] + cu[T]) - np.diag(cd[T, 1:], -1) - np.diag(cu[T, :-1], 1)
        Ab = np.diag(diag[T]) + np.diag(sub[T, 1:], -1) + np.diag(sup[T, :-1], 1)
        assert np.abs(Ad - Ab).max() <= 1e-13 * np.abs(Ab).max()
        d = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 93 + T, n_r)
        xs = ns.column_solve2(cd[T], cu[T], m[T], d)
        xd = np.linalg.solve(Ad, d)
        assert np.linalg.norm(xs - xd) <= 1e-12 * np.linalg.norm(xd)
    # general xi as an outer product equals the factorised one; BiCGStab on the operator
    prof = o._profiles
    xi_gen = np.outer(prof[7], prof[6])
    o.set_outer_profiles(beta=np.ones((n, n_r)), alphar=np.ones((n, n_r + 1)), alphaS=np.ones((n, n_r)), xi=xi_gen)
    assert np.max(np.abs(o.apply_outer(x) - o.apply(x))) <= 1e-13 * np.max(np.abs(o.apply(x)))
    o.set_outer_profiles()
    A = o.dense_operator()
    assert np.abs(A - A.T).max() > 1e-8 * np.abs(A).max()
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 94, N)
    res = o.bicgstab(f, rtol=1e-13, max_iter=200)
    assert res["status"] == 0
    ud = np.linalg.solve(A, f)
    assert np.linalg.norm(res["u"] - ud) <= 1e-9 * np.linalg.norm(ud)
    o.set_profiles()


def pin_linear_prolongation(ns):
    """Linear prolongation (Sec. 5: the solution is prolongated by linear interpolation;
    reading C25: a least-squares gradient in the tangent plane from the 3 coarse
    neighbours).  Constants are reproduced exactly; interpolating a smooth field from
    the coarse centres to the fine ones errs by O(h^2) (the error falls about 4x per
    refinement) where the piecewise-constant P = R^T errs by O(h) (about 2x); the
    V-cycle with it converges, and BiCGStab with it reaches the dense solution."""
    o = ns.Oracle(refinement=6, n_levels=4, n_r=1, H=0.01, courant_c=8.0)
    n1 = o.level_cells(1)
    o.set_prolongation(True)
    c = 0.375
    out = o.prolong_add(np.full(n1, c), np.zeros(4 * n1), 2)
    assert np.all(out == c)
    a, b = np.array([0.3, -0.7, 0.5]), np.array([0.6, 0.2, -0.4])
    F = lambda x: x @ a + 2.0 * (x @ b) ** 2 + np.sin(3.0 * x[:, 2])
    errs = {}
    for linear in (True, False):
        o.set_prolongation(linear)
        e = []
        for lf in (1, 2, 3):
            xc = o.grid(o.level_ref(lf - 1))["centre"]
            xf = o.grid(o.level_ref(lf))["centre"]
            e.append(np.max(np.abs(o.prolong_add(F(xc), np.zeros(len(xf)), lf) - F(xf))))
        errs[linear] = e
    lin, con = errs[True], errs[False]
    assert all(lin[i] / lin[i + 1] > 3.3 for i in range(2)), lin
    assert all(con[i] / con[i + 1] < 2.5 for i in range(2)), con
    assert lin[-1] < 0.2 * con[-1]
    # in a V-cycle (sum restriction, linear prolongation): Richardson converges, and
    # BiCGStab reaches the dense solution
    o = ns.Oracle(refinement=3, n_levels=3, n_r=8, grading=1.1, H=0.05, courant_c=20.0)
    o.set_prolongation(True)
    rho = convergence_factor(o)
    assert rho < 0.5, rho
    o = ns.Oracle(refinement=2, n_levels=2, n_r=6, grading=1.1, H=0.05, courant_c=20.0)
    o.set_prolongation(True)
    f = inputs.uniform_pm1(inputs.SEED_UNIFORM_SMALL + 95, o.size())
    res = o.bicgstab(f, rtol=1e-12, max_iter=200)
    assert res["status"] == 0
    A = o.dense_operator()
    ud = np.linalg.solve(A, f)
    assert np.linalg.norm(res["u"] - ud) <= 1e-9 * np.linalg.norm(ud)


def pin_manufactured(ns):
    """Manufactured solution: f = A u*, solve to rtol 1e-12, recover u* in the
    energy norm to 1e-9 (a residual drop of 1e-12 bounds the error by cond-weighted 1e-12)."""
    o = ns.Oracle(refinement=3, n_levels=3, n_r=16, grading=1.05, courant_c=80.0)
    g, v = o.grid(o.refinement), o.vertical()
    ustar = inputs.manufactured_solution(g["centre"], v["r"], inputs.SEED_MANUFACTURED)
    f = o.apply(ustar)
    res = o.pcg(f, rtol=1e-12, max_iter=200)
    assert res["status"] == 0
    e = res["u"] - ustar
    assert math.sqrt(e @ o.apply(e)) <= 1e-9 * math.sqrt(ustar @ f)


def convergence_factor(o, n_iter: int = 8, seed: int = 77) -> float:
    """Asymptotic residual reduction per Richardson step u <- u + B(f - A u), f = 0."""
    u0 = inputs.uniform_pm1(seed, o.size())
    _, hist = o.richardson(np.zeros(o.size()), u0, n_iter)
    return float((hist[-1] / hist[-4]) ** (1.0 / 3.0))


def pin_robust_convergence(ns):
    """Theorem (Sec. 3.2.1): the TPMG V-cycle factor is bounded away from 1
    independently of h and of the vertical aspect ratio.  Measured over grids and
    anisotropies: every factor < 0.5 and their spread (max/min) <= 2."""
    rhos = []
    for ref in (3, 4):
        for n_r in (16, 64):
            for gr in (1.0, 1.05):
                for C in (8.0, 80.0):
                    o = ns.Oracle(refinement=ref, n_levels=4, n_r=n_r, grading=gr, courant_c=C,
                                  nu_pre=2, nu_post=2, nu_coarse=1)
                    rhos.append(convergence_factor(o))
    assert max(rhos) < 0.5, rhos
    assert max(rhos) / min(rhos) <= 2.0, rhos


ALL_PINS = [
    pin_mesh_counts, pin_mesh_areas, pin_level0_closed_forms, pin_mesh_topology, pin_vertical,
    pin_constants_in_kernel, pin_symmetric_spd, pin_kronecker, pin_horizontal_consistency,
    pin_vertical_consistency, pin_thomas, pin_column_solve_exact, pin_transfers, pin_vcycle_dense, pin_preconditioner_symmetric,
    pin_invariant_subspaces, pin_pcg_dense, pin_bf16_rounding, pin_flexible_cg, pin_bf16_vcycle,
    pin_manufactured, pin_robust_convergence, pin_bicgstab, pin_profiles, pin_outer_operator,
    pin_partial_profiles, pin_advection, pin_linear_prolongation,
]
