"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds none of the solver's arithmetic: it only turns a seed into
numbers.  Both sides of every parity check receive the identical bytes it
produces.  Numpy only; no torch, no CUDA.

* ``splitmix64`` -- Steele, Lea & Flood's SplitMix64 generator (counter-based:
  output i is mix(seed + (i+1) * 0x9E3779B97F4A7C15)).
* ``uniform_pm1`` -- 53-bit doubles in [-1, 1).
* ``real_sph_harm`` -- orthonormal real spherical harmonics evaluated at points
  of the unit sphere, from the three-term recurrence of the associated Legendre
  functions.
* ``manufactured_solution`` -- a sum of low-order spherical harmonics times
  vertical cosines (the cosines satisfy the zero-flux vertical conditions).
* ``smooth_field`` -- a random band-limited field on the shell.
* ``balanced_flow_profiles`` -- the factorised profile shapes of the balanced-flow
  atmosphere with two mid-latitude jets (Sec. 5), at the buoyancy frequency where they
  factorise exactly.
* ``balanced_flow`` -- the same atmosphere at any buoyancy frequency N >= N*: its exact,
  non-factorising profiles per unknown and their factorised approximation.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_UNIFORM_SMALL = 2981001   # 1280 cells x 16 uniform levels, RHS uniform[-1, 1]
SEED_MANUFACTURED = 2981002    # 81920 cells x 64 graded levels, manufactured solution
SEED_MIXED = 2981003           # 327680 cells x 128 graded levels, RHS uniform[-1, 1]
SEED_BATCH = 2981004           # batch of uneven problems
SEED_LEARNED = 2981005         # learned coarse solve / warm start data
SEED_SWEEP = 2981010           # n_r sweep


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """53-bit doubles in [0, 1)."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """53-bit doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, n, offset) - 1.0


def randint(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive)."""
    u = uniform01(seed, n, offset)
    return lo + np.minimum(np.floor(u * (hi - lo + 1)), hi - lo).astype(np.int64)


def real_sph_harm(l: int, m: int, xyz: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonic Y_lm at unit vectors ``xyz`` [n, 3].

    m > 0 uses cos(m phi), m < 0 uses sin(|m| phi); no Condon-Shortley phase.
    """
    if l < 0 or abs(m) > l:
        raise ValueError("need 0 <= |m| <= l")
    xyz = np.asarray(xyz, dtype=np.float64)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    ct = np.clip(z, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    phi = np.arctan2(y, x)
    am = abs(m)
    # P_am^am = (2am-1)!! st^am, then the upward recurrence in l
    pmm = np.ones_like(ct)
    for i in range(1, am + 1):
        pmm = pmm * (2 * i - 1) * st
    if l == am:
        plm = pmm
    else:
        pm1 = ct * (2 * am + 1) * pmm
        if l == am + 1:
            plm = pm1
        else:
            p_prev, p_cur = pmm, pm1
            for ll in range(am + 2, l + 1):
                p_next = ((2 * ll - 1) * ct * p_cur - (ll + am - 1) * p_prev) / (ll - am)
                p_prev, p_cur = p_cur, p_next
            plm = p_cur
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    if m == 0:
        return norm * plm
    if m > 0:
        return math.sqrt(2.0) * norm * plm * np.cos(am * phi)
    return math.sqrt(2.0) * norm * plm * np.sin(am * phi)


def manufactured_params(seed: int, n_terms: int = 8, l_max: int = 4, n_max: int = 3) -> list[tuple]:
    """(a_i, l_i, m_i, n_i) for the manufactured solution, all drawn from ``seed``."""
    u = uniform01(seed, 4 * n_terms)
    out = []
    for i in range(n_terms):
        l = int(min(math.floor(u[4 * i] * (l_max + 1)), l_max))
        m = int(min(math.floor(u[4 * i + 1] * (2 * l + 1)), 2 * l)) - l
        n = int(min(math.floor(u[4 * i + 2] * (n_max + 1)), n_max))
        a = 2.0 * float(u[4 * i + 3]) - 1.0
        out.append((a, l, m, n))
    return out


def manufactured_solution(centres: np.ndarray, r_faces: np.ndarray, seed: int,
                          n_terms: int = 8, l_max: int = 4, n_max: int = 3) -> np.ndarray:
    """u*[T, k] = sum_i a_i Y_{l_i m_i}(c_T) cos(n_i pi (r_{k+1/2} - 1) / H), flattened [T][k].

    ``centres`` [n_cells, 3] unit vectors, ``r_faces`` [n_r + 1] radii of the
    level faces, ``H = r_faces[-1] - r_faces[0]``.
    """
    centres = np.asarray(centres, dtype=np.float64)
    r_faces = np.asarray(r_faces, dtype=np.float64)
    H = r_faces[-1] - r_faces[0]
    zmid = 0.5 * (r_faces[:-1] + r_faces[1:]) - r_faces[0]
    u = np.zeros((centres.shape[0], zmid.shape[0]))
    for a, l, m, n in manufactured_params(seed, n_terms, l_max, n_max):
        u += a * np.outer(real_sph_harm(l, m, centres), np.cos(n * math.pi * zmid / H))
    return u.reshape(-1)


def smooth_field(centres: np.ndarray, r_faces: np.ndarray, seed: int, l_max: int = 16,
                 n_max: int = 3, decay: float = 1.0) -> np.ndarray:
    """Random band-limited field: sum over l <= l_max, |m| <= l, n <= n_max of
    c_{lmn} Y_lm(c_T) cos(n pi z / H), c uniform[-1, 1] / (1 + l)^decay."""
    centres = np.asarray(centres, dtype=np.float64)
    r_faces = np.asarray(r_faces, dtype=np.float64)
    H = r_faces[-1] - r_faces[0]
    zmid = 0.5 * (r_faces[:-1] + r_faces[1:]) - r_faces[0]
    n_coef = (l_max + 1) ** 2 * (n_max + 1)
    c = uniform_pm1(seed, n_coef)
    out = np.zeros((centres.shape[0], zmid.shape[0]))
    idx = 0
    for l in range(l_max + 1):
        for m in range(-l, l + 1):
            y = real_sph_harm(l, m, centres) / (1.0 + l) ** decay
            for n in range(n_max + 1):
                out += c[idx] * np.outer(y, np.cos(n * math.pi * zmid / H))
                idx += 1
    return out.reshape(-1)


def jet_function(phi: np.ndarray, u0: float = 100.0, phi_m: float = math.pi / 4, sigma: float = 0.1,
                 radius: float = 6.371e6, omega: float = 2.0 * math.pi / (24 * 3600), n_quad: int = 20001) -> np.ndarray:
    """F(phi) with dF/dphi = 2 R Omega u(phi) sin(phi) + u(phi)^2 tan(phi), F(0) = 0, for the
    two-jet zonal wind u(phi) = u0 cos(phi) / cos(phi_M) exp(-(cos(phi) - cos(phi_M))^2 / (2 sigma^2))
    (m^2 s^-2; trapezoidal quadrature on a fine latitude grid, then interpolation)."""
    grid = np.linspace(0.0, math.pi / 2 * (1 - 1e-9), n_quad)
    u = u0 * np.cos(grid) / math.cos(phi_m) * np.exp(-(np.cos(grid) - math.cos(phi_m)) ** 2 / (2 * sigma ** 2))
    dF = 2 * radius * omega * u * np.sin(grid) + u * u * np.tan(grid)
    F = np.concatenate([[0.0], np.cumsum(0.5 * (dF[1:] + dF[:-1]) * np.diff(grid))])
    return np.interp(np.abs(np.asarray(phi, dtype=np.float64)), grid, F)   # F is even in phi


def balanced_flow_profiles(centres: np.ndarray, r_faces: np.ndarray, cp: float = 1005.0, rd: float = 287.0,
                           t0: float = 273.0, g: float = 9.81, radius: float = 6.371e6) -> dict:
    """Factorised profiles (horizontal x vertical) of the balanced atmosphere at the buoyancy
    frequency N = N* = g / sqrt(cp T0), where the Exner pressure pi = e_H e_V factorises:
    e_H = exp(-N^2 F(phi) / g^2), e_V = exp(-N^2 R (r - 1) / g) (r in units of the earth's
    radius).  Then rho theta and rho / pi are both proportional to (e_H e_V)^gamma with
    gamma = cv / rd, so alpha_S = rho theta, alpha_r = r^2 Lambda rho theta (Lambda = 1) and
    beta = gamma rho / pi factorise into (e_H)^gamma times a vertical factor.  Each factor is
    normalised to 1 at the equator and the surface.  Returns the tpmg_profiles fields."""
    centres = np.asarray(centres, dtype=np.float64)
    r_faces = np.asarray(r_faces, dtype=np.float64)
    n_star = g / math.sqrt(cp * t0)
    gamma = (cp - rd) / rd
    phi = np.arcsin(np.clip(centres[:, 2], -1.0, 1.0))
    e_h = np.exp(-n_star ** 2 * jet_function(phi) / g ** 2)
    rc = 0.5 * (r_faces[:-1] + r_faces[1:])
    e_v = lambda r: np.exp(-n_star ** 2 * radius * (r - 1.0) / g)
    h = e_h ** gamma
    vc = e_v(rc) ** gamma / e_v(rc[0]) ** gamma
    vf = r_faces ** 2 * e_v(r_faces) ** gamma / (r_faces[0] ** 2 * e_v(r_faces[0]) ** gamma)
    return dict(beta_r=vc, alphaS_r=vc, alphar_r=vf, beta_s=h, alphar_s=h, alphaS_s=h)


def balanced_flow(centres: np.ndarray, r_faces: np.ndarray, n_freq: float, cp: float = 1005.0, rd: float = 287.0,
                  t0: float = 273.0, g: float = 9.81, radius: float = 6.371e6,
                  advection: bool = False) -> tuple[dict, dict, float]:
    """The balanced atmosphere at buoyancy frequency N (Sec. 5, after Davies 2005): with
    eps = (N / N*)^2 - 1, e_H = exp(-N^2 F(phi) / g^2), e_V = exp(-N^2 R (r - 1) / g),
    the Exner pressure pi = (eps + e_H e_V) / (1 + eps), theta = T0 / (e_H e_V),
    rho = p0 / (Rd T0) pi^gamma e_H e_V (gamma = cv / Rd), and the profiles
    alpha_S = rho theta, alpha_r = r^2 Lambda rho theta (Lambda = 1), beta = gamma rho / pi.
    Returns (exact profiles per unknown: beta, alphaS [n, n_r] at the cell centres,
    alphar [n, n_r + 1] at the faces; the factorised approximation from
    pi^x = (eps + e_V) / (1 + eps) * e_H as tpmg_profiles fields; eps).  Every profile
    is normalised by its value at the equator and the surface, where pi = pi^x = 1.
    advection: also the vertical advection xi_r = Lambda rho d_r theta of eq. profiles.
    theta = T0 / (e_H e_V) gives d_r theta = theta N^2 R / g (r in earth radii), so
    xi_r = rho theta N^2 R / g: alpha_S's shape (normalised alike) times N^2 R / g, at the
    faces ("xi" of the exact profiles; "xi_r", "xi_s" of the factorised ones, from
    rho^x theta = (pi^x)^gamma)."""
    centres = np.asarray(centres, dtype=np.float64)
    r_faces = np.asarray(r_faces, dtype=np.float64)
    n_star = g / math.sqrt(cp * t0)
    eps = (n_freq / n_star) ** 2 - 1.0
    gamma = (cp - rd) / rd
    phi = np.arcsin(np.clip(centres[:, 2], -1.0, 1.0))
    e_h = np.exp(-n_freq ** 2 * jet_function(phi) / g ** 2)
    rc = 0.5 * (r_faces[:-1] + r_faces[1:])
    e_v = lambda r: np.exp(-n_freq ** 2 * radius * (r - 1.0) / g)

    def exact(r):   # [n, len(r)]: rho theta and rho / pi up to constants
        ehv = np.outer(e_h, e_v(r))
        pi = (eps + ehv) / (1.0 + eps)
        return pi ** gamma, pi ** (gamma - 1.0) * ehv

    a_c, b_c = exact(rc)
    a_f, _ = exact(r_faces)
    outer = dict(beta=b_c, alphaS=a_c, alphar=a_f * (r_faces / r_faces[0]) ** 2)
    pv = lambda r: (eps + e_v(r)) / (1.0 + eps)
    fac = dict(alphaS_r=pv(rc) ** gamma, beta_r=pv(rc) ** (gamma - 1.0) * e_v(rc),
               alphar_r=pv(r_faces) ** gamma * (r_faces / r_faces[0]) ** 2,
               alphaS_s=e_h ** gamma, alphar_s=e_h ** gamma, beta_s=e_h ** gamma)
    if advection:
        k_adv = n_freq ** 2 * radius / g
        outer["xi"] = a_f * k_adv
        fac["xi_r"] = pv(r_faces) ** gamma * k_adv
        fac["xi_s"] = e_h ** gamma
    return outer, fac, eps
