"""Planted mistakes: every plausible one-line error in the oracle must fail a pin.

Each mutant is the oracle source with one textual change (a dropped term, a
wrong sign, index, operand or loop order), compiled into a temporary library
and run against all pins of ``pins.py`` in a child process.  The test passes
when some pin rejects the mutant.  The mistakes are planted in the CPU oracle
only; nothing here touches a GPU.
"""
import concurrent.futures
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

MUTANTS = {
    "drop_horizontal_flux": ("for (e = 0; e < 3; ++e) s += alphaS_hat(o, G, T, e, k) * (u[i] - u[",
                             "for (e = 0; e < 3; ++e) s += 0.0 * alphaS_hat(o, G, T, e, k) * (u[i] - u["),
    "vertical_flux_sign": ("s += vert_down(o, G, T, k) * (u[i] - u[i - 1]);",
                           "s += vert_down(o, G, T, k) * (u[i] + u[i - 1]);"),
    "upper_face_index": ("const double a = alphar_hat(o, G, T, k + 1);",
                         "const double a = alphar_hat(o, G, T, k);"),
    "neighbour_slot_shift": ("(u[i] - u[(size_t)G->nbr[3 * T + e] * n + k]);",
                             "(u[i] - u[(size_t)G->nbr[3 * T + (e + 1) % 3] * n + k]);"),
    "column_solve_excess": ("e = m[k] + cd[k] * e / piv[k - 1];", "e = m[k] + cd[k] / piv[k - 1];"),
    "column_solve_back": ("x[k] = y[k] + cu[k] / piv[k] * x[k + 1];", "x[k] = y[k] + cd[k] / piv[k] * x[k + 1];"),
    "column_solve_forward": ("y[k] = (d[k] + cd[k] * y[k - 1]) / piv[k];", "y[k] = (d[k] - cd[k] * y[k - 1]) / piv[k];"),
    "column_solve_pivot_coupling": ("piv[k] = e + (k < n - 1 ? cu[k] : 0.0);", "piv[k] = e + (k < n - 1 ? cd[k] : 0.0);"),
    "advection_sign": ("return has_xi(o) ? a - o->dr[k] * xi_hat(o, G, T, k) : a;",
                       "return has_xi(o) ? a + o->dr[k] * xi_hat(o, G, T, k) : a;"),
    "advection_one_sided": ("return has_xi(o) ? a + o->dr[k] * xi_hat(o, G, T, k + 1) : a;",
                            "return has_xi(o) ? a + 2.0 * o->dr[k] * xi_hat(o, G, T, k + 1) : a;"),
    "advection_without_r2": ("(0.5 * o->arv[face]) * vfac(o->pr_xi, face)",
                             "(0.5 * o->arv[face] / (o->r[face] * o->r[face])) * vfac(o->pr_xi, face)"),
    "advection_neighbour_thickness": ("return has_xi(o) ? a - o->dr[k] * xi_hat(o, G, T, k) : a;",
                                      "return has_xi(o) ? a - o->dr[k > 0 ? k - 1 : k] * xi_hat(o, G, T, k) : a;"),
    "outer_advection_sign": ("up += o->dr[k] * (o->omega2 * G->area[T] * (0.5 * o->arv[k + 1]) * o->pf_xi[fa + 1]);",
                             "up -= o->dr[k] * (o->omega2 * G->area[T] * (0.5 * o->arv[k + 1]) * o->pf_xi[fa + 1]);"),
    "thomas_forward_index": ("dp[i] = (d[i] - a[i] * dp[i - 1]) / den;", "dp[i] = (d[i] - a[i - 1] * dp[i - 1]) / den;"),
    "thomas_backward_index": ("x[i] = dp[i] - cp[i] * x[i + 1];", "x[i] = dp[i] - cp[i + 1] * x[i + 1];"),
    "restrict_child_index": ("s += rf[(size_t)(4 * T + j) * n + k];", "s += rf[(size_t)(4 * T) * n + k];"),
    "post_smooth_order": ("smooth(o, l, f, u, o->nu_post, -1);", "smooth(o, l, f, u, o->nu_post, +1);"),
    "volume_factor": ("o->r[k + 1] * o->r[k + 1] + o->r[k + 1] * o->r[k] + o->r[k] * o->r[k]",
                      "o->r[k + 1] * o->r[k + 1] + o->r[k + 1] * o->r[k + 1] + o->r[k] * o->r[k]"),
    "area_half_excess": ("G->area[T] = 2.0 * atan2(num, den);", "G->area[T] = atan2(num, den);"),
    "g_without_edge_length": ("gval = len * v_dot(n, d) / v_dot(d, d);", "gval = v_dot(n, d) / v_dot(d, d);"),
    "g_distance_power": ("gval = len * v_dot(n, d) / v_dot(d, d);", "gval = len * v_dot(n, d) / sqrt(v_dot(d, d));"),
    "pcg_beta_inverted": ("beta = rz_new / rz;", "beta = rz / rz_new;"),
    "profile_edge_one_side": ("edge = 0.5 * (hfac(o, o->ps_aS, G, T) + hfac(o, o->ps_aS, G, G->nbr[3 * T + e]));",
                              "edge = hfac(o, o->ps_aS, G, T);"),
    "profile_coarse_unweighted": ("s += aj * p[l + 1][4 * T + j];", "s += p[l + 1][4 * T + j];"),
    "outer_edge_one_side": ("const double edge = 0.5 * (o->pf_aS[i] + o->pf_aS[(size_t)Tn * n + k]);",
                            "const double edge = o->pf_aS[i];"),
    "outer_upper_face": ("double up = o->omega2 * G->area[T] * o->arv[k + 1] * o->pf_ar[fa + 1];",
                         "double up = o->omega2 * G->area[T] * o->arv[k + 1] * o->pf_ar[fa];"),
    "bicgstab_omega_sign": ("r[i] = sv[i] - omega * t[i];", "r[i] = sv[i] + omega * t[i];"),
    "bicgstab_beta_ratio": ("beta = (rho / rho_prev) * (alpha / omega);", "beta = (rho / rho_prev) * (omega / alpha);"),
    "prolong_half": ("double s = uT;", "double s = 0.5 * uT;"),
    "correction_sign": ("uf[(size_t)(4 * T + j) * n + k] += s;", "uf[(size_t)(4 * T + j) * n + k] -= s;"),
    "horizontal_uses_volume": ("return coeff(o, o->omega2 * o->dr[k] * G->g[3 * T + e] * vfac(o->pr_aS, k) * edge);",
                               "return coeff(o, o->omega2 * o->vol[k] * G->g[3 * T + e] * vfac(o->pr_aS, k) * edge);"),
    "partial_takes_general_beta": ("static int full_now(const octx *o) { return o->vc_full == 1 && o->pl_beta; }",
                                   "static int full_now(const octx *o) { return o->vc_full >= 1 && o->pl_beta; }"),
    "partial_keeps_factorised_alphar": ("static int general_ar_now(const octx *o) { return o->vc_full >= 1 && o->pl_ar; }",
                                        "static int general_ar_now(const octx *o) { return o->vc_full == 1 && o->pl_ar; }"),
    "linear_parent_not_subtracted": ("s += w[j][e] * (uc[(size_t)Gc->nbr[3 * T + e] * n + k] - uT);",
                                     "s += w[j][e] * uc[(size_t)Gc->nbr[3 * T + e] * n + k];"),
    "linear_inverse_transposed": ("const double qx = (px * m11 - py * m01) / det",
                                  "const double qx = (px * m00 - py * m01) / det"),
    "linear_same_child": ("vec3 v = v_sub(Gf->centre[4 * T + j], c);", "vec3 v = v_sub(Gf->centre[4 * T], c);"),
    "bf16_truncates": ("return ldexp(rint(ldexp(m, 8)), e - 8);", "return ldexp(floor(ldexp(m, 8)), e - 8);"),
    "vertical_missing_r2": ("2.0 * o->r[k] * o->r[k] / (o->zeta[k + 1] - o->zeta[k - 1])",
                            "2.0 / (o->zeta[k + 1] - o->zeta[k - 1])"),
    "vertical_distance": ("2.0 * o->r[k] * o->r[k] / (o->zeta[k + 1] - o->zeta[k - 1])",
                          "2.0 * o->r[k] * o->r[k] / (o->zeta[k + 1] - o->zeta[k])"),
    "skip_last_colour": ("for (c = 0; c < G->n_colours; ++c) colour_pass(o, l, c, f, u);",
                         "for (c = 0; c < G->n_colours - 1; ++c) colour_pass(o, l, c, f, u);"),
    "child_orientation": ("c[3] = v0;  c[4] = m01; c[5] = m20;", "c[3] = v0;  c[4] = m20; c[5] = m01;"),
    "residual_sign": ("o->mg_r[l][i] = f[i] - o->mg_r[l][i];", "o->mg_r[l][i] = o->mg_r[l][i] - f[i];"),
    "vertex_mean_centre": ("G->centre[T] = v_unit(v_add(v_add(a, b), c));", "G->centre[T] = v_unit(v_add(a, b));"),
    "colouring_ignores_colour0": ("            if (c >= 0) used[c] = 1;", "            if (c >= 1) used[c] = 1;"),
    "colouring_lowest_saturation": ("for (s = 3; s >= 0 && T < 0; --s)", "for (s = 0; s < 4 && T < 0; ++s)"),
    "grading_exponent": ("pow(grading, (double)k)", "pow(grading, (double)(k + 1))"),
    "relaxation_ignored": ("u_in[(size_t)T * n + k] + o->relax * x[k];", "u_in[(size_t)T * n + k] + x[k];"),
    "diag_misses_mass": ("b[k] = beta_hat(o, G, T, k) + hs;", "b[k] = hs;"),
    "pcg_alpha_inverted": ("alpha = rz / pq;", "alpha = pq / rz;"),
    "coarse_sweep_one_way": ("smooth(o, l, f, u, o->nu_coarse, 0);", "smooth(o, l, f, u, o->nu_coarse, +1);"),
}

DRIVER = textwrap.dedent("""
    import functools, sys, types
    sys.path[:0] = [{root!r}, {tests!r}]
    import oracle, pins
    lib = sys.argv[1]
    ns = types.SimpleNamespace(Oracle=functools.partial(oracle.Oracle, lib_path=lib),
                               thomas=functools.partial(oracle.thomas, lib_path=lib),
                               column_solve=functools.partial(oracle.column_solve, lib_path=lib),
                               column_solve2=functools.partial(oracle.column_solve2, lib_path=lib),
                               bf16=functools.partial(oracle.bf16, lib_path=lib))
    for p in pins.ALL_PINS:
        try:
            p(ns)
        except Exception as exc:
            print("REJECTED_BY", p.__name__, type(exc).__name__)
            sys.exit(0)
    print("ALL_PINS_PASSED")
    sys.exit(3)
""")


def _run_mutant(name: str, work: str):
    """Compile the oracle with one planted mistake and run every pin on it in a child
    process; returns (mutation site found, return code, stdout, stderr tail)."""
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    if src.count(old) < 1:
        return False, None, "", ""
    d = os.path.join(work, name)
    os.makedirs(d, exist_ok=True)
    c_path = os.path.join(d, "mutant.c")
    with open(c_path, "w") as fh:
        fh.write(src.replace(old, new, 1))
    lib = oracle.compile_source(c_path, os.path.join(d, "libmutant.so"))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    proc = subprocess.run([sys.executable, "-c", DRIVER.format(root=ROOT, tests=TESTS), lib],
                          capture_output=True, text=True, timeout=600, env=env)
    return True, proc.returncode, proc.stdout, proc.stderr[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """All mutants, compiled and checked in parallel (independent child processes)."""
    work = str(tmp_path_factory.mktemp("mutants"))
    workers = max(1, min(len(MUTANTS), len(os.sched_getaffinity(0))))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        futures = {name: ex.submit(_run_mutant, name, work) for name in MUTANTS}
        return {name: f.result() for name, f in futures.items()}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, mutant_results):
    found, rc, out, err = mutant_results[name]
    assert found, f"mutation site for {name} not found"
    assert rc == 0 and "REJECTED_BY" in out, (rc, out, err)
