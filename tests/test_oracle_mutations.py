"""The oracle's pins catch plausible mistakes.  Each mistake below is planted, one at a time, in a
copy of the oracle's source (on the CPU, in a temporary directory), the copy is built, and the
pin named beside it must then fail; the unchanged copy passes the same pins.  The mistakes are
those a restatement of the method could plausibly contain: a wrong quadrature point, Jacobian or
local node order, a transposed band index, a missed Dirichlet elimination, a wrong child cell, a
dropped band, flipped signs, a missing damping factor or square root, wrong transfer weights,
rounding ties away from even, a wrong subnormal threshold, a signed maximum for the FP16 scale,
a short row sum, swapped smoothing counts, an unscaled correction, wrong Cholesky indices, CG and
PCG update mistakes, stopping rules that are off by a factor or a cycle, a swapped side bit,
transfers that skip the free sides as if they were Dirichlet, Dirichlet rows kept in the load,
wrong load-vector quadrature or source factor, a wrong corner of the error's interpolant, a wrong
FP16 subnormal decoding, a float accumulator for the dot product, two roundings in axpy, a dropped
band and swapped operands or sign in the shallow-water step.

Four further changes leave the oracle's results unchanged and are therefore not mistakes: the
sign of every y-derivative of the element basis (the stiffness is quadratic in it), the weight of
a coarse node that is never a parent of the fine node, prolongation into fine Dirichlet nodes
(all their coarse parents are Dirichlet nodes, so nothing is added), and the scale of the PCG
preconditioner's output (conjugate gradients are invariant under a positive scaling of the
preconditioned residual at each step, up to rounding)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py"

# (name, text in hn_oracle.cpp, planted text, pin that must fail)
MUTATIONS = [
    ("stiffness_gauss_point", "const double g = 0.5 / std::sqrt(3.0);", "const double g = 0.5 / std::sqrt(2.0);",
     "test_element_stiffness_closed_form"),
    ("stiffness_jacobian", "const double w = wts[qx] * wts[qy] * h * h;     // |Jacobian| = h^2",
     "const double w = wts[qx] * wts[qy] * h;",
     "test_element_stiffness_closed_form"),
    ("stiffness_node_order",
     "const int lx[4] = {0, 1, 1, 0}, ly[4] = {0, 0, 1, 1};\n  for (int a = 0; a < 4; ++a)\n    for (int b = 0; b < 4; ++b) K[a][b] = 0.0;",
     "const int lx[4] = {0, 1, 0, 1}, ly[4] = {0, 0, 1, 1};\n  for (int a = 0; a < 4; ++a)\n    for (int b = 0; b < 4; ++b) K[a][b] = 0.0;",
     "test_element_stiffness_closed_form"),
    ("assembly_transposed_band", "const int k = band_of((int)(jy - iy), (int)(jx - ix));",
     "const int k = band_of((int)(jx - ix), (int)(jy - iy));",
     "test_variable_coefficient_matches_independent_quadrature"),
    ("assembly_no_elimination", "if (!on_grid(jx, jy, n) || is_boundary(jx, jy, n)) bands[k * N + i] = 0.0;",
     "if (!on_grid(jx, jy, n)) bands[k * N + i] = 0.0;", "test_band_layout_exact"),
    ("coarsening_wrong_child", "af[(y + 1) * ncf + x + 1]) * 0.25;", "af[(y + 1) * ncf + x]) * 0.25;",
     "test_coarsen_coef_linear_field"),
    ("spmv_dropped_band",
     "      for (int k = 0; k < 9; ++k) {\n        const long jx = ix + band_dx(k), jy = iy + band_dy(k);\n        if (jx < 0 || jy < 0 || jx >= n || jy >= n) continue;\n        s += bands[k * N + i] * x[jy * n + jx];",
     "      for (int k = 0; k < 8; ++k) {\n        const long jx = ix + band_dx(k), jy = iy + band_dy(k);\n        if (jx < 0 || jy < 0 || jx >= n || jy >= n) continue;\n        s += bands[k * N + i] * x[jy * n + jx];",
     "test_spmv_eigenpairs"),
    ("defect_sign", "for (long i = 0; i < N; ++i) r[i] = b[i] - ax[i];", "for (long i = 0; i < N; ++i) r[i] = ax[i] - b[i];",
     "test_mg_matches_dense_lu"),
    ("jacobi_without_damping", "x_out[i] = x_in[i] + omega * r[i] / diag_of<T>(bands, N, i);",
     "x_out[i] = x_in[i] + r[i] / diag_of<T>(bands, N, i);", "test_jacobi_error_propagation"),
    ("norm_without_sqrt", "s += (double)v[i] * (double)v[i];\n  return std::sqrt(s);",
     "s += (double)v[i] * (double)v[i];\n  return s;", "test_mg_matches_dense_lu"),
    ("restriction_quarter_prefactor", "if (w != 0.0) rc[Cy * nc + Cx] += (T)w * rf[fy * nf + fx];",
     "if (w != 0.0) rc[Cy * nc + Cx] += (T)(0.25 * w) * rf[fy * nf + fx];", "test_restriction_of_modes"),
    ("interpolation_even_weight", "if (f % 2 == 0) return (f / 2 == C) ? 1.0 : 0.0;",
     "if (f % 2 == 0) return (f / 2 == C) ? 0.5 : 0.0;", "test_prolongation_reproduces_bilinear"),
    ("fp16_ties_away", "double m = std::nearbyint(std::ldexp(a, 10 - e));", "double m = std::round(std::ldexp(a, 10 - e));",
     "test_fp16_rne_matches_ieee"),
    ("fp16_subnormal_threshold", "if (a < std::ldexp(1.0, -14)) {", "if (a < std::ldexp(1.0, -15)) {",
     "test_fp16_rne_matches_ieee"),
    ("fp16_signed_scale", "for (long i = 0; i < N; ++i) mx = std::fmax(mx, std::fabs(v[i]));",
     "for (long i = 0; i < N; ++i) mx = std::fmax(mx, v[i]);", "test_quantize_fp16_bands"),
    ("fp16_short_row_sum", "    for (int k = 0; k < 9; ++k) rho[i] += bands[k * N + i];",
     "    for (int k = 0; k < 8; ++k) rho[i] += bands[k * N + i];", "test_mixed_precision_reaches_fp64_tolerance"),
    ("rowsum_diagonal_sign", "    if (k != 4) d -= bands[k * N + i];", "    if (k != 4) d += bands[k * N + i];",
     "test_mixed_precision_reaches_fp64_tolerance"),
    ("rowsum_without_centre", "      float s = bands[4 * N + i] * x[i];", "      float s = 0.0f;",
     "test_mixed_precision_reaches_fp64_tolerance"),
    ("cycle_post_count_from_pre",
     "  for (int s = 0; s < post; ++s) { jacobi<T>(lv.L, A, omega, b, x, t.data()); std::copy(t.begin(), t.end(), x); }\n}",
     "  for (int s = 0; s < pre; ++s) { jacobi<T>(lv.L, A, omega, b, x, t.data()); std::copy(t.begin(), t.end(), x); }\n}",
     "test_one_cycle_equals_its_dense_composition"),
    ("correction_unscaled", "      for (long i = 0; i < N; ++i) x[i] += dn * (double)c[i];",
     "      for (long i = 0; i < N; ++i) x[i] += (double)c[i];", "test_mixed_precision_reaches_fp64_tolerance"),
    ("cholesky_index", "        for (long k = 0; k < j; ++k) s -= chol[i * m + k] * chol[j * m + k];",
     "        for (long k = 0; k < j; ++k) s -= chol[i * m + k] * chol[i * m + k];", "test_coarse_solve_matches_dense"),
    ("cholesky_back_substitution", "      for (long k = i + 1; k < m; ++k) s -= chol[k * m + i] * y[k];",
     "      for (long k = i + 1; k < m; ++k) s -= chol[i * m + k] * y[k];", "test_coarse_solve_matches_dense"),
    ("cg_beta_inverted", "      const double beta = rr_new / rr;", "      const double beta = rr / rr_new;",
     "test_coarse_cg_matches_cholesky"),
    ("pcg_direction_from_residual", "      for (long i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];",
     "      for (long i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];", "test_pcg_follows_scipy_cg"),
    ("inner_cap_one_short", "      for (int k = 0; k < inner_max; ++k) {", "      for (int k = 0; k < inner_max - 1; ++k) {",
     "test_inner_cycles_per_outer_step_are_capped"),
    ("inner_stop_absolute", "        if (norm2<float>(N, t.data()) <= inner_tol * dhn) break;",
     "        if (norm2<float>(N, t.data()) <= inner_tol * 0.5) break;",
     "test_inner_solve_stops_like_the_fp32_solve_of_the_scaled_defect"),
    ("outer_stop_loose", "      if (rr <= tol) { s.converged = 1; break; }", "      if (rr <= 10 * tol) { s.converged = 1; break; }",
     "test_stopping_rule_is_the_first_iterate_within_tolerance"),
    ("mg_stop_one_cycle_late",
     "    while (rr > tol && s.cycles < max_cycles) {\n      vcycle<double>(H, 0, x, b, pre, post, omega);",
     "    while (rr > 0.1 * tol && s.cycles < max_cycles) {\n      vcycle<double>(H, 0, x, b, pre, post, omega);",
     "test_stopping_rule_is_the_first_iterate_within_tolerance"),
    ("side_mask_bit", "(ix == n - 1 && (m & 2u))", "(ix == n - 1 && (m & 4u))",
     "test_mixed_bc_operator_symmetric_and_natural"),
    ("load_quadrature_weights", "  const double wts[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};\n  const int lx[4]",
     "  const double wts[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};\n  const int lx[4]",
     "test_load_vector_matches_the_exact_integral"),
    ("load_source_factor", "const double f = 2.0 * M_PI * M_PI * u(px, py);", "const double f = M_PI * M_PI * u(px, py);",
     "test_load_vector_matches_the_exact_integral"),
    ("l2_error_interpolant_corner",
     "xi * eta * x[(ey + 1) * n + ex + 1] + (1 - xi) * eta * x[(ey + 1) * n + ex];",
     "xi * eta * x[(ey + 1) * n + ex] + (1 - xi) * eta * x[(ey + 1) * n + ex + 1];",
     "test_l2_error_of_zero_and_of_interpolant"),
    ("fp16_decode_subnormal", "if (e == 0) v = std::ldexp((double)f, -24);", "if (e == 0) v = std::ldexp((double)f, -25);",
     "test_fp16_decoding_matches_ieee"),
    ("dot_float_accumulator", "double or_dot_f32(long n, const float* x, const float* y) {\n  long double s = 0.0L;",
     "double or_dot_f32(long n, const float* x, const float* y) {\n  float s = 0.0f;",
     "test_oracle_dot_closed_form_and_exact_sum"),
    ("axpy_two_roundings", "void or_axpy_f32(long n, float a, const float* x, float* y) {\n  for (long i = 0; i < n; ++i) y[i] = std::fma(a, x[i], y[i]);",
     "void or_axpy_f32(long n, float a, const float* x, float* y) {\n  for (long i = 0; i < n; ++i) y[i] = a * x[i] + y[i];",
     "test_oracle_axpy_single_rounding"),
    ("band4_first_band_dropped", "  for (int k = 0; k < 4; ++k) {\n    const long long j = (long long)i + off[k];",
     "  for (int k = 1; k < 4; ++k) {\n    const long long j = (long long)i + off[k];", "test_band4_against_scipy_diagonals"),
    ("swe_operands_swapped", "const T* xs[4] = {v, w, u, u};", "const T* xs[4] = {w, v, u, u};",
     "test_swe_predict_exact_on_integers"),
    ("swe_source_sign", "u_new[i] = s ? t + s[i] : t;", "u_new[i] = s ? t - s[i] : t;",
     "test_swe_predict_exact_on_integers"),
    ("coarse_cg_tolerance", "constexpr double kCgTol = 1e-13;", "constexpr double kCgTol = 1e-4;",
     "test_coarse_cg_matches_cholesky"),
    ("fp16_quotient_in_float", "codes[k * N + i] = fp16_rne(v[i] / (double)s);",
     "codes[k * N + i] = fp16_rne((double)((float)v[i] / s));", "test_quantize_fp16_bands"),
    ("hierarchy_without_coarsening", "        coarsen_coef(l, a.data(), ac.data());\n        a.swap(ac);",
     "        coarsen_coef(l, a.data(), ac.data());", "test_mg_matches_dense_lu"),
    ("restriction_skips_free_sides", "      if (is_boundary(fx, fy, nf)) continue;\n      for (long Cy",
     "      if (fx == 0 || fy == 0 || fx == nf - 1 || fy == nf - 1) continue;\n      for (long Cy",
     "test_mixed_bc_transfers_adjoint_and_exact"),
    ("prolongation_skips_free_sides", "      if (is_boundary(fx, fy, nf)) continue;\n      T s = 0;",
     "      if (fx == 0 || fy == 0 || fx == nf - 1 || fy == nf - 1) continue;\n      T s = 0;",
     "test_mixed_bc_transfers_adjoint_and_exact"),
    ("load_dirichlet_rows_kept", "      if (is_boundary(ix, iy, n)) b[iy * n + ix] = 0.0;\n}", "      if (false) b[iy * n + ix] = 0.0;\n}",
     "test_load_vector_matches_the_exact_integral"),
    ("pcg_alpha_denominator", "      const double alpha = rho / dot64(N, p.data(), q.data());",
     "      const double alpha = rho / dot64(N, r.data(), q.data());", "test_pcg_follows_scipy_cg"),
]


def _copy_tree(dst):
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("__init__.py", "build.py", "hn_oracle.cpp"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))


def _run(dst, old, new, pin):
    """Plant `new` for `old` (None: nothing), build the copy, run the pin; (exit code, tail)."""
    src = os.path.join(dst, "oracle", "hn_oracle.cpp")
    if old is not None:
        text = open(src).read()
        assert text.count(old) == 1, "the text to change must occur once"
        open(src, "w").write(text.replace(old, new))
    subprocess.run([sys.executable, os.path.join(dst, "oracle", "build.py"), "--force"], check=True,
                   capture_output=True)
    env = dict(os.environ, PYTHONPATH=dst + os.pathsep + ROOT)
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-q", "-p", "no:cacheprovider", "-k", pin],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("oracle_mutations")
    jobs = [("unchanged", None, None, " or ".join(sorted({m[3] for m in MUTATIONS})))] + MUTATIONS
    for name, *_ in jobs:
        _copy_tree(str(base / name))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        res = ex.map(lambda j: (j[0], _run(str(base / j[0]), j[1], j[2], j[3])), jobs)
        return dict(res)


def test_unchanged_copy_passes_the_pins(outcomes):
    rc, out = outcomes["unchanged"]
    assert rc == 0, out


@pytest.mark.parametrize("name,pin", [(m[0], m[3]) for m in MUTATIONS], ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(outcomes, name, pin):
    rc, out = outcomes[name]
    assert rc == 1, out            # pytest's exit code for failed tests (not an error or a crash)
    assert " failed" in out and pin in out
