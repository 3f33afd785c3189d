"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle into a temporary directory, plants one mistake
in the copy of oracle.c (a dropped term, a wrong sign, index or operand, a
wrong preconditioner), builds it with gcc and runs the pins against it: at
least one pin must fail.  The committed oracle is never modified.
"""
import importlib.util
import os
import shutil
import sys

import pytest

import test_oracle_pins as P

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTANTS = {
    "spmv_row_index_for_column": ("s += vals[k] * x[colidx[k]];\n        y[i] = s;\n    }\n}\n\n/* The same product in binary32",
                                  "s += vals[k] * x[i];\n        y[i] = s;\n    }\n}\n\n/* The same product in binary32"),
    "spmv_skips_last_entry": ("double s = 0.0;\n        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)",
                              "double s = 0.0;\n        for (int64_t k = rowptr[i]; k + 1 < rowptr[i + 1]; ++k)"),
    "residual_update_sign": ("orc_axpy(n, -alpha, q, r);", "orc_axpy(n, alpha, q, r);"),
    "beta_inverted": ("double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    "no_preconditioner_in_loop": ("for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];\n            double rho_new",
                                  "for (int64_t i = 0; i < n; ++i) z[i] = r[i];\n            double rho_new"),
    "dinv_not_inverted": ("dinv[i] = 1.0 / d;", "dinv[i] = d;"),
    "aypx_roles_swapped": ("y[i] = x[i] + beta * y[i];", "y[i] = beta * x[i] + y[i];"),
    "norm_without_sqrt": ("return sqrt(orc_dot(n, x, x));", "return orc_dot(n, x, x);"),
    "pi_from_wrong_operands": ("double pi = orc_dot(n, p, q);", "double pi = orc_dot(n, q, q);"),
    "x_update_with_z": ("orc_axpy(n, alpha, p, x);", "orc_axpy(n, alpha, z, x);"),
    "rho_unpreconditioned": ("double rho = orc_dot(n, r, z);", "double rho = orc_dot(n, r, r);"),
    "dot2_drops_product_error": ("s += e + r;", "s += e;"),
    "f32_residual_sign": ("r[i] = -alpha * q[i] + r[i];", "r[i] = alpha * q[i] + r[i];"),
    "mixed_update_unscaled": ("x[i] += rn * (double)d32[i];", "x[i] += (double)d32[i];"),
    "csr_check_allows_duplicates": ("colidx[k] <= colidx[k - 1]", "colidx[k] < colidx[k - 1]"),
    "cheb_direction_unpreconditioned": ("d[i] = a1 * d[i] + a2 * (dinv[i] * r[i]);",
                                        "d[i] = a1 * d[i] + a2 * r[i];"),
    "cheb_rho_frozen": ("rho = delta / c;", "rho = delta / theta;"),
    "cheb_first_direction_unscaled": ("d[i] = (dinv[i] * r[i]) / theta;", "d[i] = dinv[i] * r[i];"),
    "cheb_residual_sign": ("r[i] = r[i] - q[i];", "r[i] = r[i] + q[i];"),
    "cheb_interval_centre_and_radius_swapped": (
        "const double theta = 0.5 * (emax + emin), delta = 0.5 * (emax - emin);",
        "const double theta = 0.5 * (emax - emin), delta = 0.5 * (emax + emin);"),
    "coo_unstable_column_sort": ("while (q >= a && tj[order[q]] > tj[key]) {",
                                 "while (q >= a && tj[order[q]] >= tj[key]) {"),
    "coo_duplicates_not_merged": ("while (p < b && tj[order[p]] == c) {", "while (0) {"),
    "coo_last_duplicate_wins": ("s = s + v[order[p]];", "s = v[order[p]];"),
    "precond_norm_of_r": ("return norm == 1 ? orc_norm2(n, w) : sqrt(orc_dot(n, v, w));",
                          "return norm == 1 ? orc_norm2(n, v) : sqrt(orc_dot(n, v, w));"),
    "natural_norm_without_sqrt": ("return norm == 1 ? orc_norm2(n, w) : sqrt(orc_dot(n, v, w));",
                                  "return norm == 1 ? orc_norm2(n, w) : orc_dot(n, v, w);"),
    "norm_reference_unpreconditioned": ("const double bnorm = orc_test_norm(norm, n, b, dinv, w);",
                                        "const double bnorm = orc_norm2(n, b);"),
    "f32_beta_inverted": ("float beta = rho_new / rho;", "float beta = rho / rho_new;"),
    "f32_no_preconditioner_in_loop": (
        "for (int64_t i = 0; i < n; ++i) z[i] = dinv32[i] * r[i];\n        float rho_new",
        "for (int64_t i = 0; i < n; ++i) z[i] = r[i];\n        float rho_new"),
    "mixed_residual_sign": ("r[i] = b[i] - r[i];", "r[i] = r[i] - b[i];"),
    "mixed_rhs_not_normalised": ("r32[i] = (float)(r[i] / rn);", "r32[i] = (float)r[i];"),
    "mixed_stagnation_test_inverted": ("if (rn > 0.5 * prev)", "if (rn < 0.5 * prev)"),
    "mixed_inner_tolerance_fixed": ("const double eta_j = fmax(inner_rtol, 0.5 * rtol * bnorm / rn);",
                                    "const double eta_j = inner_rtol;"),
    "mixed_inner_tolerance_full_target": (
        "const double eta_j = fmax(inner_rtol, 0.5 * rtol * bnorm / rn);",
        "const double eta_j = fmax(inner_rtol, rtol * bnorm / rn);"),
    "spmv_f32_row_index_for_column": (
        "float s = 0.0f;\n        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)\n"
        "            s += vals[k] * x[colidx[k]];",
        "float s = 0.0f;\n        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)\n"
        "            s += vals[k] * x[i];"),
    "aypx_fused_roles_swapped": ("y[i] = fma(beta, y[i], x[i]);", "y[i] = fma(beta, x[i], y[i]);"),
    "axpy_fused_rounds_twice": ("y[i] = fma(alpha, x[i], y[i]);", "y[i] = alpha * x[i] + y[i];"),
    "block_alpha_operands_swapped": ("if (orc_ldl_solve(k, pi, rho, alpha))",
                                     "if (orc_ldl_solve(k, rho, pi, alpha))"),
    "block_residual_sign": ("r = r - Q[i + m * n] * alpha[m + j * k];",
                            "r = r + Q[i + m * n] * alpha[m + j * k];"),
    "block_rho_unpreconditioned": ("orc_gram(n, k, Z, R, rho2);", "orc_gram(n, k, R, R, rho2);"),
    "block_beta_transposed": ("p = p + P[i + m * n] * beta[m + j * k];",
                              "p = p + P[i + m * n] * beta[j + m * k];"),
    "block_alpha_transposed_in_x": ("x = x + P[i + m * n] * alpha[m + j * k];",
                                    "x = x + P[i + m * n] * alpha[j + m * k];"),
    "block_no_preconditioner": ("for (size_t e = 0; e < nk; ++e) Z[e] = dinv[e % (size_t)n] * R[e];",
                                "for (size_t e = 0; e < nk; ++e) Z[e] = R[e];"),
    "ldl_pivot_update_dropped": ("for (int m = 0; m < j; ++m) d -= L[j + m * k] * L[j + m * k] * D[m];",
                                 "for (int m = 0; m < j; ++m) d -= L[j + m * k] * D[m];"),
}

PINS = [
    lambda o: P.test_spmv_dense_bruteforce_nonsymmetric_rectangular(o),
    lambda o: P.test_spmv_exact_inputs_bitwise(o),
    lambda o: P.test_spmv_laplacian_row_sums(o),
    lambda o: P.test_csr_check(o),
    lambda o: P.test_dot_norm_exact(o),
    lambda o: P.test_dot2_is_twice_working_precision(o),
    lambda o: P.test_axpy_aypx_roles(o),
    lambda o: P.test_fused_axpy_aypx_round_the_exact_value_once(o),
    lambda o: P.test_spmv_f32_matches_rounded_double(o),
    lambda o: P.test_jacobi_dinv(o),
    lambda o: P.test_pcg_iterates_are_krylov_minimisers(o, 3),
    lambda o: P.test_pcg_finite_termination(o, lambda: P.I.lap2d5(2), 3),
    lambda o: P.test_pcg_iteration_bound_2d(o),
    lambda o: P.test_pcg_diagonal_matrix_one_step(o),
    lambda o: P.test_pcg_f32_close_to_fp64(o),
    lambda o: P.test_mixed_refinement_reaches_fp64_accuracy(o),
    lambda o: P.test_mixed_last_step_stops_at_half_the_target(o),
    lambda o: P.test_chebyshev_error_is_the_scaled_chebyshev_polynomial(o, 5),
    lambda o: P.test_chebyshev_rate_with_exact_bounds(o),
    lambda o: P.test_chebyshev_single_eigenvalue_and_arguments(o),
    lambda o: P.test_coo_assembly_equals_dense_accumulation_and_scipy(o),
    lambda o: P.test_coo_duplicates_are_summed_in_triplet_order(o),
    lambda o: P.test_coo_degenerate_and_invalid(o),
    lambda o: P.test_pcg_norms_with_constant_diagonal_scale_exactly(o),
    lambda o: P.test_pcg_norms_follow_their_definitions(o),
    lambda o: P.test_block_pcg_iterates_are_block_krylov_minimisers(o, 2),
    lambda o: P.test_block_pcg_finite_termination(o, 2, 3),
    lambda o: P.test_block_pcg_against_dense_solve_and_fewer_steps(o),
]


def _load_mutant(tmp_path, name, old, new):
    d = tmp_path / f"oracle_{name}"
    shutil.copytree(ORACLE_DIR, d, ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp"))
    src = (d / "oracle.c").read_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    (d / "oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    mod.build()
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    mut = _load_mutant(tmp_path, name, old, new)
    caught = []
    for pin in PINS:
        try:
            pin(mut)
        except Exception:          # an assertion, or a failure to converge
            caught.append(pin)
    assert caught, f"no pin fails with mutation {name}"
