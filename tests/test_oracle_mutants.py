"""Planted mistakes in the oracle: each pin set must catch its mutant.

The oracle is trusted because independent pins (closed forms, KKT and
duality certificates, brute-force Hopf-Lax minimisation, finite differences)
agree with it.  This file checks that the pins would notice a plausible
mistake: each case copies the oracle, the tests and the input generators to a
scratch directory, plants one mistake in the copy of ``hopf_oracle.c`` (a
dropped term, a wrong sign, scale or index, a transposed operand, a swapped
min and max), rebuilds it there and runs the named pins, which must fail.
The copy in the repository is never touched, and nothing here runs on a GPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in hopf_oracle.c, planted replacement, pins that must fail (-k))
MUTANTS = [
    # split Bregman, eq. 3.4(a)-(c)
    ("vupdate_drops_lambda", "tmp[i] = y[i] + lam * (d[i] - b[i]);", "tmp[i] = y[i] + (d[i] - b[i]);",
     "test_paper_example_l1_ellipsoid"),
    ("tau_is_t", "const double lam = p->lambda, tau = t / p->lambda;", "const double lam = p->lambda, tau = t;",
     "test_paper_example_l1_ellipsoid"),
    ("bregman_sign", "b[i] = b[i] + v[i] - dn[i];", "b[i] = b[i] - v[i] + dn[i];",
     "test_workload1_closed_form"),
    ("gradient_is_v", "for (int i = 0; i < n; ++i) grad[i] = d[i];", "for (int i = 0; i < n; ++i) grad[i] = v[i];",
     "test_dense_wl1_kkt_certificate"),
    # the paper's stop rule (Section 4.5): residuals from the wrong iterates
    ("paper_residual_v_from_d", "r1 += (v[i] - vprev[i]) * (v[i] - vprev[i]);",
     "r1 += (dn[i] - vprev[i]) * (dn[i] - vprev[i]);", "test_paper_stop_rule_exact_iterations"),
    ("paper_residual_gap_is_b", "r3 += (dn[i] - v[i]) * (dn[i] - v[i]);",
     "r3 += (dn[i] - d[i]) * (dn[i] - d[i]) * 0.25;", "test_paper_stop_rule_exact_iterations"),
    ("diag_solve_drops_lambda", "v[i] = r[i] / (p->A[i] + p->lambda);", "v[i] = r[i] / p->A[i];",
     "test_workload1_closed_form"),
    # the factorisation of A + lambda I and its solve
    ("factor_drops_lambda", "double s = A[(int64_t)i * n + j] + (i == j ? lambda : 0.0);",
     "double s = A[(int64_t)i * n + j];", "test_dense_wl1_kkt_certificate"),
    ("backsolve_transposed", "for (int k = i + 1; k < n; ++k) s -= L[(int64_t)k * n + i] * v[k];",
     "for (int k = i + 1; k < n; ++k) s -= L[(int64_t)i * n + k] * v[k];", "test_dense_wl1_kkt_certificate"),
    # the objective of eq. 3.3 and the outputs
    ("c0_sign", "return s - 0.5 * quad_A(p, v) - p->c0", "return s - 0.5 * quad_A(p, v) + p->c0",
     "test_paper_example_sphere"),
    ("centre_dropped", "s += (x[i] - (p->c ? p->c[i] : 0.0)) * v[i];", "s += x[i] * v[i];",
     "test_weighted_l1_with_centre"),
    ("jstar_diag_unweighted", "s += p->A[i] * v[i] * v[i];", "s += v[i] * v[i];", "test_workload1_closed_form"),
    ("dphidt_sign", "res->dphidt = -orc_H(p->h_kind, n, p->w, d);", "res->dphidt = orc_H(p->h_kind, n, p->w, d);",
     "test_time_derivative_and_gradient_fd"),
    # the proxes (Sections 1, 4.2-4.4)
    ("weights_ignored", "double a = tau * (h_kind == ORC_H_WL1 && w ? w[i] : 1.0);", "double a = tau;",
     "test_weighted_l1_with_centre"),
    ("dnorm_H_not_rooted", "s += w[i] * q[i] * q[i];\n        return sqrt(s);", "s += w[i] * q[i] * q[i];\n        return s;",
     "test_l2sq_initial_data_closed_forms_new_H"),
    ("shrink2_half_tau", "double m = nz - tau > 0.0 ? nz - tau : 0.0;",
     "double m = nz - 0.5 * tau > 0.0 ? nz - 0.5 * tau : 0.0;", "test_paper_example_sphere"),
    ("linf_H_is_l1", "for (int i = 0; i < n; ++i) s = fabs(q[i]) > s ? fabs(q[i]) : s;\n        return s;\n    }\n    if (h_kind == ORC_H_DNORM)",
     "for (int i = 0; i < n; ++i) s += fabs(q[i]);\n        return s;\n    }\n    if (h_kind == ORC_H_DNORM)",
     "test_l2sq_initial_data_closed_forms_new_H"),
    ("l1ball_mu_off_by_one", "const double mu = (S - radius) / k;", "const double mu = (S - radius) / (k + 1);",
     "test_new_prox_against_their_definition"),
    ("ellipsoid_prox_is_projection", "out[i] = z[i] * mu / (s2[i] + mu);", "out[i] = z[i] * s2[i] / (s2[i] + mu);",
     "test_new_prox_against_their_definition"),
    ("ellipsoid_radius_not_squared", "s2[i] = tau * tau * w[i];", "s2[i] = tau * w[i];",
     "test_new_prox_against_their_definition"),
    ("anorm_rotation_transposed", "for (int i = 0; i < n; ++i) s += P[(int64_t)i * n + k] * z[i];",
     "for (int i = 0; i < n; ++i) s += P[(int64_t)k * n + i] * z[i];", "test_anorm_prox_against_its_definition"),
    ("l1sq_beta_drops_alpha", "const double beta = alpha * S / (1.0 + alpha * k);",
     "const double beta = alpha * S / (1.0 + k);", "test_l1sq_beta_fixed_point_including_ties"),
    ("breakpoints_ascending", "return x < y ? 1 : (x > y ? -1 : 0);", "return x < y ? -1 : (x > y ? 1 : 0);",
     "test_l1sq_beta_fixed_point_including_ties"),
    # the non-quadratic initial data of Section 4.4
    ("jstar_moreau_swap", "p->a_kind == ORC_J_LINFSQ ? alpha : 1.0 / alpha, tmp);",
     "p->a_kind == ORC_J_LINFSQ ? 1.0 / alpha : alpha, tmp);", "test_nonquadratic_initial_data_bruteforce_n2"),
    ("jstar_linf_not_squared", "for (int i = 0; i < p->n; ++i) s = fabs(v[i]) > s ? fabs(v[i]) : s;\n        return s * s;",
     "for (int i = 0; i < p->n; ++i) s = fabs(v[i]) > s ? fabs(v[i]) : s;\n        return s;",
     "test_nonquadratic_initial_data_bruteforce_n2"),
    # unions, the maximum over Hamiltonians, the level-set distance (Sections 2.2, 3.2)
    ("union_takes_max", "double best = INFINITY;\n            int bi = -1, it = 0;\n            for (int i = 0; i < K; ++i) {\n                orc_result r;\n                orc_solve(&parts[i], L[i], x + q * n, t[q], g, &r, work, NULL);\n                it += r.iters;\n                if (r.phi < best) {",
     "double best = -INFINITY;\n            int bi = -1, it = 0;\n            for (int i = 0; i < K; ++i) {\n                orc_result r;\n                orc_solve(&parts[i], L[i], x + q * n, t[q], g, &r, work, NULL);\n                it += r.iters;\n                if (r.phi > best) {",
     "test_union_min_rule"),
    ("maxH_takes_min", "double best = -INFINITY;\n            int bi = -1, it = 0;\n            for (int i = 0; i < K; ++i) {\n                orc_result r;\n                orc_solve(&parts[i], L, x + q * n, t[q], g, &r, work, NULL);\n                it += r.iters;\n                if (r.phi > best) {",
     "double best = INFINITY;\n            int bi = -1, it = 0;\n            for (int i = 0; i < K; ++i) {\n                orc_result r;\n                orc_solve(&parts[i], L, x + q * n, t[q], g, &r, work, NULL);\n                it += r.iters;\n                if (r.phi < best) {",
     "test_max_over_hamiltonians_solves_the_min_hamiltonian_pde"),
    ("union_ties_to_last", "it += r.iters;\n                if (r.phi < best) {", "it += r.iters;\n                if (r.phi <= best) {",
     "test_ties_go_to_the_smallest_index"),
    ("maxH_ties_to_last", "it += r.iters;\n                if (r.phi > best) {", "it += r.iters;\n                if (r.phi >= best) {",
     "test_ties_go_to_the_smallest_index"),
    ("closest_ties_to_last", "if (sb < best) {", "if (sb <= best) {", "test_ties_go_to_the_smallest_index"),
    ("newton_step_scaled", "double ds = r.phi / gn;", "double ds = r.phi / gn / gn;",
     "test_closest_point_against_ellipsoid_projection"),
    ("closest_takes_farthest", "if (sb < best) {", "if (sb > best) {",
     "test_closest_point_against_ellipsoid_projection"),
    ("projection_sign", "for (int i = 0; i < n; ++i) proj[i] = y[i] - s * g[i] / gn;",
     "for (int i = 0; i < n; ++i) proj[i] = y[i] + s * g[i] / gn;", "test_closest_point_against_ellipsoid_projection"),
    # gradients with respect to the data, and the control
    ("gA_drops_half", "g_A[(int64_t)i * n + j] -= 0.5 * g_phi[q] * v[i] * v[j];",
     "g_A[(int64_t)i * n + j] -= g_phi[q] * v[i] * v[j];", "test_backward_envelope_fd"),
    ("gw_dnorm_drops_half", "g_w[i] -= g_phi[q] * t[q] * v[i] * v[i] / (2.0 * H);",
     "g_w[i] -= g_phi[q] * t[q] * v[i] * v[i] / H;", "test_parameter_gradients_against_finite_differences"),
    ("gc0_sign", "*g_c0 -= g_phi[q];", "*g_c0 += g_phi[q];", "test_parameter_gradients_against_finite_differences"),
    ("control_drops_centre", "(xi - (p->c ? p->c[i] : 0.0) - ap) / t[q]", "(xi - ap) / t[q]",
     "test_control_is_a_subgradient_and_the_hopf_lax_minimiser"),
    ("warm_start_stops_at_k1", "(k >= 2 && ru <= p->tol)", "(ru <= p->tol)", "test_closest_point_against_ellipsoid_projection"),
    ("ellipsoid_newton_loose", "if (fabs(dmu) <= 1e-15 * (mu > 1.0 ? mu : 1.0)) break;",
     "if (fabs(dmu) <= 1e-3 * (mu > 1.0 ? mu : 1.0)) break;", "test_l2sq_initial_data_closed_forms_new_H"),
    ("gt_sign", "g_t[q] = -g_phi[q] * orc_H(h_kind, n, w, v);", "g_t[q] = g_phi[q] * orc_H(h_kind, n, w, v);",
     "test_backward_envelope_fd"),
    ("gA_diag_drops_half", "for (int i = 0; i < n; ++i) g_A[i] -= 0.5 * g_phi[q] * v[i] * v[i];",
     "for (int i = 0; i < n; ++i) g_A[i] -= g_phi[q] * v[i] * v[i];", "test_backward_diagonal_A_fd"),
    ("gw_wl1_signed", "g_w[i] -= g_phi[q] * t[q] * fabs(v[i]);", "g_w[i] -= g_phi[q] * t[q] * v[i];",
     "test_parameter_gradients_against_finite_differences"),
    ("union_grad_of_last_part", "                    bi = i;\n                    memcpy(grad + q * n, g, sizeof(double) * (size_t)n);\n                }\n            }\n            phi[q] = best;\n            argmin[q] = bi;",
     "                    bi = i;\n                }\n                memcpy(grad + q * n, g, sizeof(double) * (size_t)n);\n            }\n            phi[q] = best;\n            argmin[q] = bi;",
     "test_union_min_rule"),
    ("maxH_grad_of_last_part", "                    bi = i;\n                    memcpy(grad + q * n, g, sizeof(double) * (size_t)n);\n                }\n            }\n            phi[q] = best;\n            argmax[q] = bi;",
     "                    bi = i;\n                }\n                memcpy(grad + q * n, g, sizeof(double) * (size_t)n);\n            }\n            phi[q] = best;\n            argmax[q] = bi;",
     "test_max_over_hamiltonians_solves_the_min_hamiltonian_pde"),
    ("control_diag_drops_A", "if (p->a_kind == ORC_A_DIAG) ap = p->A[i] * g[i];", "if (p->a_kind == ORC_A_DIAG) ap = g[i];",
     "test_control_is_a_subgradient_and_the_hopf_lax_minimiser"),
    ("shrink2_not_normalised", "out[i] = z[i] / nz * m;", "out[i] = z[i] * m;", "test_paper_example_sphere"),
    ("gx_drops_weight", "g_x[q * n + i] = g_phi[q] * v[i];", "g_x[q * n + i] = v[i];", "test_backward_diagonal_A_fd"),
    ("gc_sign", "g_c[i] -= g_phi[q] * v[i];", "g_c[i] += g_phi[q] * v[i];",
     "test_parameter_gradients_against_finite_differences"),
    ("jstar_l1_not_squared", "for (int i = 0; i < p->n; ++i) s += fabs(v[i]);\n        return s * s;",
     "for (int i = 0; i < p->n; ++i) s += fabs(v[i]);\n        return s;", "test_nonquadratic_initial_data_bruteforce_n2"),
    ("H_weights_ignored", "s += (h_kind == ORC_H_WL1 && w ? w[i] : 1.0) * fabs(q[i]);", "s += fabs(q[i]);",
     "test_weighted_l1_with_centre"),
    ("terminal_point_sign", "x_T[q * n + i] = xi - t[q] * b;", "x_T[q * n + i] = xi + t[q] * b;",
     "test_control_is_a_subgradient_and_the_hopf_lax_minimiser"),
    ("urel_not_relative", "ru = du / (un > 1.0 ? un : 1.0);", "ru = du;", "test_relative_stop_rule_exact_iterations"),
    ("urel_no_floor", "ru = du / (un > 1.0 ? un : 1.0);", "ru = du / un;",
     "test_relative_stop_rule_exact_iterations"),
    ("urel_previous_u_from_v", "double uold = d[i] + b[i];", "double uold = vprev[i] + b[i];",
     "test_relative_stop_rule_exact_iterations"),
    ("urel_norm_of_v", "un += u * u;", "un += v[i] * v[i];", "test_relative_stop_rule_exact_iterations"),
    ("cholesky_no_sqrt", "L[(int64_t)i * n + i] = sqrt(s);", "L[(int64_t)i * n + i] = s;",
     "test_dense_wl1_kkt_certificate"),
    ("forward_solve_transposed", "for (int k = 0; k < i; ++k) s -= L[(int64_t)i * n + k] * v[k];",
     "for (int k = 0; k < i; ++k) s -= L[(int64_t)k * n + i] * v[k];", "test_dense_wl1_kkt_certificate"),
    ("factor_inner_transposed", "s -= L[(int64_t)i * n + k] * L[(int64_t)j * n + k];",
     "s -= L[(int64_t)i * n + k] * L[(int64_t)k * n + j];", "test_dense_wl1_kkt_certificate"),
    ("solve_centre_dropped", "for (int i = 0; i < n; ++i) y[i] = x[i] - (p->c ? p->c[i] : 0.0);",
     "for (int i = 0; i < n; ++i) y[i] = x[i];", "test_weighted_l1_with_centre"),
    ("prox_argument_drops_b", "double u = v[i] + b[i];", "double u = v[i];", "test_workload1_closed_form"),
    ("dense_quad_diagonal_only", "for (int j = 0; j < p->n; ++j) r += p->A[(int64_t)i * p->n + j] * v[j];",
     "r += p->A[(int64_t)i * p->n + i] * v[i];", "test_dense_duality_gap"),
    ("l2_H_not_rooted", "for (int i = 0; i < n; ++i) s += q[i] * q[i];\n        return sqrt(s);",
     "for (int i = 0; i < n; ++i) s += q[i] * q[i];\n        return s;", "test_paper_example_sphere"),
    ("anorm_H_not_rooted", "return sqrt(s > 0.0 ? s : 0.0);", "return s > 0.0 ? s : 0.0;",
     "test_anorm_l2sq_initial_data_closed_form or test_anorm_bruteforce_n2"),
    ("gradient_negated", "for (int i = 0; i < n; ++i) grad[i] = d[i];", "for (int i = 0; i < n; ++i) grad[i] = -d[i];",
     "test_phi_convex_in_x_with_supporting_gradient"),
]


def _scratch_copy(dst):
    ign = shutil.ignore_patterns("_build", "__pycache__")
    for d in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d), ignore=ign)


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, pins):
    _scratch_copy(str(tmp_path))
    src = os.path.join(str(tmp_path), "oracle", "hopf_oracle.c")
    text = open(src).read()
    assert text.count(old) == 1, "the mutated text must occur exactly once in hopf_oracle.c"
    open(src, "w").write(text.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q", "-p",
                        "no:cacheprovider", "-k", pins], cwd=str(tmp_path), env=env, capture_output=True,
                       text=True, timeout=600)
    # exit code 1: tests ran and at least one failed (2-5 would be an
    # interruption, an internal error, a usage error or no test selected)
    assert r.returncode == 1, "%s: pins %r did not fail (exit %d)\n%s" % (name, pins, r.returncode,
                                                                             r.stdout[-1500:])
    assert " failed" in r.stdout.splitlines()[-1]
