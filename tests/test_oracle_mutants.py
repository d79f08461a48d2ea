"""Planted mistakes: every plausible slip in the oracle must fail a pin.

Each case applies one textual mutation to a temporary copy of
oracle/amgd_oracle.c (a dropped term, a wrong sign, a wrong index, a swapped
operand, a non-strict comparison ...), compiles it with gcc on the CPU and
runs all pins of test_oracle_pins.py against it.  The committed oracle is
never touched.
"""
import os

import pytest

import oracle
import test_oracle_adjoint as adj
import test_oracle_cr as cr
import test_oracle_graph as graph
import test_oracle_interp as interp
import test_oracle_pins as pins

PINS = [pins.pin_philox_numpy, pins.pin_tv_init, pins.pin_jacobi_dense_power,
        pins.pin_mcgs_proper_coloring_is_gauss_seidel, pins.pin_mcgs_snapshot_matrix_form,
        pins.pin_target, pins.pin_ls_lstsq, pins.pin_ls_brute_force, pins.pin_ls_invariants,
        pins.pin_ls_exact_cases, pins.pin_integer_weights_repeat_vectors,
        pins.pin_degree_one_rows, pins.pin_threshold,
        pins.pin_strength_csr, adj.pin_adjoint_fd, adj.pin_adjoint_homogeneity,
        adj.pin_adjoint_special_cases, graph.pin_distance_graph_matrix_power,
        graph.pin_edge_ls_graph, interp.pin_interp_brute_force, interp.pin_interp_single_point,
        interp.pin_interp_monotone_and_exact, cr.pin_cr_stage_brute_force,
        cr.pin_cr_spectral_limit, cr.pin_cr_red_black_closed_form, cr.pin_cr_special_cases]

# (name, text to find, replacement, occurrence index)
MUTANTS = [
    ("philox_hi_lo_swapped", "uint64_t n1 = lo1;", "uint64_t n1 = hi1;", 0),
    ("philox_key_not_bumped", "k1 += W1;", "k1 += 0;", 0),
    ("philox_wrong_multiplier_input", "orc_mulhilo64(M1, c2,", "orc_mulhilo64(M1, c1,", 0),
    ("tv_map_halves_swapped", "(kappa % 2 == 0) ?", "(kappa % 2 == 1) ?", 0),
    ("tv_map_wrong_word", "out[(kappa / 2) % 4]", "out[(kappa / 2 + 1) % 4]", 0),
    ("tv_map_not_centred", "((double)(2 * m + 1))", "((double)(2 * m))", 0),
    ("jacobi_sign", "Xn[i * K + kappa] = fma(-c, s,", "Xn[i * K + kappa] = fma(c, s,", 0),
    ("jacobi_drops_diagonal", "s = fma(val[p], X[(int64_t)col[p] * K + kappa], s);",
     "if (col[p] != i) s = fma(val[p], X[(int64_t)col[p] * K + kappa], s);", 0),
    ("jacobi_wrong_row", "s = fma(val[p], X[(int64_t)col[p] * K + kappa], s);",
     "s = fma(val[p], X[i * K + kappa], s);", 0),
    ("jacobi_ignores_omega", "double c = omega / orc_diag", "double c = 1.0 / orc_diag", 0),
    ("mcgs_same_color_new", "(color[j] < c) ?", "(color[j] <= c) ?", 0),
    ("mcgs_all_old", "(color[j] < c) ?", "(0) ?", 0),
    ("mcgs_ignores_omega", "double ci = omega / orc_diag", "double ci = 1.0 / orc_diag", 0),
    ("target_modes_swapped", "if (mode == 1) {", "if (mode == 0) {", 0),
    ("ls_sxx_uses_y", "sxx += w[kappa] * x[kappa] * x[kappa];",
     "sxx += w[kappa] * y[kappa] * y[kappa];", 0),
    ("ls_unweighted_residual", "res += w[kappa] * e * e;", "res += e * e;", 0),
    ("ls_residual_sign", "double e = y[kappa] - pij * x[kappa];",
     "double e = y[kappa] + pij * x[kappa];", 0),
    ("ls_transposed_roles", "const double *y = Y + i * K;", "const double *y = Y + j * K;", 0),
    ("degree_one_sign", "a[p] = -val[p] / aii;", "a[p] = val[p] / aii;", 0),
    ("threshold_not_strict", "(theta * ls[p] < m)", "(theta * ls[p] <= m)", 0),
    ("threshold_uses_max", "if (col[p] != i && ls[p] < m) m = ls[p];",
     "if (col[p] != i && (m == INFINITY || ls[p] > m)) m = ls[p];", 0),
    ("threshold_counts_diagonal", "strong = (ls[p] == 0.0) || (theta * ls[p] < m);",
     "strong = (ls[p] == 0.0) || (theta * ls[p] < m); else strong = 1;", 0),
    ("csr_writes_slot_not_column", "if (flag[p]) s_col[k++] = col[p];",
     "if (flag[p]) s_col[k++] = (int32_t)(p - rp[i]);", 0),
    ("adj_drops_target_diagonal", "val_bar[pd] += yr / (aii * aii);", "val_bar[pd] += 0.0 * yr;", 0),
    ("adj_drops_sweep_diagonal", "val_bar[pd] += omega * xr / (aii * aii);",
     "val_bar[pd] += 0.0 * xr;", 0),
    ("adj_omega_sign", "wbar -= xr / aii;", "wbar += xr / aii;", 0),
    ("adj_ybar_missing_two", "Ybar[i * K + kappa] += lsb[p] * 2.0 * w[kappa] * e;",
     "Ybar[i * K + kappa] += lsb[p] * w[kappa] * e;", 0),
    ("adj_envelope_sign", "Xbar[j * K + kappa] += -lsb[p] * 2.0 * w[kappa] * a[p] * e;",
     "Xbar[j * K + kappa] += lsb[p] * 2.0 * w[kappa] * a[p] * e;", 0),
    ("adj_not_transposed", "Xbar[j * K + kappa] -= omega * (val[p] / aii) * Xnext[i * K + kappa];",
     "Xbar[i * K + kappa] -= omega * (val[p] / aii) * Xnext[j * K + kappa];", 0),
    ("adj_uses_later_iterate", "const double *Xc = Xs + (size_t)s * nk;",
     "const double *Xc = Xs + (size_t)(s + 1) * nk;", 0),
    ("adj_loss_power", "lsb[p] = -2.0 / (ls[p] * ls[p] * ls[p]);",
     "lsb[p] = -1.0 / (ls[p] * ls[p] * ls[p]);", 0),
    ("graph_depth_short", "for (int32_t step = 0; step < d; ++step)",
     "for (int32_t step = 1; step < d; ++step)", 0),
    ("graph_unsorted", "qsort(list, (size_t)len, sizeof(int32_t), orc_cmp_i32);", ";", 0),
    ("graph_no_self", "list[len++] = (int32_t)i;", ";", 0),
    ("graph_exact_rule_any_neighbour", "if (mode == 0 && off == 1 && j == col[p1]) {",
     "if (mode == 0 && off == 1) {", 0),
    ("graph_target_from_x", "const double *y = Y + i * K;", "const double *y = X + i * K;", 1),
    ("interp_penalty_absolute", "pow(cur, gamma * (double)(m - chosen))",
     "pow(cur, gamma * (double)m)", 0),
    ("interp_not_normalised", "if (bestls[m] / syy < pow(cur,", "if (bestls[m] < pow(cur,", 0),
    ("interp_ties_last", "if (!have[m] || res < bestls[m]) {", "if (!have[m] || res <= bestls[m]) {", 0),
    ("interp_residual_sign", "for (int a = 0; a < m; ++a) e -= p[a] * X[", "for (int a = 0; a < m; ++a) e += p[a] * X[", 0),
    ("interp_gram_unweighted", "for (int32_t k = 0; k < K; ++k) g += w[k] * xa[k] * xb[k];",
     "for (int32_t k = 0; k < K; ++k) g += xa[k] * xb[k];", 0),
    ("interp_fine_candidates", "if (coarse[pcol[q]]) cand[nc++] = pcol[q];",
     "if (pcol[q] != i) cand[nc++] = pcol[q];", 0),
    ("cr_coarse_rows_relaxed", "if (coarse[i]) { un[i] = 0.0; continue; }",
     "if (coarse[i] && 0) { un[i] = 0.0; continue; }", 0),
    ("cr_sor_ignores_omega", "acc = fma(val[p], color[j] < cc ? un[j] : u[j], acc);\n                        }\n                        un[i] = fma(-c, acc, u[i]);",
     "acc = fma(val[p], color[j] < cc ? un[j] : u[j], acc);\n                        }\n                        un[i] = fma(-c / omega, acc, u[i]);", 0),
    ("cr_rho_no_root", "pow(unorm, 1.0 / (double)nu)", "unorm", 0),
    ("cr_candidates_signed", "fabs(u[i]) / unorm > tol", "u[i] / unorm > tol", 0),
    ("cr_min_over_all_neighbours", "if (j != i && !coarse[j] && ls[q] < m) m = ls[q];",
     "if (j != i && ls[q] < m) m = ls[q];", 0),
    ("cr_lambda_out_degree", "if (strong[q] && inz[pcol[q]]) ++lam[pcol[q]];",
     "if (strong[q] && inz[pcol[q]]) ++lam[j];", 0),
    ("cr_priority_reversed", "if (la != lb) return la > lb;", "if (la != lb) return la < lb;", 0),
    ("cr_key_wrong_word", "key[i] = out[0];", "key[i] = out[1];", 0),
    ("cr_key_no_stage", "uint64_t ctr[4] = {(uint64_t)i, (uint64_t)stage, 1, 0};",
     "uint64_t ctr[4] = {(uint64_t)i, 0, 1, 0};", 0),
    ("cr_ignores_in_edges", "if (inset[tsrc[e]]) blocked = 1;", "if (0) blocked = 1;", 0),
    ("cr_not_restarted", "u[i] = coarse[i] ? 0.0 : 1.0;", "u[i] = coarse[i] ? 0.0 : (stage ? u[i] : 1.0);", 0),
    ("adj_weights_dropped", "Xbar[j * K + kappa] += -lsb[p] * 2.0 * w[kappa] * a[p] * e;",
     "Xbar[j * K + kappa] += -lsb[p] * 2.0 * a[p] * e;", 0),
    ("ls_syx_unweighted", "syx += w[kappa] * y[kappa] * x[kappa];",
     "syx += y[kappa] * x[kappa];", 0),
    ("ls_sxx_unweighted", "sxx += w[kappa] * x[kappa] * x[kappa];",
     "sxx += x[kappa] * x[kappa];", 0),
    ("graph_syx_unweighted", "syx += w[kappa] * y[kappa] * x[kappa];",
     "syx += y[kappa] * x[kappa];", 1),
]


def _mutate(text, find, repl, occ):
    pos = -1
    for _ in range(occ + 1):
        pos = text.index(find, pos + 1)
    return text[:pos] + repl + text[pos + len(find):]


@pytest.mark.parametrize("name,find,repl,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, find, repl, occ):
    src = oracle.source_text()
    assert find in src, "mutation anchor missing: %s" % name
    mutant = oracle.compile_variant(_mutate(src, find, repl, occ),
                                    os.path.join(str(tmp_path), "liborc_%s.so" % name))
    caught = []
    for pin in PINS:
        try:
            pin(mutant)
        except Exception:          # a failed assertion, or a pin that cannot even run
            caught.append(pin.__name__)
    assert caught, "planted mistake %r passed every pin" % name
