"""Sensitivity of the oracle's pins: a plausible mistake planted anywhere in the
oracle must make at least one pin fail.

Each mutant is a copy of one oracle routine with one change a careful author
could still make: a dropped term, a flipped sign, the wrong endpoint's degree,
a transposed operand, an off-by-one length, a lost factor. The copy is built
on the CPU (the C routines compiled into a scratch library, the Python modules
executed from edited source) and swapped in for the duration of one test; the
oracle on disk is never touched. The pins are the existing pin tests, called
with fixed arguments. Only changes to what the paper or the mathematics fixes
are planted: conventions of this implementation that the paper leaves open
(which Philox counter feeds which walk) are pinned by the GPU tests' bit-exact
comparison, not here. A control runs every battery on the unmodified oracle
first, so that a battery cannot "kill" a mutant by being broken itself, and
only the failures a wrong value causes count as kills (an assertion, or the
oracle's own error for an impossible state), not a typo in the mutation.
CPU only.
"""
from __future__ import annotations

import inspect
import os
import sys
import types

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import _native, exact, learned, meet, philox, series, tgtplus, truncation

import test_oracle_caltau as tc
import test_oracle_exact as te
import test_oracle_learned as tl
import test_oracle_meet as tm
import test_oracle_series as ts
import test_oracle_tgtplus as tt

KILLS = (AssertionError, RuntimeError, ValueError, FloatingPointError, np.linalg.LinAlgError,
         ZeroDivisionError, OverflowError)

# ---------------------------------------------------------------- batteries

SERIES = [
    ("K_n closed form", lambda: ts.test_complete_graph_closed_form(5, 3)),
    ("C_n closed form", lambda: ts.test_cycle_closed_form(9, 5)),
    ("exact rational series, lollipop", lambda: ts.test_matches_exact_rational_series(lambda: gg.lollipop(4, 2), 3)),
    ("exact rational series, tree + G(n,p)",
     lambda: ts.test_matches_exact_rational_series(lambda: gg.tree_plus_gnp(7, 3.0, 1), 6)),
    ("odd-tau lower bound, monotone", lambda: ts.test_odd_tau_lower_bound_and_monotone(0)),
    ("bipartite 1/m bias, end correction", lambda: ts.test_bipartite_bias_and_end_correction(8)),
    ("end-corrected grid bounds", ts.test_end_corrected_grid_lower_bound_and_tail_bound),
    ("plain tail bound", lambda: ts.test_plain_tail_bound(0)),
    ("Theorem 3.2 guarantee", lambda: ts.test_theorem_3_2_eps_guarantee(1e-2, 0)),
    ("per-entry lengths", ts.test_per_entry_lengths_match_global_runs),
    ("tail bounds tight", ts.test_tail_bounds_are_tight_at_large_tau),
]

TRUNCATION = [
    ("least odd length", ts.test_tau_is_smallest_odd_meeting_the_bound),
    ("Theorem 3.2 guarantee", lambda: ts.test_theorem_3_2_eps_guarantee(1e-3, 1)),
    ("C_n spectrum", lambda: ts.test_spectrum_cycle(8)),
    ("named spectra", ts.test_spectrum_named),
    ("ARPACK vs dense", ts.test_spectrum_sparse_path_matches_dense),
]

EXACT = [
    ("enumeration = matrix tree = dense", lambda: te.test_kirchhoff_matches_matrix_tree_and_dense(te.SMALL[4])),
    ("golden fractions", te.test_golden_fractions),
    ("K_a,b closed form", lambda: te.test_complete_bipartite_closed_form(2, 3)),
    ("bridges", te.test_bridges_are_one),
    ("Foster", lambda: te.test_foster_random(0)),
    ("CG and LU vs dense", lambda: te.test_cg_and_sparse_lu_match_dense(lambda: gg.tree_plus_gnp(300, 6.0, 5))),
    ("blocked CG vs dense and single solves",
     lambda: te.test_blocked_cg_matches_dense_and_single_solves(gg.barabasi_albert(3000, 4, 9))),
]

TGTPLUS = [
    ("Philox known answers", tt.test_philox_known_answers),
    ("uniform index ends", tt.test_uniform_index_range_and_ends),
    ("Lemma 4.1, unbiased walks", tt.test_lemma_4_1_and_unbiased_walk_estimator),
    ("Lemma 4.3 by enumeration", lambda: tt.test_lemma_4_3_bounds_by_enumeration(0, 2)),
    ("rho_hat bound", tt.test_rho_hat_upper_bound_and_literal_counterexample),
    ("Eq. 15", tt.test_eq15_gamma_zero),
    ("Eq. 13 Hoeffding", tt.test_walk_count_formula_and_hoeffding),
    ("TGT+ within eps", tt.test_full_tgt_plus_within_eps_on_small_graph),
    ("frontier = degree of the exact reach", lambda: tt.test_frontier_volume_is_the_degree_of_the_exact_reach(
        lambda: gg.lollipop(6, 4))),
    ("per-source switch", tt.test_per_source_switch_is_the_first_hop_where_eq14_holds),
    ("even-hop bound vs the exact tail",
     lambda: tt.test_even_hop_bound_holds_against_the_exact_tail(lambda: gg.barbell(6, 2))),
    ("learned TGT+ at the cap", tt.test_learned_tgt_plus_at_the_cap_is_per_source_tgt_plus),
    ("learned TGT+ extends short lengths", lambda: tt.test_learned_tgt_plus_extends_short_lengths_and_meets_eps(1)),
]

LEARNED = [
    ("features on named graphs", tl.test_features_on_named_graphs),
    ("features by hand", tl.test_features_by_hand_on_lollipop),
    ("features independent of the size", tl.test_features_do_not_depend_on_the_graph_size),
    ("p2 feature = P^2", lambda: tl.test_p2_feature_is_two_step_return_probability(0)),
    ("hop terms vs powers", tl.test_hop_terms_match_series_and_powers),
    ("certified lengths", lambda: tl.test_certified_lengths(lambda: gg.tree_plus_gnp(500, 8.0, 2), 1e-2)),
    ("gradient vs finite differences", tl.test_mlp_gradient_matches_finite_differences),
    ("Adam first step", tl.test_adam_first_step_closed_form),
    ("odd prediction with slack", tl.test_prediction_rounds_to_an_odd_length_with_a_quarter_slack),
    ("tail estimate sums a power law", lambda: tl.test_tail_estimate_sums_a_power_law(2.0, 11)),
    ("tail estimate overshoots a geometric tail", lambda: tl.test_tail_estimate_overshoots_a_geometric_tail(0.5, 11)),
    ("tail estimate special cases", tl.test_tail_estimate_special_cases),
    ("tail estimate on a lattice", tl.test_tail_estimate_on_a_perturbed_lattice),
    ("estimated lengths, two routes", tl.test_estimated_lengths_two_routes),
    ("bipartite extension loop", tl.test_learned_bipartite_within_eps),
]

CALTAU = [
    ("eigenpairs reproduce Eq. 2", lambda: tc.test_eigenpairs_reproduce_the_series_terms(lambda: gg.lollipop(5, 3))),
    ("omega = 2 is Eq. 6", lambda: tc.test_omega_two_is_eq6(lambda: gg.lollipop(8, 3), 1e-2)),
    ("bound exact at omega = n", lambda: tc.test_bound_is_the_exact_tail_with_every_eigenpair(
        lambda: gg.tree_plus_gnp(40, 4.0, 3))),
    ("bound holds from t", lambda: tc.test_bound_holds_for_every_odd_tau_from_t(5)),
    ("Theorem 3.2, bottleneck", lambda: tc.test_theorem_3_2_with_caltau(lambda: gg.barbell(12, 1), 1e-2)),
    ("Theorem 3.2, G(n,p)", lambda: tc.test_theorem_3_2_with_caltau(lambda: gg.gnp_lcc(200, 5.0, 2), 1e-3)),
    ("bottleneck", tc.test_bottleneck_needs_far_fewer_hops),
    ("direct search", lambda: tc.test_caltau_matches_a_direct_search(lambda: gg.lollipop(8, 3), 3)),
    ("remainder form, leading mode left out", lambda: tc.test_remainder_form_matches_a_direct_search(
        lambda: gg.lollipop(8, 3), [2])),
    ("remainder form, a gap", lambda: tc.test_remainder_form_matches_a_direct_search(
        lambda: gg.barbell(6, 1), [1, 3, 4])),
]

MEET = [
    ("equals Algorithm 2, lollipop", lambda: tm.test_equals_algorithm_2_at_per_entry_lengths(lambda: gg.lollipop(7, 4))),
    ("K_n closed form", lambda: tm.test_complete_graph_closed_form(7)),
    ("matrix powers, even terms", tm.test_terms_equal_matrix_powers_and_even_terms_are_non_negative),
]

BATTERIES = {"series": SERIES, "truncation": TRUNCATION, "exact": EXACT, "tgtplus": TGTPLUS, "meet": MEET,
             "learned": LEARNED, "caltau": CALTAU}


def _first_kill(battery):
    """Name of the first pin that fails, else None."""
    for name, fn in battery:
        try:
            fn()
        except KILLS:
            return name
    return None


# ---------------------------------------------------------------- mutants
# (id, target, battery, old text, new text); target "c" edits oracle/csrc/oracle.c,
# otherwise the named oracle module. The old text must occur exactly once.

C_MUTANTS = [
    ("blocked CG: a converged column keeps iterating", "exact",
     "alpha[c] = active[c] ? rz[c] / pq[c] : 0.0;", "alpha[c] = rz[c] / pq[c];"),
    ("blocked CG: the Laplacian product adds the neighbours", "exact",
     "for (int c = 0; c < CG_W; ++c) acc[c] -= pj[c];", "for (int c = 0; c < CG_W; ++c) acc[c] += pj[c];"),
    ("hop term sign", "series",
     "const double term = p_next[i] / d_i - p_next[j] / d_i;",
     "const double term = p_next[j] / d_i - p_next[i] / d_i;"),
    ("neighbour term over d_j", "series",
     "const double term = p_next[i] / d_i - p_next[j] / d_i;",
     "const double term = p_next[i] / d_i - p_next[j] / (double)(row_ptr[j + 1] - row_ptr[j]);"),
    ("hop 0 dropped", "series",
     "g_out[k] = 1.0 / d_i;",
     "g_out[k] = 0.0;"),
    ("one hop short", "series",
     "if (l <= tau[k]) g_out[k] += term;",
     "if (l < tau[k]) g_out[k] += term;"),
    ("one hop long", "series",
     "if (l <= tau[k]) g_out[k] += term;",
     "if (l <= tau[k] + 1) g_out[k] += term;"),
    ("push over the sender's degree (P transposed)", "series",
     "p_next[x] += pj / d_x;",
     "p_next[x] += pj / (double)(row_ptr[j + 1] - row_ptr[j]);"),
    ("source length = min over its edges", "series",
     "if (tau[k] > tau_p) tau_p = tau[k];",
     "if (k == k0 || tau[k] < tau_p) tau_p = tau[k];"),
    ("first omitted term taken one hop late", "series",
     "else if (l == tau[k] + 1) { if (t1_out) t1_out[k] = term; }",
     "else if (l == tau[k] + 2) { if (t1_out) t1_out[k] = term; }"),
    ("resistance read as x_u + x_v", "exact",
     "r_out[t] = x[a] - x[b];",
     "r_out[t] = x[a] + x[b];"),
    ("signless Laplacian", "exact",
     "acc -= x[col_idx[e]];",
     "acc += x[col_idx[e]];"),
    ("per-hop term sign", "learned",
     "= p_next[i] / d_i - p_next[col_idx[k]] / d_i;",
     "= p_next[col_idx[k]] / d_i - p_next[i] / d_i;"),
    ("per-hop terms from hop 1 on", "learned",
     "o[(int64_t)(k - k0) * (L + 1)] = 1.0 / d_i;",
     "o[(int64_t)(k - k0) * (L + 1)] = 0.0;"),
]

PY_MUTANTS = [
    # series.py
    ("series", "halves: g(i,j) twice", "series", "s = g + g[rev]", "s = g + g"),
    ("series", "end correction: whole term", "series", "s = s + 0.5 * tf1", "s = s + tf1"),
    ("series", "end-corrected bound without the 2", "series",
     "return q / (2.0 * (1.0 - lam_plus))", "return q / (1.0 - lam_plus)"),
    ("series", "plain bound over 1 - lambda", "series",
     "return q / (1.0 - lam_star * lam_star)", "return q / (1.0 - lam_star)"),
    # truncation.py
    ("truncation", "Eq. 6 without the -1", "truncation",
     "(1.0 - lam * lam))) / math.log(1.0 / lam) - 1.0", "(1.0 - lam * lam))) / math.log(1.0 / lam)"),
    ("truncation", "Eq. 6 over 1 - lambda", "truncation",
     "(eps * (1.0 - lam * lam))", "(eps * (1.0 - lam))"),
    ("truncation", "X_e sign", "truncation",
     "d_j = np.asarray(d_j, dtype=np.float64)\n    x_e = 1.0 / d_i + 1.0 / d_j - 2.0 / (d_i * d_j)",
     "d_j = np.asarray(d_j, dtype=np.float64)\n    x_e = 1.0 / d_i + 1.0 / d_j + 2.0 / (d_i * d_j)"),
    ("truncation", "rounded to even", "truncation",
     "np.where(t % 2 == 0, t + 1, t)", "np.where(t % 2 == 1, t + 1, t)"),
    ("truncation", "lambda_plus = 1 (trivial mode kept)", "truncation",
     "lam_plus = float(w[-2])", "lam_plus = float(w[-1])"),
    ("truncation", "lambda_star without the modulus", "truncation",
     "lam_star = max(abs(lam_plus), abs(lam_minus))", "lam_star = max(lam_plus, lam_minus)"),
    ("truncation", "ARPACK: lambda_minus from the wrong end", "truncation",
     'which="SA"', 'which="LA"'),
    # truncation.py: CalTau with omega eigenpairs (Algorithm 1, Eq. 6-8)
    ("truncation", "eigenvalues sorted by value", "caltau",
     "order = np.lexsort((-w, -np.abs(w)))[:omega]", "order = np.argsort(-w)[:omega]"),
    ("truncation", "f_k without sqrt(2m)", "caltau",
     "F = np.sqrt(deg.sum()) * (vec[:, order]", "F = (vec[:, order]"),
    ("truncation", "Eq. 7 without 1 + lambda", "caltau",
     "ups = ((1.0 + mid) @ c) / two_m", "ups = (np.ones_like(mid) @ c) / two_m"),
    ("truncation", "Eq. 8 at lambda^t", "caltau",
     "delta = ((mid ** (t + 1) / (1.0 - mid)) @ c[:, idx]) / two_m",
     "delta = ((mid ** t / (1.0 - mid)) @ c[:, idx]) / two_m"),
    ("truncation", "Eq. 8 over 1 + lambda", "caltau",
     "delta = ((mid ** (t + 1) / (1.0 - mid)) @ c[:, idx]) / two_m",
     "delta = ((mid ** (t + 1) / (1.0 + mid)) @ c[:, idx]) / two_m"),
    ("truncation", "lambda_omega one place early", "caltau",
     "lam_w = abs(lam[omega - 1])", "lam_w = abs(lam[omega - 2])"),
    ("truncation", "spent budget read as nothing left", "caltau",
     "spent = (budget < 0.0) | (~none_left & (budget == 0.0))", "spent = ~none_left & (budget <= 0.0)"),
    ("truncation", "CalTau returns the previous t", "caltau",
     "out[idx[stop]] = t\n", "out[idx[stop]] = t - 2\n"),
    ("truncation", "X_e sign in CalTau", "caltau",
     "d_i, d_j = deg[rows], deg[cols]\n    x_e = 1.0 / d_i + 1.0 / d_j - 2.0 / (d_i * d_j)",
     "d_i, d_j = deg[rows], deg[cols]\n    x_e = 1.0 / d_i + 1.0 / d_j + 2.0 / (d_i * d_j)"),
    ("truncation", "remainder modulus from the last given pair", "caltau",
     "lam = np.append(lam, float(lam_rest))", "lam = np.append(lam, float(abs(lam[-1])))"),
    ("truncation", "lambda_star from the first given pair", "caltau",
     "lam_top = float(np.max(np.abs(lam[1:])))", "lam_top = float(abs(lam[1]))"),
    # tgtplus.py: Algorithm 4's per-source switch (Eq. 14)
    ("tgtplus", "Eq. 14's walks at the full length", "tgtplus",
     "            L = int(tau_row[t]) - ell\n            if L > 0:\n                rhs +=",
     "            L = int(tau_row[t])\n            if L > 0:\n                rhs +="),
    ("tgtplus", "frontier counts nodes, not degrees", "tgtplus", "return int(deg[p != 0].sum())",
     "return int((p != 0).sum())"),
    # meet.py
    ("meet", "odd hop split as a + a", "meet", "        b = ell - a\n", "        b = a\n"),
    ("meet", "inner product without D^-1", "meet",
     "np.sum(U[a] * U[b] / deg[None, :], axis=1)", "np.sum(U[a] * U[b], axis=1)"),
    ("meet", "u from one endpoint", "meet", "U = [Rh[rows] - Rh[cols] for Rh in R]", "U = [Rh[rows] for Rh in R]"),
    ("meet", "columns of P^h for distributions", "meet", "U = [Rh[rows] - Rh[cols] for Rh in R]",
     "U = [(Rh[:, rows] - Rh[:, cols]).T for Rh in R]"),
    # exact.py
    ("exact", "resistance without the cross factor 2", "exact",
     "dg[rows] + dg[cols] - 2.0 * m[rows, cols]", "dg[rows] + dg[cols] - m[rows, cols]"),
    ("exact", "grounding deletes the first row, the last column", "exact",
     "return lap[:-1, :-1]", "return lap[1:, :-1]"),
    ("exact", "enumeration counts cyclic subsets", "exact",
     "continue  # n-1 acyclic edges on n nodes always span", "pass"),
    ("exact", "matrix tree: T(G-e)/T(G) itself", "exact",
     "out[e] = 1 - Fraction(_spanning_tree_count(n, rest), total)",
     "out[e] = Fraction(_spanning_tree_count(n, rest), total)"),
    ("exact", "sparse LU: x_u + x_v", "exact",
     "out[s:s + chunk] = x[pp[:, 0], cols] - x[pp[:, 1], cols]",
     "out[s:s + chunk] = x[pp[:, 0], cols] + x[pp[:, 1], cols]"),
    ("exact", "sparse LU: a mis-grounded matrix", "exact",
     "grounded = lap[:-1, :-1]  # node n-1 deleted", "grounded = lap[1:, :-1]  # node n-1 deleted"),

    # philox.py
    ("philox", "Philox words swapped", "tgtplus",
     "c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]", "c = [hi0 ^ c[1] ^ k0, lo0, hi1 ^ c[3] ^ k1, lo1]"),
    ("philox", "Philox key not advanced", "tgtplus", "k1 = k1 + W1", "k1 = k1"),
    ("philox", "neighbour index by modulo", "tgtplus",
     "return ((np.asarray(u32, dtype=np.uint64) * np.asarray(d, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)",
     "return (np.asarray(u32, dtype=np.uint64) % np.asarray(d, dtype=np.uint64)).astype(np.int64)"),
    # tgtplus.py
    ("tgtplus", "LB with L terms of min p", "tgtplus",
     "lb = nb.min() + (L - 1) * p.min()", "lb = nb.min() + L * p.min()"),
    ("tgtplus", "UB with L - 2 terms of rho", "tgtplus",
     "(L - 1) * rho / 2.0", "(L - 2) * rho / 2.0"),
    ("tgtplus", "UB without the halving", "tgtplus",
     "ub = nb.max() / 2.0 + p.max() / 2.0", "ub = nb.max() / 2.0 + p.max() / 4.0"),
    ("tgtplus", "rho_hat as printed (edges inside C only)", "tgtplus",
     "    return max(best, two)", "    return best if best > -np.inf else two"),
    ("tgtplus", "candidates = smallest entries", "tgtplus",
     "order = np.lexsort((np.arange(p.size), -p))", "order = np.lexsort((np.arange(p.size), p))"),
    ("tgtplus", "Eq. 13 constant 4", "tgtplus",
     "r = 8.0 * chi * chi", "r = 4.0 * chi * chi"),
    ("tgtplus", "Eq. 13 union bound over m / delta", "tgtplus",
     "math.log(2.0 * m / delta)", "math.log(m / delta)"),
    ("tgtplus", "walk counts its start node", "tgtplus",
     "        cur = col_idx[row_ptr[cur] + idx]\n        total += p[cur]\n",
     "        total += p[cur]\n        cur = col_idx[row_ptr[cur] + idx]\n"),
    ("tgtplus", "walk estimate sign", "tgtplus",
     "return float(np.mean(si - sj))", "return float(np.mean(sj - si))"),
    ("tgtplus", "source column pushed over the sender's degree", "tgtplus",
     "            q[nb] += p[v] / deg[nb]\n        p = q\n    return p",
     "            q[nb] += p[v] / deg[v]\n        p = q\n    return p"),
    ("tgtplus", "even-hop bound one power of lambda too many", "tgtplus",
     "    for _ in range(tau + 1 - ell):\n        f *= lam_star", "    for _ in range(tau + 2 - ell):\n        f *= lam_star"),
    ("tgtplus", "even-hop bound over 1 - lambda^2", "tgtplus",
     "    return f / (1.0 - lam_star) * t_l", "    return f / (1.0 - lam_star * lam_star) * t_l"),
    ("tgtplus", "Eq. 15 without the factor L", "tgtplus",
     "return 2.0 * L * (p.max() - p.min())", "return 2.0 * (p.max() - p.min())"),
    # learned.py
    ("learned", "triangles counted twice", "learned", "        tri //= 2", "        tri //= 1"),
    ("learned", "largest neighbour degree", "learned",
     "F[i, 1] = math.log(deg[nb].min())", "F[i, 1] = math.log(deg[nb].max())"),
    ("learned", "p2 feature without 1/d_i", "learned",
     "F[i, 4] = np.sum(1.0 / deg[nb]) / d", "F[i, 4] = np.sum(1.0 / deg[nb])"),
    ("learned", "neighbour degree feature not per neighbour", "learned",
     "F[i, 3] = math.log(deg[nb].sum() / d / mean_deg)", "F[i, 3] = math.log(deg[nb].sum() / mean_deg)"),
    ("learned", "p3 feature with the closing node's degree twice", "learned",
     "cyc += 1.0 / (deg[j] * deg[y])", "cyc += 1.0 / (deg[y] * deg[y])"),
    ("learned", "p3 feature without 1/d_i", "learned", "F[i, 5] = cyc / d", "F[i, 5] = cyc"),
    ("learned", "backprop through W2 transposed", "learned",
     "dh1 = (dh2 @ W2) * (z1 > 0)", "dh1 = (dh2 @ W2.T) * (z1 > 0)"),
    ("learned", "ReLU gate of layer 2 dropped", "learned",
     "dh2 = np.outer(dy, W3) * (z2 > 0)", "dh2 = np.outer(dy, W3)"),
    ("learned", "Adam without bias correction", "learned",
     "mhat = m / (1 - b1 ** t)", "mhat = m"),
    ("learned", "prediction rounded up without slack", "learned",
     "e = np.ceil(np.exp(y) - 0.25)", "e = np.ceil(np.exp(y))"),
    ("learned", "certificate from one term", "learned",
     "(factor * (full[:, t - 1] + full[:, t]) <= eps)", "(factor * full[:, t] <= eps)"),
    ("learned", "tail estimate without the half unit per hop", "learned",
     "/ (2.0 * (pd - 1.0))", "/ (pd - 1.0)"),
    ("learned", "power fitted over abscissae tau - 2, tau", "learned",
     "np.log((x + 1.0) / (x - 1.0))", "np.log(x / (x - 2.0))"),
    ("learned", "tail estimate zero where nothing decays", "learned",
     "    dec = p > 1.0\n", "    dec = p > 0.0\n"),
    ("learned", "labels from the pair after tau", "learned",
     "est = tail_estimate(full[:, t - 1] + full[:, t], full[:, t + 1] + full[:, t + 2], t)",
     "est = tail_estimate(full[:, t + 1] + full[:, t + 2], full[:, t + 1] + full[:, t + 2], t)"),
    ("learned", "extension loop fits one pair twice", "learned",
     "np.maximum(tau - 2, 0), end_corrected=True)", "tau, end_corrected=True)"),
    ("learned", "extension loop plain estimator", "learned",
     "s, q = series.series_entries(n, row_ptr, col_idx, tau, end_corrected=True)",
     "s, q = series.series_entries(n, row_ptr, col_idx, tau, end_corrected=False)"),
]


# ---------------------------------------------------------------- machinery

def _edit(src, old, new):
    assert src.count(old) == 1, f"mutation anchor must occur once: {old!r}"
    return src.replace(old, new)


def _swap_module(monkeypatch, orig, mutant):
    """Point every loaded oracle and test module at the mutant: module globals
    bound to ``orig`` and functions imported from it by name."""
    monkeypatch.setitem(sys.modules, orig.__name__, mutant)
    monkeypatch.setattr(oracle, orig.__name__.rsplit(".", 1)[1], mutant)
    for mod in list(sys.modules.values()):
        name = getattr(mod, "__name__", "")
        if mod is mutant or not (name.startswith("oracle") or name.startswith("test_")):
            continue
        for k, v in list(vars(mod).items()):
            if v is orig:
                monkeypatch.setattr(mod, k, mutant)
            elif callable(v) and getattr(v, "__module__", None) == orig.__name__ and getattr(orig, k, None) is v:
                monkeypatch.setattr(mod, k, getattr(mutant, k))


def _py_mutant(orig, old, new):
    src = _edit(inspect.getsource(orig), old, new)
    mod = types.ModuleType(orig.__name__)
    mod.__file__ = orig.__file__
    mod.__package__ = "oracle"
    exec(compile(src, orig.__file__, "exec"), mod.__dict__)
    return mod


@pytest.fixture(scope="module")
def c_source():
    with open(os.path.join(os.path.dirname(oracle.__file__), "csrc", "oracle.c")) as fh:
        return fh.read()


@pytest.mark.parametrize("battery", sorted(BATTERIES))
def test_control_batteries_pass_on_the_oracle(battery):
    assert _first_kill(BATTERIES[battery]) is None


@pytest.mark.parametrize("mid,battery,old,new", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_killed(mid, battery, old, new, c_source, tmp_path, monkeypatch):
    src = tmp_path / "oracle_mutant.c"
    src.write_text(_edit(c_source, old, new))
    so = str(tmp_path / "liboracle_mutant.so")
    _native.compile_to(str(src), so)
    monkeypatch.setattr(_native, "_lib", _native.bind(so))
    assert _first_kill(BATTERIES[battery]) is not None, f"no pin fails for C mutant: {mid}"


MODULES = {"series": series, "truncation": truncation, "exact": exact, "philox": philox,
           "tgtplus": tgtplus, "learned": learned, "meet": meet}


@pytest.mark.parametrize("module,mid,battery,old,new", PY_MUTANTS, ids=[m[1] for m in PY_MUTANTS])
def test_py_mutant_is_killed(module, mid, battery, old, new, monkeypatch):
    orig = MODULES[module]
    _swap_module(monkeypatch, orig, _py_mutant(orig, old, new))
    assert _first_kill(BATTERIES[battery]) is not None, f"no pin fails for mutant of {module}: {mid}"
