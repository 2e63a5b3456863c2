"""Plants plausible mistakes in a copy of oracle.c (on the CPU) and checks that
the pins of test_oracle_pins.py catch every one of them."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle as O
import test_oracle_pins as P

MUTANTS = {
    "tie_to_largest_label": ("(W[c] == bestw && c < best)", "(W[c] == bestw && c > best)"),
    "self_loop_counted": ("if (j == i) continue;                       /* scanCommunities: i != j */", ""),
    "strict_stop_test": ("if ((double)dn / (double)n <= tau) break;   /* converged? */",
                         "if ((double)dn / (double)n < tau) break;"),
    "gauss_seidel_reads": ("next[i] = best_label(i, off, col, w, prev, W, touched);\n    if (next[i] != prev[i]) ++dn;",
                           "{ int32_t b = best_label(i, off, col, w, prev, W, touched);\n"
                           "    if (b != prev[i]) ++dn; next[i] = b; ((int32_t*)prev)[i] = b; }"),
    "weights_ignored": ("W[c] += (w ? w[e] : 1);", "W[c] += 1;"),
    "first_neighbour_dropped": ("for (int64_t e = off[i]; e < off[i + 1]; ++e) {\n    int32_t j = col[e];\n    if (j == i)",
                                "for (int64_t e = off[i] + 1; e < off[i + 1]; ++e) {\n    int32_t j = col[e];\n    if (j == i)"),
    "dn_counts_everything": ("if (next[i] != prev[i]) ++dn;", "++dn;"),
    "split_ignores_community": ("if (!vis[j] && C[j] == c) {             /* f_if */", "if (!vis[j]) {"),
    "split_labels_by_self": ("Cp[u] = (int32_t)i;                       /* f_do */", "Cp[u] = u;"),
    "s1_counts_all_edges": ("if (C[col[e]] == C[i]) s1 += we;", "s1 += we;"),
    "sigma_not_squared_over_2m2": ("(double)s2 / (dm * dm)", "(double)s2 / dm"),
    "sigma_indexed_by_vertex": ("Sigma[C[i]] += K;", "Sigma[i] += K;"),
    "seq_no_reactivation": ("for (int64_t e = off[i]; e < off[i + 1]; ++e) processed[col[e]] = 0;", ""),
    "alg4_off_by_one": ("if (reached < S[c])", "if (reached <= S[c])"),
    "lp_split_no_community_test": ("if (C[j] == C[i] && Cp[j] < cmin) cmin = Cp[j];", "if (Cp[j] < cmin) cmin = Cp[j];"),
    "float_tie_to_largest_label": (
        "(W[c] == bestw && c < best)) { best = c; bestw = W[c]; }\n  }\n  for (int64_t k = 0; k < nt; ++k) W[touched[k]] = 0.0;",
        "(W[c] == bestw && c > best)) { best = c; bestw = W[c]; }\n  }\n  for (int64_t k = 0; k < nt; ++k) W[touched[k]] = 0.0;"),
    "float_weights_ignored": ("W[c] += (double)w[e];", "W[c] += 1.0;"),
    "float_sigma_indexed_by_vertex": ("Sigma[C[i]] += K;\n  }\n  double s2 = 0.0;", "Sigma[i] += K;\n  }\n  double s2 = 0.0;"),
    "float_self_loop_counted": ("    if (j == i) continue;\n    int32_t c = C[j];\n    if (W[c] == 0.0)",
                                "    int32_t c = C[j];\n    if (W[c] == 0.0)"),
}

PINS = [
    (P.test_two_k5_bridge_sweeps_by_hand, {}),
    (P.test_stop_rule_boundaries, {}),
    (P.test_single_edge_oscillates, {}),
    (P.test_path4_two_sweeps_by_hand, {}),
    (P.test_weights_override_counts_and_ties, {}),
    (P.test_self_loop_is_ignored_and_isolated_vertex_keeps_label, {}),
    (P.test_complete_graph, {"n": 7}),
    (P.test_all_graphs_on_5_vertices_one_sweep, {}),
    (P.test_random_weighted_multigraphs_one_sweep, {}),
    (P.test_sequential_in_place_path4_by_hand, {}),
    (P.test_sequential_reactivation_by_hand, {}),
    (P.test_sequential_converged_state_is_a_fixed_point, {}),
    (P.test_split_path_by_hand, {}),
    (P.test_split_equals_scipy_components, {}),
    (P.test_split_lp_and_lpp_reach_the_bfs_labels, {}),
    (P.test_modularity_two_k5_closed_form, {}),
    (P.test_modularity_path_split_by_hand, {}),
    (P.test_modularity_matches_networkx_and_pair_sum, {}),
    (P.test_disconnected_checker_by_hand_and_vs_scipy, {}),
    (P.test_float_sweep_matches_dense_product, {}),
    (P.test_float_self_loop_is_ignored_by_hand, {}),
    (P.test_float_lpa_with_integer_weights_equals_integer_lpa, {}),
    (P.test_float_modularity_matches_networkx, {}),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_kill_mutant(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(O.__file__), "oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(c)])
    monkeypatch.setattr(O, "_handle", O.configure(ctypes.CDLL(str(so))))
    killed = []
    for fn, kw in PINS:
        try:
            fn(**kw)
        except Exception as e:  # noqa: BLE001 -- any failure kills the mutant
            killed.append(fn.__name__)
    assert killed, f"mutant {name} survived every pin"
