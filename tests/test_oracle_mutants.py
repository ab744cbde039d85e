"""Plants one plausible mistake at a time in a copy of the oracle source
(compiled on the CPU into a temporary library) and checks that at least one
pin fails on it, so that the pins would notice such a mistake in the oracle."""
import pytest

import oracle
from tests import _pins

# (name, text in cg_oracle.c, replacement)
MUTANTS = [
    ("suffix_complement", "out[k].contrib = suf ? suf[x] : 0;", "out[k].contrib = suf ? len[w] - suf[x] : 0;"),
    ("entry_end_from_own_bit", "o = (code[x] >> 1) & 1;", "o = code[x] & 1;"),
    ("leave_through_entry_end", "edge_at_end(rp, col, code, is_branch, cur, 1 - o)", "edge_at_end(rp, col, code, is_branch, cur, o)"),
    ("rc_without_complement", "3 - stored_base(packed, off, first - t)", "stored_base(packed, off, first - t)"),
    ("rc_without_reversal", "3 - stored_base(packed, off, first - t)", "3 - stored_base(packed, off, first + t)"),
    ("prefix_not_suffix", "s->first = o == 0 ? L - s->contrib : s->contrib - 1;", "s->first = o == 0 ? 0 : L - 1;"),
    ("xdrop_post_from_pre", ": post[s->x_in];", ": pre[s->x_in];"),
    ("xdrop_exclusive_end", "o == 0 ? last - first + 1 : first - last + 1;", "o == 0 ? last - first : first - last;"),
    ("xdrop_alpha_flipped", "s->x_in < 0 ? (o == 0 ? 0 : L - 1)", "s->x_in < 0 ? (o == 0 ? L - 1 : 0)"),
    ("xdrop_beta_flipped", "s->x_out < 0 ? (o == 0 ? L - 1 : 0)", "s->x_out < 0 ? (o == 0 ? 0 : L - 1)"),
    ("xdrop_cycle_keeps_closing_edge", "if (w == r) { *edges_touched += 2; break; }",
     "if (w == r) { *edges_touched += 2; out[k - 1].x_out = x; break; }"),
    ("tr_ignores_end_at_u", "if (v == w || (code[y] & 1) != eu) continue;", "if (v == w) continue;"),
    ("tr_ignores_pass_through", "if ((code[z] & 1) != 1 - ev_in) continue;", "if (0) continue;"),
    ("tr_ignores_end_at_w", "if (((code[z] >> 1) & 1) != ew) continue;", "if (0) continue;"),
    ("tr_one_direction", "if (trans[x] || mirror_trans) continue;", "if (trans[x]) continue;"),
    ("tr_tolerance_one_sided", "if (d <= fuzz && d >= -fuzz)", "if (d <= fuzz)"),
    ("xdrop_validate_pre_against_v", "if (pre[x] < 0 || pre[x] > len[u] - 1)", "if (pre[x] < 0 || pre[x] > len[v] - 1)"),
    ("degree_threshold_4", "b1[v] = (uint8_t)(d >= 3);", "b1[v] = (uint8_t)(d >= 4);"),
    ("degree_threshold_2", "b1[v] = (uint8_t)(d >= 3);", "b1[v] = (uint8_t)(d >= 2);"),
    ("no_same_end_rule", "if (cnt == 2 && ends[0] == ends[1]) br = 1;", "if (0) br = 1;"),
    ("same_end_rule_inverted", "if (cnt == 2 && ends[0] == ends[1]) br = 1;", "if (cnt == 2 && ends[0] != ends[1]) br = 1;"),
    ("same_end_counts_masked_nbrs", "if (b1[col[x]]) continue;\n        if (cnt < 2)", "if (0) continue;\n        if (cnt < 2)"),
    ("root_orientation_flipped", "o_root = 1 - e;", "o_root = e;"),
    ("larger_root_first", "          o_root = 0;\n        }\n        break;", "          o_root = 0;\n        }\n        continue;"),
    ("cycle_starts_reverse", "if (root < 0) { root = c; o_root = 0; cycle = 1; }", "if (root < 0) { root = c; o_root = 1; cycle = 1; }"),
    ("no_min_chain_filter", "if (q < min_chain_reads) continue;", "if (0) continue;"),
    ("min_chain_off_by_one", "if (q < min_chain_reads) continue;", "if (q <= min_chain_reads) continue;"),
    ("lone_read_reverse", "        } else {\n          o_root = 0;\n        }", "        } else {\n          o_root = 1;\n        }"),
    ("validate_allows_self_overlap", 'if (v == u) BAD("entry %lld: self overlap", (long long)x);', 'if (0) BAD("entry %lld: self overlap", (long long)x);'),
    ("validate_stream_end_off_by_one", "off[v] + len[v] > packed_bytes * 4", "off[v] + len[v] > packed_bytes * 4 + 1"),
    ("validate_xdrop_full_post", "post[x] > len[v] - 1", "post[x] > len[v]"),
    ("validate_xdrop_negative_pre", "if (pre[x] < 0 ||", "if (pre[x] < -1 ||"),
    ("uf_root_larger", "if (a < b) parent[b] = a; else parent[a] = b;", "if (a > b) parent[b] = a; else parent[a] = b;"),
    ("cycle_starts_at_largest", "if (root < 0) { root = c; o_root = 0; cycle = 1; }",
     "if (root < 0) { root = members[cnt[c + 1] - 1]; o_root = 0; cycle = 1; }"),
    ("same_end_uses_far_end", "if (cnt < 2) ends[cnt] = code[x] & 1;", "if (cnt < 2) ends[cnt] = (code[x] >> 1) & 1;"),
    ("xdrop_single_base_piece_dropped", "s->contrib = c > 0 ? c : 0;", "s->contrib = c > 1 ? c : 0;"),
    ("validate_skips_row_ptr_end", 'if (rp[n] != m) BAD("row_ptr[n] != n_entries");', "if (0) {}"),
    ("validate_allows_negative_off", "if (off[v] < 0 || off[v] + len[v] > packed_bytes * 4)",
     "if (off[v] + len[v] > packed_bytes * 4)"),
    ("walk_into_branch_reads", "if (!is_branch[col[x]] && (code[x] & 1) == e) return x;", "if ((code[x] & 1) == e) return x;"),
    ("deg_L_counts_masked", "for (int64_t x = rp[v]; x < rp[v + 1]; ++x) d += !is_branch[col[x]];",
     "for (int64_t x = rp[v]; x < rp[v + 1]; ++x) d += 1;"),
    ("tr_suffix_terms_swapped", "const int64_t d = (int64_t)suf[y] + suf[z] - suf[x];",
     "const int64_t d = (int64_t)suf[y] + suf[x] - suf[z];"),
    ("tr_output_mirror_code", "out_col[k] = col[x]; out_code[k] = code[x];",
     "out_col[k] = col[x]; out_code[k] = (uint8_t)(((code[x] & 1) << 1) | (code[x] >> 1));"),
    ("tr_tolerance_off_by_one", "if (d <= fuzz && d >= -fuzz)", "if (d <= fuzz + 1 && d >= -fuzz - 1)"),
    ("lpt_assign_by_position", "assign[order[i]] = best;", "assign[i] = best;"),
    ("lpt_load_of_wrong_job", "loads[best] += sizes[order[i]];", "loads[best] += sizes[i];"),
    ("revcomp_without_reversal", "char c = in[n - 1 - i], d = 'N';", "char c = in[i], d = 'N';"),
    ("revcomp_c_not_complemented", "case 'C': d = 'G'; break;", "case 'C': d = 'C'; break;"),
    ("bfs_crosses_branch_reads", "if (is_branch[v] || label[v] != -2) continue;", "if (label[v] != -2) continue;"),
    ("bfs_label_of_last_reached", "label[v] = (int32_t)s; queue[tail++] = v;", "label[v] = (int32_t)v; queue[tail++] = v;"),
    ("ascii_table_swapped", "{'A', 'C', 'G', 'T'}", "{'A', 'G', 'C', 'T'}"),
    ("packed_bit_order", "return (packed[q >> 2] >> (2 * (q & 3))) & 3;", "return (packed[q >> 2] >> (6 - 2 * (q & 3))) & 3;"),
    ("validate_skips_mirror_code", "if (code[y] != swapped) BAD", "if (0) BAD"),
    ("validate_allows_full_suffix", "suf[x] > len[v] - 1", "suf[x] > len[v]"),
    ("lpt_most_loaded", "if (loads[b] < loads[best]) best = b;", "if (loads[b] > loads[best]) best = b;"),
    ("lpt_ascending", "while (j > 0 && sizes[order[j - 1]] < sizes[t])", "while (j > 0 && sizes[order[j - 1]] > sizes[t])"),
    ("lpt_unstable_order", "while (j > 0 && sizes[order[j - 1]] < sizes[t])", "while (j > 0 && sizes[order[j - 1]] <= sizes[t])"),
    ("lpt_tie_to_last_part", "if (loads[b] < loads[best]) best = b;", "if (loads[b] <= loads[best]) best = b;"),
    ("uf_ignores_mask", "int64_t v = col[x];\n      if (is_branch[v]) continue;\n      int64_t a = uf_find",
     "int64_t v = col[x];\n      int64_t a = uf_find"),
    ("contigs_in_root_order", "r->chain_id[s->read] = (int32_t)c;", "r->chain_id[s->read] = (int32_t)root;"),
    ("rank_off_by_one", "r->rank[s->read] = (int32_t)i;", "r->rank[s->read] = (int32_t)(i + 1);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = oracle.source()
    assert src.count(old) == 1, f"mutation site for {name} must be unique"
    mut = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    caught = []
    for pin in _pins.ALL_PINS:
        try:
            pin(mut)
        except Exception as e:  # an assertion or a crash-free error report both count
            caught.append(f"{pin.__name__}: {type(e).__name__}")
    assert caught, f"no pin notices the planted mistake {name}"
