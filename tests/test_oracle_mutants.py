"""Planted mistakes in the oracle, on the CPU: each case is the oracle's source
with one plausible mistake -- a dropped term, a wrong sign, a wrong index, a
reversed or lost tie-break, a wrong rounding or constant, a wrong step of the
descent, the wrong candidate expanded first -- built into a library of its
own.  The named pins
(the oracle's own tests, which check it against closed forms, numpy, torch's
casts and hand-worked goldens) must fail on every such copy; on the real oracle they
pass (they run in the suite).  This is the evidence that the pins would catch
the mistake, not only that the oracle agrees with itself."""
import gc
import os
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle as O
import test_oracle_formats as TF
import test_oracle_levels as TL
import test_oracle_pq as TP
import test_oracle_rerank as TR
import test_oracle_search as TS
import test_oracle_sparse as TSp
from oracle import build as OB

# name: (text in kann_oracle.cpp, its replacement, pins that must fail)
MUTANTS = {
    "l2_drops_the_last_dimension": (
        "for (int k = 0; k < d; ++k) { double t = q[k] - x(j, k); s += t * t; }",
        "for (int k = 0; k + 1 < d; ++k) { double t = q[k] - x(j, k); s += t * t; }",
        [lambda: TS.test_brute_force_when_ef_covers_n(O.L2)]),
    "ip_with_the_wrong_sign": (
        "for (int k = 0; k < d; ++k) s -= q[k] * x(j, k);",
        "for (int k = 0; k < d; ++k) s += q[k] * x(j, k);",
        [lambda: TS.test_brute_force_when_ef_covers_n(O.IP)]),
    "pq_table_reads_the_wrong_query_subvector": (
        "double qq = qv[j * dsub + t], cc = C[t];",
        "double qq = qv[t], cc = C[t];",
        [TP.test_adc_equals_exact_distance_to_reconstruction]),
    "sparse_ip_drops_the_query_weight": (
        "s += (double)wa[i] * wb;",
        "s += (double)wa[i];",
        [TSp.test_sparse_ip_equals_densified_ip]),
    "ties_go_to_the_higher_id": (
        "return a.id < b.id;",
        "return a.id > b.id;",
        [TS.test_duplicates_ordered_by_id_and_self_query,
         lambda: TR.test_rerank_equals_numpy_lexsort_on_tied_integer_rows(O.L2, False)]),
    "rerank_keeps_candidate_order_on_ties": (
        "std::sort(cs.begin(), cs.end(), CandLess());",
        "std::stable_sort(cs.begin(), cs.end(), [](const Cand& a, const Cand& b) { return a.d < b.d; });",
        [lambda: TR.test_rerank_equals_numpy_lexsort_on_tied_integer_rows(O.L2, True)]),
    "level_law_with_base_m_plus_one": (
        "std::log((double)M)",
        "std::log((double)M + 1.0)",
        [lambda: TL.test_level_law_chi_square(16)]),
    "fp16_rounds_ties_away_from_zero": (
        "double r = std::nearbyint(a / quantum);",
        "double r = std::round(a / quantum);",
        [TF.test_f16_encode_matches_numpy_rne]),
    "e4m3_scale_divides_by_447": (
        "float s = mx / 448.0f;",
        "float s = mx / 447.0f;",
        [TF.test_e4m3_rows_match_torch_cast_and_error_bound]),
    "u8_table_forgets_the_subspace_minimum": (
        "const float r = std::fmin(std::fmax((e[(size_t)j * ksub + c] - mn[j]) / t.scale, 0.f), 255.f);",
        "const float r = std::fmin(std::fmax((e[(size_t)j * ksub + c]) / t.scale, 0.f), 255.f);",
        [lambda: TP.test_u8_table_equals_its_definition_written_in_numpy(O.L2)]),
    "pq_encode_ties_to_the_highest_centroid": (
        "if (s < best) { best = s; bc = c; }\n      }\n      codes[(size_t)i * m + j] = (uint8_t)bc;",
        "if (s <= best) { best = s; bc = c; }\n      }\n      codes[(size_t)i * m + j] = (uint8_t)bc;",
        [TP.test_encode_picks_nearest_and_lowest_on_ties]),
    "greedy_descent_takes_the_first_better_neighbour": (
        "if (cand_less(ce, best)) best = ce;",
        "if (cand_less(ce, cur)) { best = ce; break; }",
        [lambda: TS.test_hand_worked_golden(O.FORM_FLAGS)]),
    "bf16_keeps_one_bit_less": (
        "double v = round_to_format((double)x, 8, -126, std::ldexp(255.0, 120), false);",
        "double v = round_to_format((double)x, 7, -126, std::ldexp(255.0, 120), false);",
        [TF.test_bf16_encode_matches_torch]),
    "e4m3_decode_exponent_bias_off_by_one": (
        "else v = std::ldexp(8.0 + m, e - 10);",
        "else v = std::ldexp(8.0 + m, e - 11);",
        [TF.test_e4m3_decode_all_codes]),
    "fp16_subnormals_start_one_binade_low": (
        "double v = round_to_format((double)x, 11, -14, 65504.0, false);",
        "double v = round_to_format((double)x, 11, -15, 65504.0, false);",
        [TF.test_f16_encode_matches_numpy_rne]),
    "rerank_scores_inner_product_as_l2": (
        "DenseSpace sp(dtype, data, scale, d, metric);\n  for (int64_t qi = 0; qi < nq; ++qi) {\n"
        "    sp.set_query(queries + (size_t)qi * d);\n    std::vector<Cand> cs;",
        "DenseSpace sp(dtype, data, scale, d, MET_L2);\n  for (int64_t qi = 0; qi < nq; ++qi) {\n"
        "    sp.set_query(queries + (size_t)qi * d);\n    std::vector<Cand> cs;",
        [lambda: TR.test_rerank_equals_numpy_lexsort_on_tied_integer_rows(O.IP, False)]),
    "two_heap_search_stops_at_the_first_equal": (
        "if (cand_less(f, c)) break;  // c is further than the furthest kept",
        "if (!cand_less(c, f)) break;",
        [lambda: TS.test_hand_worked_golden(O.FORM_TWO_HEAP)]),
    "multi_expansion_takes_one_entry_too_many": (
        "for (size_t c = 0; c < W.size() && (int)chosen.size() < p; ++c) {",
        "for (size_t c = 0; c < W.size() && (int)chosen.size() <= p; ++c) {",
        [TS.test_multi_expansion_hand_worked_golden]),
    "search_lets_a_forgotten_id_into_w_twice": (
        "if (pos < W.size() && W[pos].id == ce.id) continue;  // already in W",
        "",
        [lambda: TS.test_forgetful_visited_set_changes_nothing_on_tied_integer_data(1)]),
    "adc_sum_skips_the_last_subspace": (
        "for (int j = 0; j < m; ++j) s += lut[(size_t)j * ksub + ci[j]];",
        "for (int j = 0; j + 1 < m; ++j) s += lut[(size_t)j * ksub + ci[j]];",
        [TP.test_pq_is_exact_when_every_subvector_is_a_centroid]),
    "u8_distance_offset_skips_a_minimum": (
        "for (int j = 0; j < m; ++j) sm += mn[j];",
        "for (int j = 0; j + 1 < m; ++j) sm += mn[j];",
        [lambda: TP.test_u8_table_equals_its_definition_written_in_numpy(O.L2)]),
    "lloyd_mean_divides_by_count_plus_one": (
        "C[(size_t)c * dsub + t] = sum[(size_t)c * dsub + t] / (double)cnt[c];",
        "C[(size_t)c * dsub + t] = sum[(size_t)c * dsub + t] / (double)(cnt[c] + 1);",
        [TP.test_pq_is_exact_when_every_subvector_is_a_centroid]),
    "e4m3_rows_ignore_their_scale": (
        "default: return decode_e4m3(((const uint8_t*)data)[o]) * (double)scale[j];",
        "default: return decode_e4m3(((const uint8_t*)data)[o]);",
        [TR.test_distances_on_stored_fp16_and_e4m3_rows_decode_them]),
    "fp16_table_keeps_one_bit_less": (
        "for (double& v : lut) v = std::ldexp(round_to_format(std::ldexp(v, -e), 11, -14, 65504.0, false), e);",
        "for (double& v : lut) v = std::ldexp(round_to_format(std::ldexp(v, -e), 10, -14, 65504.0, false), e);",
        [TP.test_fp16_table_is_the_scaled_half_rounding_of_the_fp64_table]),
    "sparse_query_loses_its_last_term": (
        "qt.assign(t, t + nnz);",
        "qt.assign(t, t + (nnz > 0 ? nnz - 1 : 0));",
        [TSp.test_sparse_ip_equals_densified_ip]),
    "search_expands_the_worst_unexpanded_entry": (
        "size_t c = 0;\n    while (c < W.size() && expanded[c]) ++c;",
        "size_t c = W.size();\n    for (size_t t = W.size(); t-- > 0;) if (!expanded[t]) { c = t; break; }",
        [lambda: TS.test_hand_worked_golden(O.FORM_FLAGS)]),
}


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_mutants")
    with open(OB.SRC) as f:
        src = f.read()

    def one(name):
        old, new, _ = MUTANTS[name]
        assert src.count(old) == 1, name  # the planted change hits exactly one place
        path = os.path.join(str(d), name + ".cpp")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        return name, OB.compile_source(path, os.path.join(str(d), name + ".so"))

    with ThreadPoolExecutor(max_workers=len(MUTANTS)) as ex:
        return dict(ex.map(one, MUTANTS))


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_the_planted_mistake(mutant_libs, name):
    real = O.lib()
    O._lib = O.load(mutant_libs[name])
    try:
        caught = 0
        for pin in MUTANTS[name][2]:
            try:
                pin()
            except AssertionError:
                caught += 1
        assert caught == len(MUTANTS[name][2]), "a pin passed on the mutant %s" % name
    finally:
        gc.collect()  # graphs built by the mutant are freed while it is loaded
        O._lib = real
