"""Planted mistakes in the C oracle fail its pins.  Each case copies the oracle package
to a temporary directory, changes one line of its C source to a plausible mistake (the
kind of slip a careful reader could miss), builds that copy and runs the pins written for
the function against it: at least one must fail.  The oracle in the tree is untouched."""
import functools
import importlib.util
import os
import shutil

import numpy as np
import pytest

import test_oracle_pins as pins
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    # the odd element of a tree level folded into the first pair instead of carried up
    "tree_carry": ("if (m & 1) v[k++] = v[m - 1];", "if (m & 1) v[0] = v[0] + v[m - 1];",
                   [pins.test_fp32_tree_golden]),
    # bfloat16 ties rounded away from zero instead of to even
    "bf16_ties_away": ("return (lo & 1) ? hi : lo;", "return hi;", [pins.test_bf16_golden_and_round_trip]),
    # E4M3 ties to the odd code
    "e4m3_ties_odd": ("(d == bd && (c & 1) == 0)", "(d == bd && (c & 1) == 1)", [pins.test_e4m3_golden_and_exhaustive]),
    # Neumaier without its compensation term in the result
    "neumaier_no_comp": ("volatile float y = sum + c;", "volatile float y = sum;",
                         [pins.test_neumaier_golden_and_exact_rational]),
    # Neumaier's magnitude test reversed
    "neumaier_branch": ("if (fabsf(sum) >= fabsf(x[i])) {", "if (fabsf(sum) <= fabsf(x[i])) {",
                        [pins.test_neumaier_golden_and_exact_rational]),
    # compare_swap storing when the values differ
    "cswap_condition": ("else if (kind == K_CSWAP) nw = (old == cond) ? (uint64_t)v : (uint64_t)old;",
                        "else if (kind == K_CSWAP) nw = (old != cond) ? (uint64_t)v : (uint64_t)old;",
                        [pins.test_amo_wraparound_cswap_xor]),
    # the serialisation checker accepting a group whatever the word's final value
    "checker_ignores_final": ("if (!has_final || cur == final) { result = 1; break; }", "if (1) { result = 1; break; }",
                              [pins.test_serialisation_checker_vs_brute_force,
                               pins.test_serialisation_checker_groups_and_long_chain]),
    # the AMO stream's compare_swap swapping when the word differs from its initial value
    "stream_cswap_condition": ("else if (code == 1) nw = ((uint64_t)old == or_cb64(table_seed, w)) ? r : (uint64_t)old;",
                               "else if (code == 1) nw = ((uint64_t)old != or_cb64(table_seed, w)) ? r : (uint64_t)old;",
                               [pins.test_amo_stream_single_kind_closed_forms]),
    # quantisation by a rounded reciprocal of the scale instead of a division
    "quantize_reciprocal": ("volatile float y = x[i] / s;", "volatile float y = x[i] * (1.0f / s);",
                            [pins.test_quantize_scales_and_codes]),
    # fcollect gathering the members in reverse rank order
    "fcollect_order": ("memcpy(tmp + (uint64_t)r * nbytes, at(&h, member(start, stride, r), src), nbytes);",
                       "memcpy(tmp + (uint64_t)r * nbytes, at(&h, member(start, stride, size - 1 - r), src), nbytes);",
                       [pins.test_fcollect_definition]),
    # the int64 max reduction keeping the smaller value
    "i64_max_is_min": ("                else if (op == R_MAX) acc = x > acc ? x : acc;\n                else acc = x < acc ? x : acc;\n            }\n            memcpy(out + k * 8, &acc, 8);",
                       "                else if (op == R_MAX) acc = x < acc ? x : acc;\n                else acc = x < acc ? x : acc;\n            }\n            memcpy(out + k * 8, &acc, 8);",
                       [functools.partial(pins.test_int_reduce_brute_force_tiny, dtype=W.DT_INT64, npdt=np.int64, bits=64),
                        pins.test_reduce_closed_form_and_one_hot]),
    # broadcast that leaves the root's own destination untouched
    "broadcast_skips_root": ("    for (int r = 0; r < size; r++) memcpy(at(&h, member(start, stride, r), dst), tmp, nbytes);\n    free(tmp);\n    return OR_OK;\n}\n\n/* fcollect",
                             "    for (int r = 0; r < size; r++) if (r != root) memcpy(at(&h, member(start, stride, r), dst), tmp, nbytes);\n    free(tmp);\n    return OR_OK;\n}\n\n/* fcollect",
                             [pins.test_broadcast_definition_root_included]),
    # put-with-signal adding where it should set
    "signal_set_adds": ("    if (sig_op == S_SET) s = v;", "    if (sig_op == S_SET) s = s + v;", [pins.test_signal_ops]),
    # dequantisation dividing by the block scale instead of multiplying
    "dequant_divides": ("    volatile float r = v * scales[i / 128];", "    volatile float r = v / scales[i / 128];",
                        [pins.test_qsum_single_member_is_dequantised_input]),
    # the quantised all-reduce accumulating the members in reverse rank order
    "qsum_reverse_order": ("col[r] = deq(at(&h, p, q_off), (const float *)at(&h, p, s_off), k, fmt);",
                           "col[size - 1 - r] = deq(at(&h, p, q_off), (const float *)at(&h, p, s_off), k, fmt);",
                           [pins.test_qsum_multi_member_golden]),
    # the quantised all-reduce dequantising every member with the first member's scales
    "qsum_scale_of_member0": ("col[r] = deq(at(&h, p, q_off), (const float *)at(&h, p, s_off), k, fmt);",
                              "col[r] = deq(at(&h, p, q_off), (const float *)at(&h, member(start, stride, 0), s_off), k, fmt);",
                              [pins.test_qsum_multi_member_golden, pins.test_serve_request_results_by_kind]),
    # alltoall without the transpose (block j of member i stays block j)
    "alltoall_no_transpose": ("memcpy(tmp + ((uint64_t)j * size + i) * m,", "memcpy(tmp + ((uint64_t)i * size + j) * m,",
                              [pins.test_alltoall_is_exact_transpose_permutation]),
}


def _mutant_oracle(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, name
    d = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), d, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (d / "oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_fail_on_a_planted_mistake(tmp_path, name):
    old, new, tests = MUTANTS[name]
    mutant = _mutant_oracle(tmp_path, name, old, new)
    failed = 0
    for t in tests:
        try:
            t(mutant)
        except (AssertionError, mutant.OracleError):
            failed += 1
    assert failed >= 1, name
