"""The pins must discriminate: plant plausible mistakes in a temporary copy of
the oracle (never in the oracle itself) and check that the pin suite fails
for every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "tie_rule_le": ("if (c <= 4096) return (2 * r < c) ? O_RUN : O_ARRAY;",
                    "if (c <= 4096) return (2 * r <= c) ? O_RUN : O_ARRAY;"),
    "array_max_4095": ("if (c <= 4096) return (2 * r < c)", "if (c < 4096) return (2 * r < c)"),
    "run_limit_2046": ("return (r <= 2047) ? O_RUN : O_BITSET;", "return (r < 2047) ? O_RUN : O_BITSET;"),
    "run_length_not_minus_one": ("uint16_t s = v[i], l = (uint16_t)(v[j] - v[i]);",
                                 "uint16_t s = v[i], l = (uint16_t)(v[j] - v[i] + 1);"),
    "xor_as_or": ("case O_XOR: keep = in_a != in_b; break;", "case O_XOR: keep = in_a || in_b; break;"),
    "andnot_transposed": ("case O_ANDNOT: keep = in_a && !in_b; break;",
                          "case O_ANDNOT: keep = !in_a && in_b; break;"),
    "runs_not_maximal": ("if (i == 0 || (uint32_t)v[i] != (uint32_t)v[i - 1] + 1) r++;",
                         "if (i == 0 || (uint32_t)v[i] != (uint32_t)v[i - 1]) r++;"),
    "bit_order": ("out->data[v[i] >> 3] |= (uint8_t)(1u << (v[i] & 7));",
                  "out->data[v[i] >> 3] |= (uint8_t)(0x80u >> (v[i] & 7));"),
    "jaccard_via_xor": ("*uni = orc_op_card(O_OR, a, b);", "*uni = orc_op_card(O_XOR, a, b);"),
    "fold_skips_last": ("for (uint32_t i = 1; i < k && acc; i++) {", "for (uint32_t i = 1; i + 1 < k && acc; i++) {"),
    "run_end_exclusive": ("r = low >= s && low <= s + l;", "r = low >= s && low < s + l;"),
    "cosine_sum": ("return (double)*inter / sqrt((double)ca * (double)cb);",
                   "return (double)*inter / sqrt((double)ca + (double)cb);"),
}

RUNNER = r"""
import sys, traceback
sys.path[:0] = [sys.argv[1], sys.argv[2], sys.argv[3]]
import oracle, workloads
oracle.build(force=True)
import test_oracle as T
fails = 0
for name in ["test_fig1_layout", "test_difference_example", "test_dedup_example",
             "test_array_bitset_union_example", "test_type_thresholds",
             "test_count_identities_and_jaccard", "test_multi_way_fold", "test_edges",
             "test_membership", "test_cosine"]:
    try:
        getattr(T, name)(oracle)
    except Exception:
        fails += 1
for s in range(6):
    try:
        T.test_ops_vs_brute_force(oracle, s)
    except Exception:
        fails += 1
print("FAILS", fails)
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found"
    dst = tmp_path / "oracle"
    dst.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), dst / "__init__.py")
    (dst / "oracle.c").write_text(src.replace(old, new))
    out = subprocess.run([sys.executable, "-c", RUNNER, str(tmp_path), os.path.join(ROOT, "tests"), ROOT],
                         capture_output=True, text=True, timeout=300)
    assert "FAILS" in out.stdout, out.stderr[-2000:]
    fails = int(out.stdout.split("FAILS")[1].split()[0])
    assert fails > 0, f"mutant {name} survived every pin"
