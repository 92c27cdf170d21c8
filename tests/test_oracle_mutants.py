"""The pins must reject plausible mistakes in the oracle.

Each case below plants one mistake in a copy of the oracle's C++ source (on
the CPU: a dropped term, a wrong comparison, an off-by-one index or a wrong
boundary value), builds it to a temporary library, and runs the pins against
that build: at least one pin has to fail.  The shipped oracle is never
modified.
"""
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "minjoin_oracle.cpp")

MUTANTS = [
    # (name, text in the source, replacement)
    ("anchor_not_strict", "if (h[i] >= h[j]) {", "if (h[i] > h[j]) {"),
    ("radius_denominator", "floor_div(slen - q + 1 - T, 2 * T + 2)", "floor_div(slen - q + 1 - T, 2 * T + 1)"),
    ("closing_anchor", "A.push_back(slen);", "A.push_back(slen - 1);"),
    ("anchor_range_lo", "for (int64_t i = r; i <= m - 1 - r; ++i) {", "for (int64_t i = r + 1; i <= m - 1 - r; ++i) {"),
    ("anchor_range_hi", "for (int64_t i = r; i <= m - 1 - r; ++i) {", "for (int64_t i = r; i <= m - r; ++i) {"),
    ("partition_len", "out_len[cnt] = A[i + 1] - A[i];", "out_len[cnt] = A[i + 1] - A[i] - 1;"),
    ("pack_shift", "code = (code << bits) | (uint64_t)rank[s[i + t]];", "code = (code << 1) | (uint64_t)rank[s[i + t]];"),
    ("position_filter_term",
     "iabs(pos - e.pos) + iabs((slen_i - pos) - (slen_j - e.pos)) <= K",
     "iabs(pos - e.pos) <= K"),
    ("position_filter_sign",
     "iabs((slen_i - pos) - (slen_j - e.pos))",
     "iabs((slen_i - pos) + (slen_j - e.pos))"),
    ("length_filter_strict", "if (iabs(slen_i - slen_j) <= K) {", "if (iabs(slen_i - slen_j) < K) {"),
    ("self_pair_kept", "<= K && e.j != i)", "<= K)"),
    ("ed_drop_insert_cost", "v = std::min(v, prev[j] + 1);\n            v = std::min(v, cur[j - 1] + 1);",
     "v = std::min(v, prev[j]);\n            v = std::min(v, cur[j - 1] + 1);"),
    ("ed_boundary_row", "for (int64_t j = 0; j <= n; ++j) prev[j] = j;", "for (int64_t j = 0; j <= n; ++j) prev[j] = 0;"),
    ("band_boundary_row", "for (int64_t j = 0; j <= std::min(n, k); ++j) prev[j] = j;",
     "for (int64_t j = 0; j <= std::min(n, k); ++j) prev[j] = 0;"),
    ("band_edge", "if (iabs(m - n) > k) return k + 1;", "if (iabs(m - n) >= k) return k + 1;"),
    ("q_rule_boundary", "while (p * t3 < n3) {", "while (p * t3 <= n3) {"),
    ("cutoff_at_k", "if (row_min > k) return k + 1;", "if (row_min >= k) return k + 1;"),
    ("cutoff_row_min_first_cell", "row_min = std::min(row_min, cur[j]);", "row_min = cur[jlo];"),
    ("eviction_of_unpaired_entries",
     "C.emplace_back(std::min(i, e.j), std::max(i, e.j));\n                    kept.push_back(e);",
     "{ C.emplace_back(std::min(i, e.j), std::max(i, e.j)); kept.push_back(e); }"),
    ("join_in_id_order", "for (int64_t i : order) {", "for (int64_t i = 0; i < n; ++i) {"),
]


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation {name} does not apply"
    mutated = src.replace(old, new, 1)
    cpp = tmp_path / f"{name}.cpp"
    so = tmp_path / f"lib{name}.so"
    cpp.write_text(mutated)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(cpp)])
    return str(so)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new):
    so = _build(tmp_path, name, old, new)
    failed = []
    with oracle.using(so):
        for pin_name, fn in pins.ALL_PINS:
            try:
                fn()
            except AssertionError:
                failed.append(pin_name)
    assert failed, f"no pin rejects the mutant {name}"
