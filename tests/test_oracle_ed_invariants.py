"""Metric invariants of the oracle's edit distances: both dynamic programs
(the textbook full DP and Ukkonen's band) on random DNA strings.  A dropped
term, a transposed operand or a wrong boundary in either breaks one of:
ED(x, x) = 0, symmetry, the triangle inequality, ||a|-|b|| <= ED <= max(|a|,
|b|), ED <= Hamming for equal lengths, ED(a, "") = |a|, and banded ED =
min(full ED, k + 1) for every band k."""
import numpy as np

import oracle


def _strings(rng, n, max_len):
    return [bytes(rng.choice(list(b"ACGT"), size=int(rng.integers(0, max_len + 1)))) for _ in range(n)]


def test_metric_axioms_and_bounds():
    rng = np.random.default_rng(21)
    S = _strings(rng, 60, 30)
    ed = {}
    for i, a in enumerate(S):
        assert oracle.ed_full(a, a) == 0
        assert oracle.ed_full(a, b"") == len(a) == oracle.ed_full(b"", a)
        for j, b in enumerate(S):
            d = oracle.ed_full(a, b)
            ed[i, j] = d
            assert abs(len(a) - len(b)) <= d <= max(len(a), len(b))
            if len(a) == len(b):
                assert d <= sum(x != y for x, y in zip(a, b))
    for i in range(len(S)):
        for j in range(len(S)):
            assert ed[i, j] == ed[j, i]
    idx = rng.integers(0, len(S), size=(3000, 3))
    for i, j, k in idx:
        assert ed[i, k] <= ed[i, j] + ed[j, k]


def test_band_is_the_capped_full_distance():
    rng = np.random.default_rng(22)
    base = _strings(rng, 40, 40)
    for a in base:
        # relatives of a at a few planted edits, and unrelated strings
        b = bytearray(a)
        for _ in range(int(rng.integers(0, 8))):
            op = int(rng.integers(0, 3))
            p = int(rng.integers(0, len(b) + 1))
            if op == 0:
                b.insert(p, int(rng.choice(list(b"ACGT"))))
            elif b and op == 1:
                del b[min(p, len(b) - 1)]
            elif b:
                b[min(p, len(b) - 1)] = int(rng.choice(list(b"ACGT")))
        for other in (bytes(b), base[int(rng.integers(0, len(base)))]):
            full = oracle.ed_full(a, other)
            for k in (0, 1, 2, 3, 5, 8, 13, 40):
                assert oracle.ed_band(a, other, k) == min(full, k + 1), (a, other, k)
