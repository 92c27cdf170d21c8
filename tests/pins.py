"""Pins of the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code.  Each function raises
AssertionError on a mismatch.  They run on the shipped oracle build
(tests/test_oracle_pins.py) and on deliberately mutated builds of the same
source, which they must reject (tests/test_oracle_mutants.py).
"""
from __future__ import annotations

import itertools
import math
import os
from collections import deque

import numpy as np

import oracle
import synth
from worked_example import load as load_example, table as example_table

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------ worked example

def pin_worked_example(atc_value: int | None = None):
    """Sec. 2.1 running example: Tables 2-4 and the candidate / output pairs of
    the text.  Partitions are compared substring by substring with Table 4."""
    ex = load_example()
    strings = [ex["string"][i] for i in sorted(ex["string"])]
    s = synth.from_strings(strings, K=ex["param"]["K"], T=ex["param"]["T"])
    p = oracle.derive_params(s.bytes, s.offsets, K=ex["param"]["K"], T=ex["param"]["T"],
                             q=ex["param"]["q"])
    assert p.sigma == 4 and p.bits == 2
    override = None if atc_value is None else {"ATC": atc_value}
    tab = example_table(ex, p.rank, p.bits, p.q, override)
    parts = oracle.partition(s.bytes, s.offsets, p, table=tab, threads=1)
    for sid in range(len(strings)):
        r_expect, subs_expect = ex["partition"][sid + 1]
        assert oracle.radius(len(strings[sid]), p.q, p.T, p.r_min) == r_expect, sid
        sel = parts.sid == sid
        subs = [strings[sid][a:a + b] for a, b in zip(parts.pos[sel], parts.len[sel])]
        assert subs == subs_expect, (sid, subs, subs_expect)
    C = oracle.candidates(s.bytes, s.offsets, p.K, parts)
    assert [tuple(x) for x in C.tolist()] == sorted(ex["candidate"]), C
    res = oracle.minjoin(s.bytes, s.offsets, K=p.K, T=p.T, q=p.q, table=tab, threads=1)
    assert [tuple(x) for x in res.pairs.tolist()] == sorted(ex["output"]), res.pairs
    # the pair the text rejects has ED > K
    rejected = set(ex["candidate"]) - set(ex["output"])
    for (i, j) in rejected:
        assert oracle.ed_full(strings[i], strings[j]) > p.K


# ------------------------------------------------------------ edit distance

def load_ed_cases():
    out = []
    for line in open(os.path.join(HERE, "golden", "ed_textbook.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b, d = line.split()
        out.append((b"" if a == "-" else a.encode(), b"" if b == "-" else b.encode(), int(d)))
    return out


def pin_ed_textbook():
    for a, b, d in load_ed_cases():
        assert oracle.ed_full(a, b) == d, (a, b, d)
        for k in range(0, d + 3):
            assert oracle.ed_band(a, b, k) == (d if d <= k else k + 1), (a, b, k)


def pin_ed_band_cutoff(seed: int = 17):
    """The banded DP with Ukkonen's cut-off returns min(ED, k + 1): against
    the breadth-first-search distances of all strings of length <= 5 over
    {A, C}, against the textbook cases, and against the full DP on planted
    pairs of DNA at several bands."""
    strings, dist = bfs_distances(b"AC", 5)
    for i, a in enumerate(strings):
        for j, b in enumerate(strings):
            d = int(dist[i, j])
            for k in (0, 1, 2, 3):
                assert oracle.ed_band_cutoff(a, b, k) == min(d, k + 1), (a, b, k, d)
    for a, b, d in load_ed_cases():
        for k in range(0, d + 3):
            assert oracle.ed_band_cutoff(a, b, k) == min(d, k + 1), (a, b, k)
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(40):
        L = int(rng.integers(30, 160))
        a = synth.DNA[rng.integers(0, 4, size=L)]
        b = synth.mutate(rng, a, float(rng.uniform(0.02, 0.3)), synth.DNA)
        d = oracle.ed_full(a.tobytes(), b.tobytes())
        for k in (0, d // 2, d - 1, d, d + 1, 2 * d + 3):
            if k >= 0:
                assert oracle.ed_band_cutoff(a.tobytes(), b.tobytes(), k) == min(d, k + 1), (d, k)


def bfs_distances(alphabet: bytes, maxlen: int) -> tuple[list[bytes], np.ndarray]:
    """Edit distance between all strings of length <= maxlen over `alphabet`,
    by breadth-first search over single insertions, deletions and
    substitutions.  Restricting the search to lengths <= maxlen is exact: an
    optimal edit script can apply its deletions first, so it never passes
    through a string longer than max(|a|, |b|)."""
    strings = [b""]
    for L in range(1, maxlen + 1):
        strings += [bytes(t) for t in itertools.product(alphabet, repeat=L)]
    index = {s: i for i, s in enumerate(strings)}

    def neighbours(s):
        for i in range(len(s)):
            yield s[:i] + s[i + 1:]
            for c in alphabet:
                if c != s[i]:
                    yield s[:i] + bytes([c]) + s[i + 1:]
        if len(s) < maxlen:
            for i in range(len(s) + 1):
                for c in alphabet:
                    yield s[:i] + bytes([c]) + s[i:]

    n = len(strings)
    dist = np.full((n, n), -1, dtype=np.int64)
    for src in range(n):
        dist[src, src] = 0
        dq = deque([strings[src]])
        while dq:
            u = dq.popleft()
            du = dist[src, index[u]]
            for v in neighbours(u):
                iv = index[v]
                if dist[src, iv] < 0:
                    dist[src, iv] = du + 1
                    dq.append(v)
    return strings, dist


def pin_ed_bfs(alphabet: bytes = b"AC", maxlen: int = 5, band_k=(0, 1, 2)):
    strings, dist = bfs_distances(alphabet, maxlen)
    for i, a in enumerate(strings):
        for j, b in enumerate(strings):
            d = int(dist[i, j])
            assert oracle.ed_full(a, b) == d, (a, b, d)
            for k in band_k:
                assert oracle.ed_band(a, b, k) == (d if d <= k else k + 1), (a, b, k, d)


def pin_ed_planted(seed: int = 7, trials: int = 60):
    """A copy made by e edit events is within ED e of its source; ED is also
    at least the length difference and at most the longer length."""
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(trials):
        L = int(rng.integers(20, 120))
        a = synth.DNA[rng.integers(0, 4, size=L)]
        e = int(rng.integers(0, 12))
        b = list(a.tolist())
        for _ in range(e):
            op = int(rng.integers(0, 3))
            if op == 0:
                b.insert(int(rng.integers(0, len(b) + 1)), int(synth.DNA[rng.integers(0, 4)]))
            elif op == 1 and b:
                del b[int(rng.integers(0, len(b)))]
            elif b:
                b[int(rng.integers(0, len(b)))] = int(synth.DNA[rng.integers(0, 4)])
        bb = bytes(b)
        d = oracle.ed_full(a.tobytes(), bb)
        assert abs(len(a) - len(bb)) <= d <= e, (d, e)
        assert d <= max(len(a), len(bb))


# ------------------------------------------------------------ parameters

def pin_q_rule():
    """q = ceil(3 log_sigma(N/T)) (Sec. 2.2), checked against floating-point
    logarithms away from integer boundaries and at exact powers."""
    for sigma in (2, 4, 5, 20, 26, 95):
        for T in (3, 10, 40, 100):
            for N in (50, 500, 4999, 5000, 20000):
                x = 3 * math.log(N / T) / math.log(sigma)
                if abs(x - round(x)) < 1e-9:
                    continue
                assert oracle.q_rule(N, T, sigma) == max(1, math.ceil(x)), (N, T, sigma)
    # exact powers: N/T = sigma^k gives q = 3k exactly
    assert oracle.q_rule(4 ** 3 * 10, 10, 4) == 9
    assert oracle.q_rule(4 ** 3 * 10 + 1, 10, 4) == 10
    assert oracle.q_rule(2 ** 5 * 7, 7, 2) == 15
    assert oracle.q_rule(10, 10, 4) == 1          # N = T: log 1 = 0, clamped to 1
    assert oracle.q_rule(500, 10, 1) == 1


def pin_radius():
    """r = floor((|s| - q + 1 - T) / (2T + 2)) (Alg. 2, neighbourhood radius), floored."""
    assert oracle.radius(21, 3, 3, 0) == 2         # Table 4: s1
    assert oracle.radius(22, 3, 3, 0) == 2         # Table 4: s2
    assert oracle.radius(500, 9, 10, 0) == 21      # (500-9+1-10)/22 = 21.9
    assert oracle.radius(5000, 10, 100, 0) == 24   # 4891/202 = 24.2
    assert oracle.radius(10, 3, 5, 0) == 0         # 3/12
    assert oracle.radius(5, 3, 5, -10) == -1       # -2/12 floors to -1
    assert oracle.radius(5, 3, 5, 1) == 1          # raised to r_min


# ------------------------------------------------------------ partitions

def pin_anchor_shape(seed: int = 3):
    """Anchors are strictly increasing, start at 0 and end at |s|; partitions
    tile the string; a periodic string with period <= r has no interior anchor
    (Sec. 2.1, Discussions)."""
    s = synth.random_set(seed, n=40, min_len=1, max_len=400, K=8, T=8)
    p = oracle.derive_params(s.bytes, s.offsets, K=8, T=8)
    parts = oracle.partition(s.bytes, s.offsets, p, threads=2)
    L = s.lengths()
    for sid in range(s.n):
        sel = parts.sid == sid
        pos, ln = parts.pos[sel], parts.len[sel]
        if L[sid] == 0:
            assert pos.shape[0] == 0
            continue
        assert pos[0] == 0 and np.all(ln > 0)
        assert np.all(pos[1:] == pos[:-1] + ln[:-1])
        assert pos[-1] + ln[-1] == L[sid]
    per = synth.from_strings([b"A" * 300, b"AC" * 150, b"ACG" * 100], K=8, T=8)
    dna = synth.from_strings([b"ACGT"], 8, 8)
    pp = oracle.derive_params(dna.bytes, dna.offsets, K=8, T=8, q=4)
    for sid in range(per.n):
        h = oracle.hash_qgrams(per.string(sid), pp)
        r = oracle.radius(300, pp.q, pp.T, pp.r_min)
        assert r >= 3
        A = oracle.find_anchors(h, 300, r)
        assert A.tolist() == [0, 300], (sid, A)


def pin_anchor_edges():
    """Hand-worked anchors at the edges of Alg. 2's range and under ties
    (tests/golden/anchor_edges.txt)."""
    cases, cand = [], []
    for line in open(os.path.join(HERE, "golden", "anchor_edges.txt")):
        line = line.strip()
        if line.startswith("edge "):
            f = line.split()
            cases.append((f[1].encode(), [x.encode() for x in f[2:]]))
        elif line.startswith("candidates-K6 "):
            f = line.split()
            cand.append((int(f[1]), int(f[2])))
    strings = [c[0] for c in cases]
    s = synth.from_strings(strings, K=2, T=2)
    p = oracle.derive_params(s.bytes, s.offsets, K=2, T=2, q=1)
    assert p.sigma == 4
    tab = np.zeros(1 << p.bits, dtype=np.uint64)
    for sym, v in zip(b"ABCD", (1, 2, 3, 4)):
        tab[p.rank[sym]] = v
    parts = oracle.partition(s.bytes, s.offsets, p, table=tab, threads=1)
    for sid, (st, expect) in enumerate(cases):
        sel = parts.sid == sid
        got = [st[a:a + b] for a, b in zip(parts.pos[sel], parts.len[sel])]
        assert got == expect, (st, got, expect)
    C = oracle.candidates(s.bytes, s.offsets, 6, parts)
    assert [tuple(x) for x in C.tolist()] == cand, C


def pin_lemma1(seed: int = 11, n: int = 300, L: int = 4000, T: int = 50):
    """Lemma 1: on random strings the number X of anchors found by Alg. 2 has
    mean w/(2r+1) ~= T and variance below T, so Pr[|X-T| >= sqrt(cT)] < 1/c."""
    rng = np.random.Generator(np.random.PCG64(seed))
    data = synth.DNA[rng.integers(0, 4, size=n * L)]
    off = np.arange(n + 1, dtype=np.int64) * L
    p = oracle.derive_params(data, off, K=T, T=T)
    parts = oracle.partition(data, off, p, threads=4)
    X = parts.n_anchor - 2                               # interior anchors only
    r = oracle.radius(L, p.q, T, p.r_min)
    w = (L - p.q + 1) - 2 * r
    mu = w / (2 * r + 1)
    assert abs(X.mean() - mu) < 2.0, (X.mean(), mu)
    assert X.var() < 1.3 * T, X.var()
    c = 4.0
    assert np.mean(np.abs(X - T) >= math.sqrt(c * T)) < 1.0 / c


def pin_hash_is_injective(seed: int = 5):
    """Pi gives equal values exactly to equal q-grams (Sec. 2.2 needs no
    collisions in a neighbourhood): checked over all q-grams of random text."""
    rng = np.random.Generator(np.random.PCG64(seed))
    for alphabet, q in ((synth.DNA, 9), (synth.DNA, 20), (synth.PROTEIN, 5), (synth.PRINTABLE, 3)):
        data = alphabet[rng.integers(0, alphabet.shape[0], size=20000)]
        off = np.array([0, data.shape[0]], np.int64)
        p = oracle.derive_params(data, off, K=10, T=10, q=q)
        h = oracle.hash_qgrams(data.tobytes(), p)
        grams = np.lib.stride_tricks.sliding_window_view(data, p.q)
        _, ginv = np.unique(grams, axis=0, return_inverse=True)
        _, hinv = np.unique(h, return_inverse=True)
        # same partition of positions into classes
        pairs = set(zip(ginv.ravel().tolist(), hinv.ravel().tolist()))
        assert len(pairs) == len(set(ginv.ravel().tolist())) == len(set(hinv.ravel().tolist()))


# ------------------------------------------------------------ join

def set_definition_candidates(s: synth.StringSet, K: int, parts: oracle.Partitions) -> set:
    """Candidates by their order-free definition: i != j share a partition
    substring, |len_i - len_j| <= K, and the position filter of Alg. 3
    holds for that matched partition pair."""
    L = s.lengths()
    groups = {}
    for sid, pos, ln in zip(parts.sid.tolist(), parts.pos.tolist(), parts.len.tolist()):
        key = s.string(sid)[pos:pos + ln]
        groups.setdefault(key, []).append((sid, pos))
    out = set()
    for members in groups.values():
        for (i, pi), (j, pj) in itertools.combinations(members, 2):
            if i == j or abs(L[i] - L[j]) > K:
                continue
            if abs(pi - pj) + abs((L[i] - pi) - (L[j] - pj)) <= K:
                out.add((min(i, j), max(i, j)))
    return out


def pin_candidates_definition(seed: int = 21):
    for (n, lo, hi, K, T, fam) in ((120, 30, 120, 6, 6, 8), (80, 1, 60, 4, 3, 4), (150, 200, 260, 12, 12, 10)):
        s = synth.random_set(seed, n=n, min_len=lo, max_len=hi, K=K, T=T, families=fam, rate=0.04)
        p = oracle.derive_params(s.bytes, s.offsets, K=K, T=T)
        parts = oracle.partition(s.bytes, s.offsets, p, threads=2)
        C = oracle.candidates(s.bytes, s.offsets, K, parts)
        got = set(map(tuple, C.tolist()))
        assert got == set_definition_candidates(s, K, parts)
        seed += 1


def pin_join_eviction_order():
    """Alg. 3 visits the strings in length order, which is what makes its
    eviction (an entry whose string length differs from the probing string's
    by more than K leaves the bucket for good) lose no pair.  Hand-worked case
    with q = 1 and Pi(A) = 1 < Pi(D) = 4, T = 10, K = 6:
      x = DDDDA + D*15 (|x| = 20, r = max(floor(10/22), 1) = 1)
      y = DDDDA + D*95 (|y| = 100, r = floor(90/22) = 4)
      z = DDDDA + D*16 (|z| = 21, r = 1)
    In each string the only interior anchor is the A at position 4 (runs of
    D tie), so each starts with the partition DDDD at position 0.  x and z
    pass both filters (|20 - 21| = 1 <= 6); y is 80 longer than x.  In length
    order (x, z, y) the pair (x, z) is found; in id order y would evict x
    before z probes.  The only candidate is (0, 2)."""
    strings = [b"DDDDA" + b"D" * 15, b"DDDDA" + b"D" * 95, b"DDDDA" + b"D" * 16]
    s = synth.from_strings(strings, K=6, T=10)
    p = oracle.derive_params(s.bytes, s.offsets, K=6, T=10, q=1)
    tab = np.zeros(1 << p.bits, dtype=np.uint64)
    tab[p.rank[ord("A")]] = 1
    tab[p.rank[ord("D")]] = 4
    parts = oracle.partition(s.bytes, s.offsets, p, table=tab, threads=1)
    for sid, st in enumerate(strings):
        sel = parts.sid == sid
        assert parts.pos[sel].tolist() == [0, 4] and parts.len[sel].tolist() == [4, len(st) - 4], sid
    C = oracle.candidates(s.bytes, s.offsets, 6, parts)
    assert [tuple(x) for x in C.tolist()] == [(0, 2)], C


def pin_join_precision(seed: int = 31):
    """MinJoin never outputs a false positive (Sec. 3): the output is a subset
    of the brute-force all-pairs truth, with the true edit distances."""
    s = synth.random_set(seed, n=150, min_len=40, max_len=80, K=6, T=6, families=10, rate=0.04)
    res = oracle.minjoin(s.bytes, s.offsets, K=6, T=6, threads=2)
    truth = {}
    for i in range(s.n):
        for j in range(i + 1, s.n):
            d = oracle.ed_full(s.string(i), s.string(j))
            if d <= 6:
                truth[(i, j)] = d
    got = {tuple(pq): int(d) for pq, d in zip(res.pairs.tolist(), res.ed.tolist())}
    for pq, d in got.items():
        assert truth.get(pq) == d, (pq, d, truth.get(pq))
    return len(got), len(truth)


ALL_PINS = [
    ("worked_example", pin_worked_example),
    ("ed_textbook", pin_ed_textbook),
    ("ed_bfs", pin_ed_bfs),
    ("ed_planted", pin_ed_planted),
    ("ed_band_cutoff", pin_ed_band_cutoff),
    ("q_rule", pin_q_rule),
    ("radius", pin_radius),
    ("anchor_shape", pin_anchor_shape),
    ("anchor_edges", pin_anchor_edges),
    ("hash_injective", pin_hash_is_injective),
    ("candidates_definition", pin_candidates_definition),
    ("join_eviction_order", pin_join_eviction_order),
    ("join_precision", pin_join_precision),
]
