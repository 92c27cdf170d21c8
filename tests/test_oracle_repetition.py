"""Pins of the oracle's parallel repetition (Sec. 2.2, Thm 1): the union of
the partitions under R independent random functions Pi.  Checked against
what the definition fixes: R = 1 is the plain partition; each repetition
tiles every string on its own; repetitions differ; the candidate and output
sets only grow with R; every output is a true pair (brute force over all
pairs) and recall does not fall."""
import numpy as np

import oracle
import synth


def _set():
    return synth.make_config(1, n_roots=20)   # 200 strings of 500 bp, K = 10


def test_one_repetition_is_the_plain_partition():
    s = _set()
    p = oracle.derive_params(s.bytes, s.offsets, K=s.K, T=s.T)
    a = oracle.partition(s.bytes, s.offsets, p)
    b = oracle.partition_repeated(s.bytes, s.offsets, p, 1)
    for x, y in ((a.sid, b.sid), (a.pos, b.pos), (a.len, b.len), (a.n_anchor, b.n_anchor)):
        assert np.array_equal(x, y)


def test_each_repetition_tiles_every_string_and_they_differ():
    s = _set()
    p = oracle.derive_params(s.bytes, s.offsets, K=s.K, T=s.T)
    R = 3
    u = oracle.partition_repeated(s.bytes, s.offsets, p, R)
    L = s.lengths()
    differ = 0
    for i in range(s.n):
        sel = u.sid == i
        pos, ln = u.pos[sel], u.len[sel]
        # the union is R tilings of [0, |s|): every position is covered R times
        cover = np.zeros(L[i], np.int64)
        for a, b in zip(pos, ln):
            cover[a:a + b] += 1
        assert np.all(cover == R), i
        assert int(ln.sum()) == R * L[i]
        first = oracle.partition(s.bytes, s.offsets, p, lo=i, hi=i + 1)
        second = oracle.partition(s.bytes, s.offsets,
                                  oracle.dataclasses.replace(p, seed=oracle.repetition_seed(p.seed, 1)),
                                  lo=i, hi=i + 1)
        differ += not np.array_equal(first.pos, second.pos)
    assert differ > s.n // 2   # independent Pi functions cut most strings differently


def test_seeds_follow_the_stated_rule():
    assert oracle.repetition_seed(0x5EED, 0) == 0x5EED
    assert oracle.repetition_seed(0x5EED, 2) == (0x5EED + 2 * 0x9E3779B97F4A7C15) % (1 << 64)
    assert oracle.repetition_seed((1 << 64) - 1, 1) == 0x9E3779B97F4A7C14


def test_candidates_grow_and_recall_does_not_fall():
    s = _set()
    n = s.n
    iu = np.triu_indices(n, 1)
    allp = np.stack(iu, 1).astype(np.int64)
    ed = oracle.ed_band_pairs(s.bytes, s.offsets, allp, s.K)
    truth = {(int(a), int(b)) for (a, b), e in zip(allp, ed) if e <= s.K}
    prev_c, prev_o, prev_recall = set(), set(), 0.0
    for R in (1, 2, 3):
        r = oracle.minjoin(s.bytes, s.offsets, s.K, T=s.T, repeats=R)
        c = {tuple(x) for x in r.candidates.tolist()}
        o = {tuple(x) for x in r.pairs.tolist()}
        assert prev_c <= c and prev_o <= o
        assert o <= truth
        recall = len(o) / len(truth)
        assert recall >= prev_recall
        prev_c, prev_o, prev_recall = c, o, recall
