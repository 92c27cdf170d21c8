"""Element-wise parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results throughout, so the bar is exact equality: partitions
(sid, pos, len), the deduplicated candidate set, and the (i, j, ED) output.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import edge_set, parity_sets, to_device
from worked_example import load as load_example, table as example_table

pytestmark = pytest.mark.gpu

_cache = {}


def get_set(name, factory):
    if name not in _cache:
        s = factory()
        p = oracle.derive_params(s.bytes, s.offsets, K=s.K, T=s.T)
        _cache[name] = (s, p)
    return _cache[name]


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    c = mj.Context(0)
    yield c
    c.close()


SETS = parity_sets()
IDS = [n for n, _ in SETS]


@pytest.mark.parametrize("name,factory", SETS, ids=IDS)
def test_derived_parameters(ctx, name, factory):
    import paper_1810_08833_gb300 as mj
    s, p = get_set(name, factory)
    data, off = to_device(s)
    d = ctx.derive(data, off, mj.params(s.K, T=s.T))
    assert (d["sigma"], d["bits"], d["q"], d["T"], d["N"]) == (p.sigma, p.bits, p.q, p.T, p.N)
    assert np.array_equal(d["rank"], p.rank)


@pytest.mark.parametrize("name,factory", SETS, ids=IDS)
def test_partition_parity(ctx, name, factory):
    import paper_1810_08833_gb300 as mj
    s, p = get_set(name, factory)
    parts = oracle.partition(s.bytes, s.offsets, p)
    data, off = to_device(s)
    sid, pos, ln, key = ctx.partition(data, off, mj.params(s.K, T=s.T))
    got = np.stack([t.cpu().numpy().astype(np.int64) for t in (sid, pos, ln)], axis=1)
    want = np.stack([parts.sid, parts.pos, parts.len], axis=1)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    # (len, key) separates different partition substrings, and equal
    # substrings (at any offset and alignment) get equal keys
    k = key.cpu().numpy()
    seen, by_sub = {}, {}
    for t in range(0, got.shape[0], max(1, got.shape[0] // 4000)):
        sub = s.bytes[s.offsets[got[t, 0]] + got[t, 1]: s.offsets[got[t, 0]] + got[t, 1] + got[t, 2]].tobytes()
        kk = (int(got[t, 2]), int(k[t]))
        if kk in seen:
            assert seen[kk] == sub
        seen[kk] = sub
        assert by_sub.setdefault(sub, kk) == kk


def test_partition_worked_example(ctx):
    import torch
    import paper_1810_08833_gb300 as mj
    ex = load_example()
    strings = [ex["string"][i] for i in sorted(ex["string"])]
    s = synth.from_strings(strings, K=ex["param"]["K"], T=ex["param"]["T"])
    p = oracle.derive_params(s.bytes, s.offsets, K=4, T=3, q=3)
    tab = torch.from_numpy(example_table(ex, p.rank, p.bits, p.q).astype(np.int64)).cuda()
    data, off = to_device(s)
    prm = mj.params(4, T=3, q=3)
    sid, pos, ln, _ = ctx.partition(data, off, prm, table=tab)
    sid, pos, ln = (t.cpu().numpy() for t in (sid, pos, ln))
    for i, st in enumerate(strings):
        sel = sid == i
        subs = [st[a:a + b] for a, b in zip(pos[sel], ln[sel])]
        assert subs == ex["partition"][i + 1][1]
    ci, cj = ctx.candidates(data, off, prm, table=tab)
    got = sorted(zip(ci.cpu().tolist(), cj.cpu().tolist()))
    assert got == sorted(ex["candidate"])


def test_partition_anchor_edges(ctx):
    import torch
    import paper_1810_08833_gb300 as mj
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "anchor_edges.txt")
    cases = [(l.split()[1].encode(), [x.encode() for x in l.split()[2:]])
             for l in open(path) if l.startswith("edge ")]
    s = synth.from_strings([c[0] for c in cases], K=2, T=2)
    p = oracle.derive_params(s.bytes, s.offsets, K=2, T=2, q=1)
    tab = np.zeros(1 << p.bits, dtype=np.int64)
    for sym, v in zip(b"ABCD", (1, 2, 3, 4)):
        tab[p.rank[sym]] = v
    data, off = to_device(s)
    sid, pos, ln, _ = ctx.partition(data, off, mj.params(2, T=2, q=1), table=torch.from_numpy(tab).cuda())
    sid, pos, ln = (t.cpu().numpy() for t in (sid, pos, ln))
    for i, (st, expect) in enumerate(cases):
        sel = sid == i
        assert [st[a:a + b] for a, b in zip(pos[sel], ln[sel])] == expect


DEDUP = {"auto": 0, "sort": 64, "bitmap": 128}   # MJ_FLAG_DEDUP_SORT, MJ_FLAG_DEDUP_BITMAP


@pytest.mark.parametrize("dedup", sorted(DEDUP))
@pytest.mark.parametrize("name,factory", SETS, ids=IDS)
def test_candidates_parity(ctx, name, factory, dedup):
    import paper_1810_08833_gb300 as mj
    s, p = get_set(name, factory)
    parts = oracle.partition(s.bytes, s.offsets, p)
    want = oracle.candidates(s.bytes, s.offsets, s.K, parts)
    data, off = to_device(s)
    ci, cj = ctx.candidates(data, off, mj.params(s.K, T=s.T, flags=mj.MJ_FLAG_KEY_CHECK | DEDUP[dedup]))
    got = np.stack([ci.cpu().numpy(), cj.cpu().numpy()], axis=1).astype(np.int64)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    st = ctx.stats()
    assert st["key_collisions"] == 0
    assert st["device_flags"] == 0


@pytest.mark.parametrize("dedup", sorted(DEDUP))
@pytest.mark.parametrize("name,factory", SETS, ids=IDS)
def test_join_parity(ctx, name, factory, dedup):
    import paper_1810_08833_gb300 as mj
    s, p = get_set(name, factory)
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
    data, off = to_device(s)
    oi, oj, oe = ctx.join(data, off, mj.params(s.K, T=s.T, flags=DEDUP[dedup]))
    got = np.stack([t.cpu().numpy() for t in (oi, oj, oe)], axis=1).astype(np.int64)
    want = np.concatenate([ref.pairs, ref.ed[:, None]], axis=1)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    st = ctx.stats()
    assert st["n_candidates"] == ref.candidates.shape[0]
    L = s.lengths()
    a, b = ref.candidates[:, 0], ref.candidates[:, 1]
    m, n = np.maximum(L[a], L[b]), np.minimum(L[a], L[b])
    # K-band cells, counted by brute force over columns
    cells = 0
    for mm, nn in zip(m.tolist(), n.tolist()):
        j = np.arange(1, nn + 1)
        cells += int(np.clip(np.minimum(mm, j + s.K) - np.maximum(1, j - s.K) + 1, 0, None).sum())
    assert st["band_cells"] == cells


REPEAT_SETS = [x for x in SETS if x[0] in ("config1", "config4_400roots", "random_mixed", "edge")]


def test_bitmap_reuse_across_joins(ctx):
    """The pair bitmap is cleared by the candidate writer when it is sparse
    (and the next join's marking then skips clearing it) and cleared before
    marking otherwise.  Joins of sparse and dense inputs, growing and
    shrinking, on one context, each equal to the oracle's join."""
    import paper_1810_08833_gb300 as mj
    sets = [synth.random_set(301, n=600, min_len=40, max_len=200, K=6, T=6, families=10, rate=0.03),
            synth.random_set(302, n=300, min_len=40, max_len=200, K=6, T=6, families=60, rate=0.02),
            synth.random_set(303, n=900, min_len=40, max_len=200, K=6, T=6, families=5, rate=0.03),
            synth.random_set(304, n=200, min_len=20, max_len=60, symbols=synth.DNA[:2], K=8, T=8),
            synth.random_set(305, n=900, min_len=40, max_len=200, K=6, T=6, families=30, rate=0.03)]
    for s in sets + sets[::-1]:
        ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
        data, off = to_device(s)
        for flags in (0, mj.MJ_FLAG_DEDUP_BITMAP):
            oi, oj, oe = ctx.join(data, off, mj.params(s.K, T=s.T, flags=flags))
            got = np.stack([t.cpu().numpy() for t in (oi, oj, oe)], axis=1).astype(np.int64)
            want = np.concatenate([ref.pairs, ref.ed[:, None]], axis=1)
            assert np.array_equal(got, want), (s.n, flags)


@pytest.mark.parametrize("name,factory", REPEAT_SETS, ids=[n for n, _ in REPEAT_SETS])
def test_repetition_parity(ctx, name, factory):
    """Parallel repetition (Sec. 2.2): the partitions under R seeds equal the
    oracle's union, and the join over that union equals the oracle's."""
    import paper_1810_08833_gb300 as mj
    s, p = get_set(name, factory)
    data, off = to_device(s)
    want = oracle.partition_repeated(s.bytes, s.offsets, p, 3)
    sid, pos, ln, _ = ctx.partition(data, off, mj.params(s.K, T=s.T, repeats=3))
    got = np.stack([t.cpu().numpy().astype(np.int64) for t in (sid, pos, ln)], axis=1)
    w = np.stack([want.sid, want.pos, want.len], axis=1)
    got, w = got[np.lexsort(got.T[::-1])], w[np.lexsort(w.T[::-1])]
    assert got.shape == w.shape and np.array_equal(got, w)
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T, repeats=2)
    ctx.band_init(seed=5)   # any network gives the plain output
    for mode in (mj.MJ_VERIFY_PLAIN, mj.MJ_VERIFY_LEARNED):
        oi, oj, oe = ctx.join(data, off, mj.params(s.K, T=s.T, repeats=2, verify_mode=mode))
        res = np.stack([t.cpu().numpy() for t in (oi, oj, oe)], axis=1).astype(np.int64)
        assert np.array_equal(res, np.concatenate([ref.pairs, ref.ed[:, None]], axis=1))
        st = ctx.stats()
        assert st["n_candidates"] == ref.candidates.shape[0] and st["device_flags"] == 0


def test_repetition_rejects_bad_counts(ctx):
    import paper_1810_08833_gb300 as mj
    s = synth.make_config(1, n_roots=2)
    data, off = to_device(s)
    for r in (0, 65):
        with pytest.raises(mj.MinJoinError):
            ctx.join(data, off, mj.params(s.K, T=s.T, repeats=r))


@pytest.mark.parametrize("which", ["config1", "config2_400roots"])
def test_join_host_matches_device(ctx, which):
    """Host buffers in (a small input, and config 2 with 400 families, 20 MB)
    give the device join's output."""
    import paper_1810_08833_gb300 as mj
    s = get_set("config1", SETS[0][1])[0] if which == "config1" else synth.make_config(2, n_roots=400)
    data, off = to_device(s)
    oi, oj, oe = ctx.join(data, off, mj.params(s.K, T=s.T))
    hi, hj, he = ctx.join_host(s.bytes, s.offsets, mj.params(s.K, T=s.T))
    assert oi.numel() > 0
    assert np.array_equal(hi, oi.cpu().numpy().astype(np.uint32))
    assert np.array_equal(hj, oj.cpu().numpy().astype(np.uint32))
    assert np.array_equal(he, oe.cpu().numpy().astype(np.uint32))


def test_join_empty_inputs(ctx):
    import torch
    import paper_1810_08833_gb300 as mj
    for strs in ([], [b""], [b"", b""], [b"A"], [b"ACGT", b"ACGT"]):
        s = synth.from_strings(strs, K=2, T=2)
        data, off = to_device(s)
        oi, oj, oe = ctx.join(data, off, mj.params(2, T=2))
        ref = oracle.minjoin(s.bytes, s.offsets, K=2, T=2)
        got = np.stack([t.cpu().numpy() for t in (oi, oj, oe)], axis=1).astype(np.int64).reshape(-1, 3)
        want = np.concatenate([ref.pairs, ref.ed[:, None]], axis=1).reshape(-1, 3)
        assert np.array_equal(got, want), strs
    torch.cuda.synchronize()


# ---------------------------------------------------------------- verification

def _pairs_set(seed, K, count, rng_len):
    """Strings and pairs whose edit distances straddle K: planted edits at
    rates that put ED near K, exact length differences K and K+1, equal
    strings and empty strings."""
    rng = np.random.Generator(np.random.PCG64(seed))
    strs, pairs = [], []
    lo, hi = rng_len
    for t in range(count):
        L = int(rng.integers(lo, hi + 1))
        a = synth.DNA[rng.integers(0, 4, size=L)]
        kind = t % 5
        if kind == 0:      # ED near K
            rate = min(0.9, max(0.0, (K + rng.integers(-3, 4)) / max(1, L) / 0.9))
            b = synth.mutate(rng, a, rate, synth.DNA)
        elif kind == 1:    # length difference exactly K (ED = K)
            b = a[:max(0, L - K)]
        elif kind == 2:    # length difference K + 1
            b = a[:max(0, L - K - 1)]
        elif kind == 3:    # light edits
            b = synth.mutate(rng, a, 0.2 * K / max(1, L), synth.DNA)
        else:              # unrelated
            b = synth.DNA[rng.integers(0, 4, size=int(rng.integers(max(0, L - K), L + K + 1)))]
        strs += [a.tobytes(), b.tobytes()]
        pairs.append((2 * t, 2 * t + 1))
    strs += [b"", b"", b"ACGT" * 10]
    n = len(strs)
    pairs += [(n - 3, n - 2), (n - 3, n - 1), (n - 1, n - 1), (0, 0)]
    return synth.from_strings(strs, K=K, T=K), np.array(pairs, dtype=np.int64)


@pytest.mark.parametrize("K", [0, 1, 2, 5, 10, 31, 32, 33, 40, 63, 64, 65, 75, 100, 127, 128, 200, 255, 256, 300,
                               511, 1000])
def test_verify_parity(ctx, K):
    import torch
    lens = (0, 3 * K + 40) if K < 300 else (K, 3 * K)
    count = 120 if K < 300 else 30
    s, pairs = _pairs_set(1000 + K, K, count, lens)
    want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    ed = ctx.verify(data, off, i, j, K)
    got = ed.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    # swapping the pair's order changes nothing
    ed2 = ctx.verify(data, off, j, i, K)
    assert np.array_equal(ed2.cpu().numpy().astype(np.int64), want)


def test_verify_exhaustive_small_alphabet(ctx):
    import itertools
    import torch
    strs = [b""] + [bytes(t) for L in range(1, 6) for t in itertools.product(b"AC", repeat=L)]
    s = synth.from_strings(strs, K=3, T=3)
    idx = np.array([(a, b) for a in range(len(strs)) for b in range(len(strs))], dtype=np.int64)
    data, off = to_device(s)
    i = torch.from_numpy(idx[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(idx[:, 1].astype(np.int32)).cuda()
    for K in (0, 1, 2, 3, 6):
        want = oracle.ed_band_pairs(s.bytes, s.offsets, idx, K)
        got = ctx.verify(data, off, i, j, K).cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want), K


def test_verify_per_pair_band(ctx):
    import torch
    s, pairs = _pairs_set(77, 40, 200, (0, 200))
    rng = np.random.Generator(np.random.PCG64(3))
    k = rng.integers(0, 41, size=pairs.shape[0])
    want = np.array([oracle.ed_band(s.string(a), s.string(b), int(kk)) for (a, b), kk in zip(pairs, k)])
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    kt = torch.from_numpy(k.astype(np.int32)).cuda()
    got = ctx.verify(data, off, i, j, 40, k=kt).cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want)


def test_verify_other_alphabets(ctx):
    import torch
    rng = np.random.Generator(np.random.PCG64(9))
    for symbols in (synth.PROTEIN, synth.PRINTABLE, np.arange(256, dtype=np.uint8)):
        strs, pairs = [], []
        for t in range(150):
            L = int(rng.integers(0, 500))
            a = symbols[rng.integers(0, symbols.shape[0], size=L)]
            b = synth.mutate(rng, a, float(rng.uniform(0, 0.1)), symbols)
            strs += [a.tobytes(), b.tobytes()]
            pairs.append((2 * t, 2 * t + 1))
        s = synth.from_strings(strs, K=30, T=30)
        pairs = np.array(pairs, np.int64)
        data, off = to_device(s)
        i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
        j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
        for K in (7, 30, 70):
            want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
            got = ctx.verify(data, off, i, j, K).cpu().numpy().astype(np.int64)
            assert np.array_equal(got, want), (symbols.shape, K)


DIGIT_ALPHABETS = {"dna": (lambda: synth.DNA, 2), "protein": (lambda: synth.PROTEIN, 5),
                   "text": (lambda: synth.PRINTABLE, 7)}


@pytest.mark.parametrize("alphabet", sorted(DIGIT_ALPHABETS))
def test_diag_digit_tables(ctx, alphabet):
    """The per-thread kernel with digit tables (2, 5 and 7 bit-planes), forced,
    at band widths of 1 to 5 words, with the last string of the input in many
    pairs (B's bytes read near the end of the buffer)."""
    import torch
    import paper_1810_08833_gb300 as mj
    symbols_of, bits = DIGIT_ALPHABETS[alphabet]
    symbols = symbols_of()
    rng = np.random.Generator(np.random.PCG64(41 + bits))
    strs = []
    for t in range(120):
        L = int(rng.integers(0, 700))
        a = symbols[rng.integers(0, symbols.shape[0], size=L)]
        strs += [a.tobytes(), synth.mutate(rng, a, float(rng.uniform(0, 0.2)), symbols).tobytes()]
    strs.append(symbols[rng.integers(0, symbols.shape[0], size=333)].tobytes())
    s = synth.from_strings(strs, K=40, T=40)
    last = s.n - 1
    pairs = [(2 * t, 2 * t + 1) for t in range(120)] + [(t, last) for t in range(0, 2 * 120, 3)]
    pairs = np.array(pairs, np.int64)
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    assert ctx.derive(data, off, mj.params(40, T=40))["bits"] == bits
    ctx.set_verify_config(1, 0)
    try:
        for K in (7, 31, 40, 75, 100, 127, 150):
            want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
            got = ctx.verify(data, off, i, j, K).cpu().numpy().astype(np.int64)
            assert np.array_equal(got, want), (K, np.nonzero(got != want)[0][:10])
            got = ctx.verify(data, off, j, i, K).cpu().numpy().astype(np.int64)
            assert np.array_equal(got, want), K
    finally:
        ctx.set_verify_config(0, 0)


def test_verify_rejects_bad_ids(ctx):
    import torch
    import paper_1810_08833_gb300 as mj
    s = synth.from_strings([b"ACGT", b"ACGA"], K=2, T=2)
    data, off = to_device(s)
    i = torch.tensor([0, 5], dtype=torch.int32, device="cuda")
    j = torch.tensor([1, 1], dtype=torch.int32, device="cuda")
    ed = ctx.verify(data, off, i, j, 2)
    torch.cuda.synchronize()
    assert ed.cpu().tolist() == [1, 3]
    assert ctx.device_flags() & 1   # the out-of-range id is reported
    ctx.verify(data, off, j[:1], i[:1], 2)
    assert ctx.device_flags() == 0


KERNEL_CASES = [(K, 1, 0) for K in (5, 40, 100, 255, 600)] + \
               [(K, 2, 0) for K in (0, 1, 7, 40, 63, 64, 100, 255, 256, 600, 1000)] + \
               [(40, 2, 8), (100, 2, 16), (100, 2, 32), (255, 2, 32)]


@pytest.mark.parametrize("K,kernel,lanes", KERNEL_CASES,
                         ids=[f"K{K}-{'diag' if k == 1 else 'wave'}{l or ''}" for K, k, l in KERNEL_CASES])
def test_verify_kernel_parity(ctx, K, kernel, lanes):
    """Each verification kernel, forced, agrees with the oracle's banded DP."""
    import torch
    lens = (0, 3 * K + 40) if K < 300 else (K, 3 * K)
    count = 100 if K < 300 else 24
    s, pairs = _pairs_set(2000 + K, K, count, lens)
    want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    ctx.set_verify_config(kernel, lanes)
    try:
        got = ctx.verify(data, off, i, j, K).cpu().numpy().astype(np.int64)
        got_swapped = ctx.verify(data, off, j, i, K).cpu().numpy().astype(np.int64)
    finally:
        ctx.set_verify_config(0, 0)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert np.array_equal(got_swapped, want)


def test_wavefront_other_alphabets(ctx):
    import torch
    rng = np.random.Generator(np.random.PCG64(19))
    for symbols in (synth.PROTEIN, synth.PRINTABLE):
        strs, pairs = [], []
        for t in range(60):
            L = int(rng.integers(0, 900))
            a = symbols[rng.integers(0, symbols.shape[0], size=L)]
            b = synth.mutate(rng, a, float(rng.uniform(0, 0.15)), symbols)
            strs += [a.tobytes(), b.tobytes()]
            pairs.append((2 * t, 2 * t + 1))
        s = synth.from_strings(strs, K=80, T=80)
        pairs = np.array(pairs, np.int64)
        data, off = to_device(s)
        i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
        j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
        want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, 80)
        ctx.set_verify_config(2, 0)
        try:
            got = ctx.verify(data, off, i, j, 80).cpu().numpy().astype(np.int64)
        finally:
            ctx.set_verify_config(0, 0)
        assert np.array_equal(got, want)
