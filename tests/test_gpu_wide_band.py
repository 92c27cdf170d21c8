"""Verification with bands wider than one warp holds (K >= 1025): one CTA of
several warps per pair (Sec. 3's banded DP; the paper's scalability study
runs K up to 20% of string lengths of 20,000, Sec. 4).  Every shape agrees
with the oracle's banded DP, and the autotuner picks among them."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu

WAVEFRONT, TUNED = 2, 3


@pytest.fixture(scope="module")
def ctx():
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build
    build.build()
    c = mj.Context(0)
    yield c
    c.close()


def _wide_pairs(seed, K, count, lo, hi):
    """Long DNA pairs whose distances straddle K: planted edits near K, length
    differences K and K + 1, light edits and unrelated strings."""
    rng = np.random.Generator(np.random.PCG64(seed))
    strs, pairs = [], []
    for t in range(count):
        L = int(rng.integers(lo, hi + 1))
        a = synth.DNA[rng.integers(0, 4, size=L)]
        kind = t % 5
        if kind == 0:
            rate = min(0.9, (K + int(rng.integers(-40, 41))) / L / 0.8)
            b = synth.mutate(rng, a, rate, synth.DNA)
        elif kind == 1:
            b = a[:L - K]
        elif kind == 2:
            b = a[:L - K - 1]
        elif kind == 3:
            b = synth.mutate(rng, a, 0.3 * K / L, synth.DNA)
        else:
            b = synth.DNA[rng.integers(0, 4, size=int(rng.integers(L - K, L + K + 1)))]
        strs += [a.tobytes(), b.tobytes()]
        pairs.append((2 * t, 2 * t + 1))
    strs += [b"", b"ACGT" * 300]
    n = len(strs)
    pairs += [(n - 2, n - 1), (n - 1, n - 1), (n - 2, n - 2)]
    return synth.from_strings(strs, K=K, T=K // 5), np.asarray(pairs, dtype=np.int64)


_cache = {}


def _case(K):
    if K not in _cache:
        lo, hi = {1025: (2000, 8000), 2000: (5000, 12000), 4000: (10000, 20000)}[K]
        s, pairs = _wide_pairs(300 + K, K, 20, lo, hi)
        want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K, cutoff=True)
        _cache[K] = (s, pairs, want)
    return _cache[K]


def _verify(ctx, s, pairs, K, kernel=0, lanes=0):
    import torch
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    ctx.set_verify_config(kernel, lanes)
    try:
        got = ctx.verify(data, off, i, j, K).cpu().numpy().astype(np.int64)
        swapped = ctx.verify(data, off, j, i, K).cpu().numpy().astype(np.int64)
    finally:
        ctx.set_verify_config(0, 0)
    return got, swapped


@pytest.mark.parametrize("K", [1025, 2000, 4000])
def test_wide_band_default_kernel(ctx, K):
    s, pairs, want = _case(K)
    assert np.any(want <= K) and np.any(want > K)
    got, swapped = _verify(ctx, s, pairs, K)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert np.array_equal(swapped, want)
    assert ctx.stats()["device_flags"] == 0


@pytest.mark.parametrize("K,lanes", [(1025, 64), (1025, 256), (2000, 128), (2000, 1024), (4000, 128), (4000, 512)])
def test_wide_band_forced_shapes(ctx, K, lanes):
    s, pairs, want = _case(K)
    got, swapped = _verify(ctx, s, pairs, K, WAVEFRONT, lanes)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert np.array_equal(swapped, want)


@pytest.mark.parametrize("K,lanes", [(100, 64), (300, 128), (1000, 64)])
def test_cta_kernel_on_narrow_bands(ctx, K, lanes):
    """The CTA form also runs bands a warp could hold: many short pairs, each
    taking and releasing the whole CTA."""
    from test_gpu_parity import _pairs_set
    lens = (0, 3 * K + 40) if K < 300 else (K, 3 * K)
    s, pairs = _pairs_set(4000 + K, K, 60 if K < 1000 else 20, lens)
    want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
    got, swapped = _verify(ctx, s, pairs, K, WAVEFRONT, lanes)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
    assert np.array_equal(swapped, want)


def test_too_few_lanes_is_unsupported(ctx):
    import paper_1810_08833_gb300 as mj
    s, pairs, _ = _case(2000)
    with pytest.raises(mj.MinJoinError):
        _verify(ctx, s, pairs, 2000, WAVEFRONT, 32)
    with pytest.raises(mj.MinJoinError):
        _verify(ctx, s, pairs, 4000, WAVEFRONT, 64)


def test_autotuner_picks_among_cta_shapes(ctx):
    import torch
    import paper_1810_08833_gb300 as mj
    K = 2000
    s, pairs, want = _case(K)
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    stream = torch.cuda.Stream()
    rep = ctx.autotune_verify(data, off, i, j, K, sample=64, stream=stream)
    lanes = [l for k, l in rep["candidates"]]
    assert all(k == WAVEFRONT for k, _ in rep["candidates"])
    assert lanes[0] == 64 and lanes == [64 * 2 ** x for x in range(len(lanes))]
    for b in rep["buckets"].values():
        assert b["kernel"] == WAVEFRONT and b["lanes"] in lanes
    try:
        for graph in (0, 1):
            ctx.set_verify_config(TUNED, 0, 0, graph)
            for _ in range(3):
                with torch.cuda.stream(stream):
                    got = ctx.verify(data, off, i, j, K, stream=stream)
                stream.synchronize()
                assert np.array_equal(got.cpu().numpy().astype(np.int64), want), graph
    finally:
        ctx.set_verify_config(0, 0, 0, 0)
