"""Length-bucketed, autotuned, graph-captured verification (the batched
verifier): every plan gives the oracle's distances."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build
    build.build()
    c = mj.Context(0)
    yield c
    c.close()


def _mixed_lengths(seed, K, count):
    """Pairs whose shorter lengths span several power-of-two buckets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    strs, pairs = [], []
    for t in range(count):
        L = int(np.exp(rng.uniform(np.log(K // 2 + 2), np.log(8 * K + 64))))
        a = synth.DNA[rng.integers(0, 4, size=L)]
        b = synth.mutate(rng, a, float(rng.uniform(0.0, 1.5 * K / max(L, 1))), synth.DNA)
        strs += [a.tobytes(), b.tobytes()]
        pairs.append((2 * t, 2 * t + 1))
    return synth.from_strings(strs, K=K, T=K), np.asarray(pairs, dtype=np.int64)


@pytest.mark.parametrize("K", [40, 300])
def test_tuned_plans_match_oracle(ctx, K):
    import torch
    import paper_1810_08833_gb300 as mj
    s, pairs = _mixed_lengths(50 + K, K, 300 if K < 100 else 80)
    want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    stream = torch.cuda.Stream()   # graph capture needs a stream of its own
    rep = ctx.autotune_verify(data, off, i, j, K, sample=64, stream=stream)
    assert len(rep["buckets"]) >= 2
    try:
        for batching in (0, 1):
            for graph in (0, 1):
                ctx.set_verify_config(mj.MJ_VERIFY_KERNEL_TUNED, 0, batching, graph)
                for _ in range(3):   # uncaptured, captured, replayed
                    with torch.cuda.stream(stream):
                        got = ctx.verify(data, off, i, j, K, stream=stream)
                    stream.synchronize()
                    assert np.array_equal(got.cpu().numpy().astype(np.int64), want), (batching, graph)
    finally:
        ctx.set_verify_config(0, 0, 0, 0)


def test_graph_recaptures_on_new_inputs(ctx):
    import torch
    import paper_1810_08833_gb300 as mj
    ctx.set_verify_config(mj.MJ_VERIFY_KERNEL_AUTO, 0, 0, 1)
    try:
        for seed in (61, 62):
            s, pairs = _mixed_lengths(seed, 60, 200)
            want = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, 60)
            data, off = to_device(s)
            i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
            j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
            stream = torch.cuda.Stream()
            for _ in range(3):
                with torch.cuda.stream(stream):
                    got = ctx.verify(data, off, i, j, 60, stream=stream)
                stream.synchronize()
                assert np.array_equal(got.cpu().numpy().astype(np.int64), want), seed
    finally:
        ctx.set_verify_config(0, 0, 0, 0)


def test_graph_after_buffers_grow(ctx):
    """Inputs verified again from the same device tensors after a larger input
    grew the context's buffers (code bytes, bit-planes, per-string table):
    the graph captured for them reads the old buffers, so it must be captured
    again, and the distances stay the oracle's."""
    import torch
    import paper_1810_08833_gb300 as mj
    ctx.set_verify_config(mj.MJ_VERIFY_KERNEL_AUTO, 0, 0, 1)
    try:
        small = _mixed_lengths(71, 60, 200)
        large = _mixed_lengths(72, 400, 600)
        inputs = []
        for s, pairs in (small, large):
            data, off = to_device(s)
            i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
            j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
            inputs.append((data, off, i, j, oracle.ed_band_pairs(s.bytes, s.offsets, pairs, 60)))
        stream = torch.cuda.Stream()
        for which in (0, 1, 0):
            data, off, i, j, want = inputs[which]
            for _ in range(3):
                with torch.cuda.stream(stream):
                    got = ctx.verify(data, off, i, j, 60, stream=stream)
                stream.synchronize()
                assert np.array_equal(got.cpu().numpy().astype(np.int64), want), which
    finally:
        ctx.set_verify_config(0, 0, 0, 0)


def test_join_with_tuned_graph_plan(ctx):
    import paper_1810_08833_gb300 as mj
    s = synth.make_config(3, n_roots=6)
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
    data, off = to_device(s)
    import torch
    stream = torch.cuda.Stream()
    ci, cj = ctx.candidates(data, off, mj.params(s.K, T=s.T), stream=stream)
    ctx.autotune_verify(data, off, ci, cj, s.K, sample=32, stream=stream)
    ctx.set_verify_config(mj.MJ_VERIFY_KERNEL_TUNED, 0, 0, 1)
    try:
        for _ in range(3):
            with torch.cuda.stream(stream):
                oi, oj, oe = ctx.join(data, off, mj.params(s.K, T=s.T), stream=stream)
            stream.synchronize()
            got = np.stack([t.cpu().numpy() for t in (oi, oj, oe)], 1).astype(np.int64)
            assert np.array_equal(got, np.concatenate([ref.pairs, ref.ed[:, None]], 1))
    finally:
        ctx.set_verify_config(0, 0, 0, 0)
