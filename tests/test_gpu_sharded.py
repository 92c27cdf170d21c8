"""The sharded join on the GPU: the library's entry points for it (global
alphabet, candidates from given records, pair dedup) against the oracle, and
the whole sharded join with 2 and 3 shards run as threads of one process on
cuda:0 (each shard its own context; the exchanges in host memory, no kernel
waits on another), whose union must be the single join's output."""
import threading

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1810_08833_gb300 import build
    build.build()


def _reference(s):
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
    return {(int(a), int(b)): int(e) for (a, b), e in zip(ref.pairs.tolist(), ref.ed.tolist())}


def _shard(s, rank, world):
    import torch
    from paper_1810_08833_gb300.sharded import Shard
    cut = np.linspace(0, s.n, world + 1).astype(np.int64)
    lo, hi = int(cut[rank]), int(cut[rank + 1])
    off = s.offsets[lo:hi + 1] - s.offsets[lo]
    data = s.bytes[s.offsets[lo]:s.offsets[hi]]
    return Shard(torch.from_numpy(np.ascontiguousarray(data)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(off)).cuda(), lo)


def _mixed_alphabet():
    s = synth.random_set(77, n=240, min_len=20, max_len=300, K=6, T=6, families=20, rate=0.03)
    data = s.bytes.copy()
    data[s.offsets[3]:s.offsets[3] + 40:7] = ord("N")
    return synth.StringSet(s.name, data, s.offsets, s.K, s.T, s.family)


CASES = {"config1": lambda: synth.make_config(1), "mixed_alphabet": _mixed_alphabet,
         "config4_200roots": lambda: synth.make_config(4, n_roots=200)}


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_sharded_join_on_one_gpu(built, name, world):
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300.sharded import GpuBackend, LocalGroup, sharded_join
    s = CASES[name]()
    group = LocalGroup(world)
    res, errors = [None] * world, []

    def run(r):
        try:
            with mj.Context(0) as ctx:
                i, j, ed, _ = sharded_join(group.comm(r), GpuBackend(ctx), _shard(s, r, world), mj.params(s.K, T=s.T))
                res[r] = (i.cpu().tolist(), j.cpu().tolist(), ed.cpu().tolist())
        except BaseException as e:   # surfaced below
            errors.append(e)
            group._barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    got = {}
    for i, j, ed in res:
        for a, b, e in zip(i, j, ed):
            assert (a, b) not in got
            got[(a, b)] = e
    assert got == _reference(s)


def test_candidates_from_records_match_the_join(built):
    import torch
    import paper_1810_08833_gb300 as mj
    s = synth.make_config(4, n_roots=300)
    data, off = to_device(s)
    p = mj.params(s.K, T=s.T)
    with mj.Context(0) as ctx:
        sid, pos, ln, key = ctx.partition(data, off, p)
        lens = (off[1:] - off[:-1]).to(torch.int32)
        slen = lens[sid.long()].contiguous()
        # records in any order
        perm = torch.randperm(sid.numel(), generator=torch.Generator().manual_seed(3)).cuda()
        ci, cj = ctx.candidates_records(sid[perm].contiguous(), pos[perm].contiguous(), ln[perm].contiguous(),
                                        key[perm].contiguous(), slen[perm].contiguous(), s.n, p)
        wi, wj = ctx.candidates(data, off, p)
        assert torch.equal(ci, wi) and torch.equal(cj, wj)
        with pytest.raises(mj.MinJoinError):   # an id beyond n_strings
            ctx.candidates_records(sid, pos, ln, key, slen, int(sid.max().item()), p)


def test_pairs_unique(built):
    import torch
    import paper_1810_08833_gb300 as mj
    rng = np.random.Generator(np.random.PCG64(5))
    a = rng.integers(0, 500, 20000).astype(np.int32)
    b = rng.integers(0, 500, 20000).astype(np.int32)
    want = np.unique(np.stack([np.minimum(a, b), np.maximum(a, b)], 1), axis=0)
    with mj.Context(0) as ctx:
        ci, cj = ctx.pairs_unique(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 500)
        got = np.stack([ci.cpu().numpy(), cj.cpu().numpy()], 1)
        assert np.array_equal(got, want)
        with pytest.raises(mj.MinJoinError):
            ctx.pairs_unique(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 400)


def test_fixed_alphabet_is_checked_and_cleared(built):
    import paper_1810_08833_gb300 as mj
    s = synth.make_config(1, n_roots=5)
    data, off = to_device(s)
    present = np.zeros(256, dtype=bool)
    present[list(b"ACG")] = True   # T missing
    with mj.Context(0) as ctx:
        ctx.set_alphabet(present, 10_000)
        with pytest.raises(mj.MinJoinError):
            ctx.derive(data, off, mj.params(s.K, T=s.T))
        present[ord("T")] = True
        present[ord("N")] = True
        ctx.set_alphabet(present, 10_000)
        d = ctx.derive(data, off, mj.params(s.K, T=s.T))
        assert d["sigma"] == 5 and d["bits"] == 3 and d["N"] == 10_000 and d["input_max_len"] == 500
        ctx.set_alphabet(None)
        d = ctx.derive(data, off, mj.params(s.K, T=s.T))
        assert d["sigma"] == 4 and d["N"] == 500
