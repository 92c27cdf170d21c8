"""The sharded join's exchanges on the CPU (no GPU): strings split by id range
over two gloo ranks (and over three in-process ranks), the library's calls
stood in for by the oracle (tests/shard_backends.py).  The union of the
ranks' outputs must be the single-rank join's output, pair for pair with the
same distances, and no pair may come from two ranks (Alg. 3's output set)."""
import os
import socket
import sys
import threading

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(name):
    if name == "config1":
        return synth.make_config(1)
    s = synth.random_set(77, n=240, min_len=20, max_len=300, K=6, T=6, families=20, rate=0.03)
    if name == "mixed_alphabet":
        # a byte value present only in the first strings: the shards must
        # agree on the global alphabet (and so on the rank codes and Pi)
        data = s.bytes.copy()
        data[s.offsets[3]:s.offsets[3] + 40:7] = ord("N")
        s = synth.StringSet(s.name, data, s.offsets, s.K, s.T, s.family)
    return s


def _shard(s, rank, world):
    import torch
    from paper_1810_08833_gb300.sharded import Shard
    cut = np.linspace(0, s.n, world + 1).astype(np.int64)
    lo, hi = int(cut[rank]), int(cut[rank + 1])
    off = s.offsets[lo:hi + 1] - s.offsets[lo]
    data = s.bytes[s.offsets[lo]:s.offsets[hi]]
    return Shard(torch.from_numpy(np.ascontiguousarray(data)), torch.from_numpy(np.ascontiguousarray(off)), lo)


def _rank_main(rank, world, port, name, out):
    import torch.distributed as dist
    sys.path[:0] = [ROOT, HERE]
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300.sharded import TorchComm, sharded_join
    from shard_backends import OracleBackend
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _workload(name)
        i, j, ed, info = sharded_join(TorchComm(), OracleBackend(), _shard(s, rank, world), mj.params(s.K, T=s.T))
        out[rank] = (i.tolist(), j.tolist(), ed.tolist(), info)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _reference(name):
    s = _workload(name)
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
    return {(int(a), int(b)): int(e) for (a, b), e in zip(ref.pairs.tolist(), ref.ed.tolist())}


def _union(results):
    got = {}
    for i, j, ed in results:
        for a, b, e in zip(i, j, ed):
            assert (a, b) not in got, "a pair came from two ranks"
            got[(a, b)] = e
    return got


@pytest.mark.parametrize("name", ["config1", "mixed", "mixed_alphabet"])
def test_two_gloo_ranks_equal_the_single_join(name):
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, name, out), nprocs=world, join=True,
                           start_method="spawn")
        got = dict(out)
    assert sorted(got) == [0, 1]
    assert _union([got[r][:3] for r in (0, 1)]) == _reference(name)
    for r in (0, 1):   # both ranks did part of the work
        assert got[r][3]["records_in"] > 0


def test_three_local_ranks_equal_the_single_join():
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300.sharded import LocalGroup, sharded_join
    from shard_backends import OracleBackend
    s = _workload("mixed")
    group = LocalGroup(3)
    res = [None] * 3
    errors = []

    def run(r):
        try:
            i, j, ed, _ = sharded_join(group.comm(r), OracleBackend(), _shard(s, r, 3), mj.params(s.K, T=s.T))
            res[r] = (i.tolist(), j.tolist(), ed.tolist())
        except BaseException as e:   # surfaced below
            errors.append(e)
            group._barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert _union(res) == _reference("mixed")
