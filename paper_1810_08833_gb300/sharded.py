"""The MinJoin join sharded over several processes, one GPU each.

Every step of the path runs in the library on each rank; this module only
moves data between ranks.  With G ranks, rank r holds the strings with global
ids first_r .. first_r + n_r - 1 (contiguous id ranges):

  1. global parameters (Sec. 2.2): the byte values present and the longest
     length, reduced over the ranks, fixed on every rank's context
     (mj_set_alphabet), so all ranks derive the same rank codes, q and Pi;
  2. every rank partitions its own strings (Alg. 1-2);
  3. one all-to-all sends every partition record to the rank owning its
     (length, key) class, so each group of equal partitions is whole on one
     rank (Alg. 3 groups by partition substring);
  4. every rank joins its groups under both filters and deduplicates
     (mj_candidates_records);
  5. a second all-to-all sends every candidate pair to the rank owning the
     pair; that rank deduplicates C (mj_pairs_unique);
  6. the strings are gathered on every rank and each rank verifies its own
     pairs (Sec. 3);
  7. each rank returns its output pairs; the ranks' outputs are disjoint.

The compute steps come from a backend (GpuBackend: the library on this
process's GPU); the exchanges from a communicator (TorchComm:
torch.distributed, NCCL on GPUs or gloo on CPU; LocalGroup: shards run as
threads of one process).  Owners are a fixed mix of the class or pair, the
same on every rank.
"""
from __future__ import annotations

import dataclasses
import threading

import numpy as np

MIX = 0x9E3779B97F4A7C15


def _mix_owner(x, world: int):
    """Owner rank of int64 tensor values x (a fixed multiplicative mix)."""
    import torch
    h = x * torch.tensor(MIX - (1 << 64), dtype=torch.int64, device=x.device)   # wraps modulo 2^64
    return ((h >> 33) & 0x7FFFFFFF) % world


@dataclasses.dataclass
class Shard:
    """This rank's strings: bytes and offsets (offsets[0] = 0), global ids
    first .. first + n - 1."""
    bytes: object
    offsets: object
    first: int = 0

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0]) - 1


# ------------------------------------------------------------ communicators

class TorchComm:
    """Collectives of the default torch.distributed process group (NCCL for
    CUDA tensors, gloo for CPU tensors)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def all_gather_int(self, v: int) -> list:
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([int(v)], dtype=torch.int64, device=dev)
        out = [torch.zeros_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t)
        return [int(x.item()) for x in out]

    def all_reduce_max(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t

    def all_to_all(self, x, send_counts: list):
        """Rows x[...] grouped by destination (send_counts[d] rows to rank d)
        -> the rows every rank sent here, in rank order."""
        import torch
        recv = self.all_to_all_counts(send_counts)
        out = torch.empty((sum(recv),) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
        self.dist.all_to_all_single(out, x.contiguous(), recv, send_counts)
        return out

    def all_to_all_counts(self, send_counts: list) -> list:
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        s = torch.tensor(send_counts, dtype=torch.int64, device=dev)
        r = torch.empty_like(s)
        self.dist.all_to_all_single(r, s)
        return [int(v) for v in r.tolist()]

    def all_gather_var(self, x) -> list:
        """Every rank's tensor (different first-dimension sizes)."""
        import torch
        sizes = self.all_gather_int(x.shape[0])
        m = max(sizes) if sizes else 0
        pad = torch.zeros((m,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
        pad[: x.shape[0]] = x
        out = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(out, pad)
        return [o[:s] for o, s in zip(out, sizes)]


class LocalGroup:
    """G shards as threads of one process, exchanging tensors in memory
    (several shards on one GPU, or tests).  comm(r) is rank r's
    communicator; every rank must make the same sequence of calls."""

    def __init__(self, world: int):
        self.world = world
        self._barrier = threading.Barrier(world)
        self._slots = [None] * world

    def _exchange(self, rank: int, value):
        self._slots[rank] = value
        self._barrier.wait()
        got = list(self._slots)
        self._barrier.wait()
        return got

    def comm(self, rank: int) -> "LocalComm":
        return LocalComm(self, rank)


class LocalComm:
    def __init__(self, group: LocalGroup, rank: int):
        self.g = group
        self.rank = rank
        self.world = group.world

    def all_gather_int(self, v: int) -> list:
        return [int(x) for x in self.g._exchange(self.rank, int(v))]

    def all_reduce_max(self, t):
        import torch
        got = self.g._exchange(self.rank, t.clone())
        res = got[0].to(t.device)
        for x in got[1:]:
            res = torch.maximum(res, x.to(t.device))
        t.copy_(res)
        return t

    def all_to_all(self, x, send_counts: list):
        import torch
        starts = np.concatenate([[0], np.cumsum(send_counts)]).tolist()
        parts = [x[starts[d]:starts[d + 1]].clone() for d in range(self.world)]
        got = self.g._exchange(self.rank, parts)
        mine = [got[src][self.rank].to(x.device) for src in range(self.world)]
        return torch.cat(mine) if mine else x[:0]

    def all_gather_var(self, x) -> list:
        got = self.g._exchange(self.rank, x.clone())
        return [t.to(x.device) for t in got]


# ------------------------------------------------------------ backend

class GpuBackend:
    """The library's calls on this process's context (tensors on its GPU)."""

    def __init__(self, ctx, stream=None):
        self.ctx = ctx
        self.stream = stream

    def local_alphabet(self, shard: Shard, p):
        d = self.ctx.derive(shard.bytes, shard.offsets, p, stream=self.stream)
        return np.asarray(d["present"], dtype=bool), int(d["input_max_len"])

    def set_alphabet(self, present, N: int):
        self.ctx.set_alphabet(present, N)

    def partition(self, shard: Shard, p):
        """(sid local, pos, len, key, slen) int32/int64 tensors on the GPU."""
        import torch
        sid, pos, ln, key = self.ctx.partition(shard.bytes, shard.offsets, p, stream=self.stream)
        lens = (shard.offsets[1:] - shard.offsets[:-1]).to(torch.int32)
        return sid, pos, ln, key, lens[sid.long()].contiguous() if sid.numel() else sid.clone()

    def candidates(self, sid, pos, ln, key, slen, n_total: int, p):
        return self.ctx.candidates_records(sid, pos, ln, key, slen, n_total, p, stream=self.stream)

    def unique(self, i, j, n_total: int):
        return self.ctx.pairs_unique(i, j, n_total, stream=self.stream)

    def verify(self, data, offsets, i, j, K: int):
        return self.ctx.verify(data, offsets, i, j, K, stream=self.stream)


# ------------------------------------------------------------ the join

def _by_owner(owner, world: int, *cols):
    """Columns reordered by owner rank, and the count per rank."""
    import torch
    order = torch.argsort(owner, stable=True)
    counts = torch.bincount(owner, minlength=world).tolist()
    return [c[order] for c in cols], counts


def sharded_join(comm, backend, shard: Shard, params):
    """Steps 1-7 above on this rank.  Returns (i, j, ed) of this rank's
    output pairs (global ids, i < j, sorted), as tensors on the shard's
    device, and a dict of counts."""
    import torch
    world = comm.world
    dev = shard.offsets.device
    counts = comm.all_gather_int(shard.n)
    n_total = sum(counts)
    first = sum(counts[: comm.rank])
    assert first == shard.first, "shards must hold consecutive id ranges in rank order"

    # 1. global alphabet and longest length
    present, max_len = backend.local_alphabet(shard, params)
    g = torch.tensor(np.concatenate([present.astype(np.int64), [max_len]]), dtype=torch.int64,
                     device=dev if dev.type == "cuda" else "cpu")
    comm.all_reduce_max(g)
    g = g.cpu().numpy()
    backend.set_alphabet(g[:256] > 0, int(g[256]))
    try:
        return _join_steps(comm, backend, shard, params, n_total, first)
    finally:
        backend.set_alphabet(None, 0)


def _join_steps(comm, backend, shard: Shard, params, n_total: int, first: int):
    import torch
    world = comm.world
    dev = shard.offsets.device

    # 2. local partitions, global string ids
    sid, pos, ln, key, slen = backend.partition(shard, params)
    sid = sid + int(first)

    # 3. records to the owners of their (length, key) classes
    owner = _mix_owner(key ^ (ln.to(torch.int64) * 0x632BE59BD9B4E019), world)
    (sid, pos, ln, key, slen), send = _by_owner(owner, world, sid, pos, ln, key, slen)
    sid, pos, ln, key, slen = (comm.all_to_all(c, send).contiguous() for c in (sid, pos, ln, key, slen))

    # 4. candidates of the owned classes
    ci, cj = backend.candidates(sid, pos, ln, key, slen, n_total, params)

    # 5. pairs to their owners; dedup of C there
    powner = _mix_owner(ci.to(torch.int64) * n_total + cj.to(torch.int64), world)
    (ci, cj), send = _by_owner(powner, world, ci, cj)
    ci, cj = (comm.all_to_all(c, send).contiguous() for c in (ci, cj))
    ci, cj = backend.unique(ci, cj, n_total)

    # 6. all strings on every rank; verify the owned pairs
    parts = comm.all_gather_var(shard.bytes)
    lens = comm.all_gather_var(shard.offsets[1:] - shard.offsets[:-1])
    data = torch.cat(parts).contiguous()
    all_len = torch.cat(lens)
    offsets = torch.zeros(n_total + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(all_len, 0)
    ed = backend.verify(data, offsets, ci, cj, params.K)

    # 7. this rank's output
    keep = ed <= params.K
    info = {"records_in": int(sid.shape[0]), "candidates": int(ci.shape[0]), "n_total": n_total}
    return ci[keep], cj[keep], ed[keep], info
