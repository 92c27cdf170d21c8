"""A CPU stand-in for the library's calls in the sharded join, built on the
oracle (test infrastructure): partitions by Alg. 1-2 under the global
alphabet, candidates by their set definition over the records, dedup by
numpy, verification by the oracle's banded DP.  Partition keys are 64-bit
digests of the partition substrings."""
import hashlib

import numpy as np

import oracle


class OracleBackend:
    def __init__(self):
        self.present = None
        self.N = 0

    def local_alphabet(self, shard, p):
        data = shard.bytes.numpy()
        present = np.zeros(256, dtype=bool)
        if data.shape[0]:
            present[np.unique(data)] = True
        lens = np.diff(shard.offsets.numpy())
        return present, int(lens.max()) if lens.shape[0] else 0

    def set_alphabet(self, present, N):
        self.present = None if present is None else np.asarray(present, dtype=bool)
        self.N = N

    def _params(self, p):
        vals = np.nonzero(self.present)[0]
        rank = np.zeros(256, dtype=np.uint8)
        rank[vals] = np.arange(vals.shape[0], dtype=np.uint8)
        sigma = int(vals.shape[0])
        bits = 1
        while (1 << bits) < sigma:
            bits += 1
        T = p.T or p.K
        q = p.q or oracle.q_rule(self.N, T, sigma)
        q = max(1, min(q, 64 // bits))
        return oracle.Params(K=p.K, T=T, q=q, r_min=p.r_min, seed=p.seed, sigma=sigma, bits=bits, rank=rank,
                             N=self.N)

    def partition(self, shard, p):
        import torch
        data, off = shard.bytes.numpy(), shard.offsets.numpy()
        parts = oracle.partition(data, off, self._params(p), threads=2)
        keys = np.array([int.from_bytes(hashlib.blake2b(data[off[s] + a:off[s] + a + b].tobytes(),
                                                        digest_size=8).digest(), "little", signed=True)
                         for s, a, b in zip(parts.sid.tolist(), parts.pos.tolist(), parts.len.tolist())],
                        dtype=np.int64)
        lens = np.diff(off)
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt))
        return (t(parts.sid, np.int32), t(parts.pos, np.int32), t(parts.len, np.int32), t(keys, np.int64),
                t(lens[parts.sid], np.int32))

    def candidates(self, sid, pos, ln, key, slen, n_total, p):
        import torch
        K = p.K
        groups = {}
        for s, a, b, k, L in zip(sid.tolist(), pos.tolist(), ln.tolist(), key.tolist(), slen.tolist()):
            groups.setdefault((b, k), []).append((s, a, L))
        out = set()
        for members in groups.values():
            for x in range(len(members)):
                for y in range(x + 1, len(members)):
                    (i, pi, Li), (j, pj, Lj) = members[x], members[y]
                    if i == j or abs(Li - Lj) > K:
                        continue
                    if abs(pi - pj) + abs((Li - pi) - (Lj - pj)) <= K:
                        out.add((min(i, j), max(i, j)))
        arr = np.array(sorted(out), dtype=np.int32).reshape(-1, 2)
        return torch.from_numpy(arr[:, 0].copy()), torch.from_numpy(arr[:, 1].copy())

    def unique(self, i, j, n_total):
        import torch
        a, b = i.numpy(), j.numpy()
        rows = np.unique(np.stack([np.minimum(a, b), np.maximum(a, b)], 1).reshape(-1, 2), axis=0)
        return torch.from_numpy(rows[:, 0].astype(np.int32).copy()), torch.from_numpy(rows[:, 1].astype(np.int32).copy())

    def verify(self, data, offsets, i, j, K):
        import torch
        pairs = np.stack([i.numpy(), j.numpy()], 1).astype(np.int64)
        ed = oracle.ed_band_pairs(data.numpy(), offsets.numpy(), pairs, K) if pairs.shape[0] else np.zeros(0)
        return torch.from_numpy(ed.astype(np.int32))
