"""Parity at the full workload sizes, in the launch configuration the benchmark
times (plain and learned verification on a side stream; for the long noisy
DNA workload also the autotuned, graph-captured plan).

The oracle cannot run these joins end to end in seconds, so the checks are
per sample, or properties that hold at any size:
  * the partitions of sampled strings equal the oracle's (Alg. 1-2);
  * every sampled candidate shares an identical partition substring with its
    partner that passes the length and position filters (Alg. 3);
  * the candidate partners of sampled strings are exactly the strings that
    share such a partition with them;
  * sampled candidates get the oracle's banded distance, and a candidate is
    in the output iff that distance is <= K, with that distance;
  * the learned first-pass band returns exactly the plain output.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# workload -> (sampled strings for partitions and partners, sampled candidates for distances)
CASES = {2: (200, 3000), 3: (60, 300), 4: (300, 3000), 5: (200, 2000)}


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


def _train_band(ctx, mj, cfg, stream):
    """A band network trained on a held-out instance (as the benchmark does,
    with fewer steps: any network must give the plain output)."""
    import torch
    tr = synth.make_config(cfg, seed=100 + cfg, n_roots=max(10, synth.CONFIGS[cfg][3] // 8))
    d = torch.from_numpy(tr.bytes).cuda()
    o = torch.from_numpy(tr.offsets).cuda()
    ctx.join(d, o, mj.params(tr.K, T=tr.T, flags=mj.MJ_FLAG_FEATURES), stream=stream)
    x, ed, _, _ = ctx.features(stream=stream)
    ctx.band_init(seed=5)
    ctx.band_train(x, ed, K=tr.K, steps=300, batch=1024, lr=2e-3, tau=0.9, seed=13, stream=stream)


class PartitionIndex:
    """Partition records grouped by (length, key) for lookups by value."""

    def __init__(self, sid, pos, ln, key):
        self.sid, self.pos, self.ln, self.key = sid, pos, ln, key
        self.order = np.lexsort((key, ln))
        self.ln_s = ln[self.order]
        self.key_s = key[self.order]

    def same(self, r):
        """Records with the length and key of record r."""
        lo = np.searchsorted(self.ln_s, self.ln[r], "left")
        hi = np.searchsorted(self.ln_s, self.ln[r], "right")
        ks = self.key_s[lo:hi]
        a = lo + np.searchsorted(ks, self.key[r], "left")
        b = lo + np.searchsorted(ks, self.key[r], "right")
        return self.order[a:b]

    def partners(self, L, K, i):
        """Strings sharing a partition (same length and key; key collisions
        are excluded by the device key check) with string i, where |L_i - L_j|
        <= K and the position filter holds for that partition pair."""
        out = set()
        lo, hi = np.searchsorted(self.sid, i, "left"), np.searchsorted(self.sid, i, "right")
        for r in range(lo, hi):
            t = self.same(r)
            j = self.sid[t]
            pi, pj = self.pos[r], self.pos[t]
            ok = (j != i) & (np.abs(L[i] - L[j]) <= K)
            ok &= np.abs(pi - pj) + np.abs((L[i] - pi) - (L[j] - pj)) <= K
            out.update(j[ok].tolist())
        return out


@pytest.mark.parametrize("cfg", sorted(CASES))
def test_fullsize_sampled_parity(ctx, cfg):
    import torch
    import paper_1810_08833_gb300 as mj
    n_str, n_pairs = CASES[cfg]
    s = synth.make_config(cfg)
    K = s.K
    L = s.lengths().astype(np.int64)
    rng = np.random.Generator(np.random.PCG64(1000 + cfg))
    p = oracle.derive_params(s.bytes, s.offsets, K=K, T=s.T)
    stream = torch.cuda.Stream()
    data = torch.from_numpy(s.bytes).cuda()
    off = torch.from_numpy(s.offsets).cuda()
    plain = mj.params(K, T=s.T, flags=mj.MJ_FLAG_KEY_CHECK)
    with torch.cuda.stream(stream):
        _train_band(ctx, mj, cfg, stream)
        pi_, pj_, pe_ = ctx.join(data, off, mj.params(K, T=s.T), stream=stream)
        li_, lj_, le_ = ctx.join(data, off, mj.params(K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED), stream=stream)
        stream.synchronize()
        assert ctx.stats()["device_flags"] == 0
        for a, b in ((pi_, li_), (pj_, lj_), (pe_, le_)):
            assert torch.equal(a, b), "learned band changed the output"
        if cfg == 3:   # the autotuned per-bucket plan, captured in a graph
            ci, cj = ctx.candidates(data, off, plain, stream=stream)
            ctx.autotune_verify(data, off, ci, cj, K, sample=2048, stream=stream)
            ctx.set_verify_config(mj.MJ_VERIFY_KERNEL_TUNED, 0, 0, 1)
            for _ in range(3):   # uncaptured, captured, replayed
                ti, tj, te = ctx.join(data, off, mj.params(K, T=s.T), stream=stream)
                stream.synchronize()
                for a, b in ((pi_, ti), (pj_, tj), (pe_, te)):
                    assert torch.equal(a, b), "tuned graph plan changed the output"
            ctx.set_verify_config(0, 0, 0, 0)
        sid, pos, ln, key = ctx.partition(data, off, plain, stream=stream)
        ci, cj = ctx.candidates(data, off, plain, stream=stream)
        stream.synchronize()
    st = ctx.stats()
    assert st["key_collisions"] == 0 and st["device_flags"] == 0
    sid, pos, ln, key = (t.cpu().numpy().astype(np.int64) for t in (sid, pos, ln, key))
    assert np.all(np.diff(sid) >= 0)   # records come in string order
    index = PartitionIndex(sid, pos, ln, key)

    # partitions of sampled strings
    sample = np.sort(rng.choice(s.n, size=min(n_str, s.n), replace=False))
    for i in sample.tolist():
        want = oracle.partition(s.bytes, s.offsets, p, lo=i, hi=i + 1)
        sel = slice(np.searchsorted(sid, i, "left"), np.searchsorted(sid, i, "right"))
        assert np.array_equal(pos[sel], want.pos) and np.array_equal(ln[sel], want.len), i

    # candidate partners of sampled strings, by the definition
    for i in sample[: max(1, len(sample) // 4)].tolist():
        got = set(cj[ci == i].cpu().tolist()) | set(ci[cj == i].cpu().tolist())
        assert got == index.partners(L, K, i), i

    # sampled candidates: definition, oracle distance, output membership
    m = ci.shape[0]
    assert m > 0
    idx = torch.from_numpy(rng.choice(m, size=min(n_pairs, m), replace=False)).cuda()
    pairs = torch.stack([ci[idx], cj[idx]], 1).cpu().numpy().astype(np.int64)
    assert np.all(pairs[:, 0] < pairs[:, 1])
    for a, b in pairs[: min(200, len(pairs))].tolist():
        assert b in index.partners(L, K, a), (a, b)
    ed = oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)
    out = {(a, b): e for a, b, e in zip(pi_.cpu().tolist(), pj_.cpu().tolist(), pe_.cpu().tolist())}
    for (a, b), e in zip(pairs.tolist(), ed.tolist()):
        if e <= K:
            assert out.get((a, b)) == e, (a, b, e, out.get((a, b)))
        else:
            assert (a, b) not in out, (a, b)

    # sampled outputs: oracle distance within K, pairs unique and ordered
    outp = np.stack([pi_.cpu().numpy(), pj_.cpu().numpy()], 1).astype(np.int64)
    assert np.all(outp[:, 0] < outp[:, 1])
    assert np.unique(outp, axis=0).shape[0] == outp.shape[0]
    if outp.shape[0]:
        k = rng.choice(outp.shape[0], size=min(n_pairs, outp.shape[0]), replace=False)
        want = oracle.ed_band_pairs(s.bytes, s.offsets, outp[k], K)
        assert np.array_equal(want, pe_.cpu().numpy()[k].astype(np.int64))
