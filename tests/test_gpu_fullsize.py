"""Exact parity at the full workload sizes, in the launch configuration the
benchmark times (plain and learned verification on a side stream; for the
long noisy DNA workload also the autotuned, graph-captured plan).

The CPU oracle's complete results on the five workloads are stored as SHA-256
digests and counts in tests/golden/fullsize_digests.json, written by
tests/golden/make_fullsize_digests.py, which calls only the oracle and the
input generators.  Here the GPU path's results on the same generated inputs
are hashed the same way and must match exactly:
  * the partitions of Alg. 1-2 ((sid, pos, len) in string order);
  * the candidate set C of Alg. 3 ((i, j), sorted);
  * min(ED, K + 1) of every candidate (mj_verify, band K, in the order of C);
  * the output of the join ((i, j, ED), sorted), in plain and learned mode.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "fullsize_digests.json")


def _golden() -> dict:
    with open(GOLDEN) as f:
        return json.load(f)


def digest_rows(*cols, chunk=1 << 24) -> str:
    """SHA-256 of the rows (c0[t], c1[t], ...) as little-endian int64, the
    byte layout of the stored digests; the columns are device or host
    tensors, copied to the host a chunk of rows at a time."""
    import torch
    h = hashlib.sha256()
    m = int(cols[0].shape[0])
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        parts = [c[lo:hi].to("cpu", torch.int64).numpy() if torch.is_tensor(c) else
                 np.asarray(c[lo:hi], dtype=np.int64) for c in cols]
        rows = np.stack(parts, axis=1) if len(parts) > 1 else parts[0]
        h.update(np.ascontiguousarray(rows.astype("<i8", copy=False)).tobytes())
    return h.hexdigest()


def input_digest(s) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s.bytes, dtype=np.uint8).tobytes())
    h.update(np.ascontiguousarray(s.offsets, dtype="<i8").tobytes())
    return h.hexdigest()


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


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
def test_fullsize_exact_parity(ctx, cfg):
    import torch
    import paper_1810_08833_gb300 as mj
    gold = _golden().get(str(cfg))
    assert gold is not None, f"no stored oracle digests for workload {cfg}"
    s = synth.make_config(cfg, n_roots=gold["roots"])
    assert input_digest(s) == gold["input_sha256"], \
        "the input generator made a different string set from the one the digests were made from"
    K = s.K
    stream = torch.cuda.Stream()
    data = torch.from_numpy(s.bytes).cuda()
    off = torch.from_numpy(s.offsets).cuda()
    checked = mj.params(K, T=s.T, flags=mj.MJ_FLAG_KEY_CHECK)
    with torch.cuda.stream(stream):
        d = ctx.derive(data, off, checked, stream=stream)
        assert {k: d[k] for k in ("sigma", "bits", "q", "N")} == gold["derived"]

        sid, pos, ln, _ = ctx.partition(data, off, checked, stream=stream)
        stream.synchronize()
        assert int(sid.shape[0]) == gold["n_partitions"]
        assert digest_rows(sid, pos, ln) == gold["partitions_sha256"]
        del sid, pos, ln

        ci, cj = ctx.candidates(data, off, checked, stream=stream)
        stream.synchronize()
        st = ctx.stats()
        assert st["key_collisions"] == 0 and st["device_flags"] == 0
        assert int(ci.shape[0]) == gold["n_candidates"]
        assert digest_rows(ci, cj) == gold["candidates_sha256"]
        ced = ctx.verify(data, off, ci, cj, K, stream=stream)
        stream.synchronize()
        assert digest_rows(ced) == gold["candidate_ed_sha256"]
        del ci, cj, ced

        oi, oj, oe = ctx.join(data, off, mj.params(K, T=s.T), stream=stream)
        stream.synchronize()
        assert ctx.stats()["device_flags"] == 0
        assert int(oi.shape[0]) == gold["n_output"]
        assert digest_rows(oi, oj, oe) == gold["output_sha256"]

        _train_band(ctx, mj, cfg, stream)
        for flags in (0, mj.MJ_FLAG_FIRST_PASS):
            li, lj, le = ctx.join(data, off, mj.params(K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED, flags=flags),
                                  stream=stream)
            stream.synchronize()
            assert ctx.stats()["device_flags"] == 0
            assert digest_rows(li, lj, le) == gold["output_sha256"], f"learned mode (flags {flags})"
            del li, lj, le

        if cfg == 3:   # the autotuned per-bucket plan, captured in a graph
            ci, cj = ctx.candidates(data, off, checked, stream=stream)
            ctx.autotune_verify(data, off, ci, cj, K, sample=2048, stream=stream)
            del ci, cj
            ctx.set_verify_config(mj.MJ_VERIFY_KERNEL_TUNED, 0, 0, 1)
            try:
                for _ in range(3):   # uncaptured, captured, replayed
                    ti, tj, te = ctx.join(data, off, mj.params(K, T=s.T), stream=stream)
                    stream.synchronize()
                    assert digest_rows(ti, tj, te) == gold["output_sha256"], "tuned graph plan"
            finally:
                ctx.set_verify_config(0, 0, 0, 0)
