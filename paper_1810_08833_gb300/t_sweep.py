"""Join time and recall for partition parameters T between K/5 and K, and
for parallel repetition.

    python -m paper_1810_08833_gb300.t_sweep --config 1 [--roots N] [--steps 3]
        [--T 2,10] [--repeats 1,2,3]

The paper studies how T trades accuracy for time (Sec. 4.2, Fig. 3 and 4,
with T between K/5 and K).  This runs that study on the synthetic workloads.
For each T it times the join on cuda:0 (warm, CUDA events on the join's
stream) and compares its output with the true pair set.  The true pairs are
every pair i < j whose banded distance is at most K, found by verifying all
n(n-1)/2 pairs with the library's verifier; the GPU tests check that
verifier against the CPU oracle.

Every output pair is verified, so precision is 1.  Recall is |output| /
|true pairs|.  The candidate and partition counts show what a larger T
costs.  --repeats adds the union of the partitions under R independent Pi
functions (Sec. 2.2's parallel repetition).  Prints one JSON line per (T, R),
then a markdown table.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def true_pairs(ctx, data, off, n: int, K: int, stream, chunk: int = 1 << 22):
    """(i, j) of every pair i < j with banded distance <= K, as an int64 key
    set i * n + j (all pairs verified in chunks)."""
    import torch
    keys = []
    iu = torch.triu_indices(n, n, offset=1, device="cuda")
    for s in range(0, iu.shape[1], chunk):
        i = iu[0, s:s + chunk].to(torch.int32).contiguous()
        j = iu[1, s:s + chunk].to(torch.int32).contiguous()
        ed = ctx.verify(data, off, i, j, K, stream=stream)
        ok = ed <= K
        keys.append(i[ok].long() * n + j[ok].long())
    return torch.cat(keys) if keys else torch.empty(0, dtype=torch.long, device="cuda")


def main(argv=None) -> list:
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--roots", type=int, default=None, help="root families (default: the workload's own)")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--T", default="", help="comma-separated T values (default K/5, 2K/5, ..., K)")
    ap.add_argument("--repeats", default="1", help="comma-separated repetition counts")
    args = ap.parse_args(argv)

    import torch
    import synth
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build

    build.build()
    s = synth.make_config(args.config, n_roots=args.roots)
    K = s.K
    stream = torch.cuda.Stream()
    rows = []
    with torch.cuda.stream(stream), mj.Context(0) as ctx:
        data = torch.from_numpy(s.bytes).cuda()
        off = torch.from_numpy(s.offsets).cuda()
        truth = true_pairs(ctx, data, off, s.n, K, stream)
        stream.synchronize()
        n_true = int(truth.numel())
        Ts = [int(x) for x in args.T.split(",") if x] or sorted({max(1, round(K * f / 5)) for f in (1, 2, 3, 4, 5)})
        grid = [(T, R) for T in Ts for R in (int(x) for x in args.repeats.split(","))]
        for T, R in grid:
            p = mj.params(K, T=T, repeats=R)
            ctx.join(data, off, p, stream=stream)   # warm-up (sizes the buffers)
            times = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                oi, oj, _ = ctx.join(data, off, p, stream=stream)
                e1.record(stream)
                stream.synchronize()
                times.append(e0.elapsed_time(e1))
            st = ctx.stats()
            got = oi.long() * s.n + oj.long()
            hit = int(torch.isin(got, truth).sum()) if got.numel() else 0
            row = {"workload": f"config {args.config}", "roots": args.roots, "n_strings": s.n, "K": K, "T": T,
                   "repeats": R,
                   "join_ms": round(sorted(times)[len(times) // 2], 3), "partitions": st["n_partitions"],
                   "candidates": st["n_candidates"], "output": int(got.numel()), "true_pairs": n_true,
                   "recall": round(hit / n_true, 5) if n_true else 1.0,
                   "precision": round(hit / got.numel(), 5) if got.numel() else 1.0}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print("\n| T | R | join (ms) | partitions | candidates | output | true pairs | recall |")
    print("|---|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['T']} | {r['repeats']} | {r['join_ms']} | {r['partitions']:,} | {r['candidates']:,} | "
              f"{r['output']:,} | {r['true_pairs']:,} | {r['recall']:.4f} |")
    return rows


if __name__ == "__main__":
    main()
