"""One join of a synthetic workload on cuda:0, with its statistics.

    python -m paper_1810_08833_gb300.join_once --config 2 [--roots 3000] [--learned] [--K K --T T]

A small, self-contained invocation of the whole hot path (parameters,
partition, candidates, verification, output), meant for profilers: it builds
the library if needed, generates the workload with the seeded generators,
runs one join (after one warm-up join unless --no-warmup) and prints the
library's statistics as one JSON line.  With --learned a band network is
first trained on a held-out instance of the workload (as the benchmark does,
with fewer steps) and the join runs in learned mode.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--roots", type=int, default=None, help="root families (default: the workload's own)")
    ap.add_argument("--learned", action="store_true")
    ap.add_argument("--no-warmup", action="store_true")
    ap.add_argument("--band-steps", type=int, default=300)
    ap.add_argument("--K", type=int, default=None, help="threshold instead of the workload's own")
    ap.add_argument("--T", type=int, default=None, help="partitions per string instead of the workload's own")
    args = ap.parse_args(argv)

    import torch
    import synth
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build

    build.build()
    s = synth.make_config(args.config, n_roots=args.roots)
    if args.K is not None:
        s.K = args.K
        s.T = args.T if args.T is not None else max(1, args.K // 5)
    elif args.T is not None:
        s.T = args.T
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), mj.Context(0) as ctx:
        if args.learned:
            tr = synth.make_config(args.config, seed=100 + args.config,
                                   n_roots=max(10, (args.roots or synth.CONFIGS[args.config][3]) // 4))
            d = torch.from_numpy(tr.bytes).cuda()
            o = torch.from_numpy(tr.offsets).cuda()
            ctx.join(d, o, mj.params(tr.K, T=tr.T, flags=mj.MJ_FLAG_FEATURES), stream=stream)
            x, ed, _, _ = ctx.features(stream=stream)
            ctx.band_init(seed=5)
            ctx.band_train(x, ed, K=tr.K, steps=args.band_steps, batch=1024, lr=2e-3, tau=0.9, seed=13,
                           stream=stream)
            del x, ed, d, o
        data = torch.from_numpy(s.bytes).cuda()
        off = torch.from_numpy(s.offsets).cuda()
        p = mj.params(s.K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED if args.learned else mj.MJ_VERIFY_PLAIN)
        if not args.no_warmup:
            ctx.join(data, off, p, stream=stream)
        ctx.join(data, off, p, stream=stream)
        stream.synchronize()
        st = ctx.stats()
    out = {"workload": f"config {args.config}", "roots": args.roots, "n_strings": s.n, "bytes": int(s.bytes.shape[0]),
           "K": s.K, "T": s.T, "learned": args.learned,
           **{k: v for k, v in st.items() if not isinstance(v, (list, tuple))}}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
