#!/usr/bin/env python
"""Writes tests/golden/fullsize_digests.json: the CPU oracle's complete result
on the five synthetic workloads at their full sizes, stored as SHA-256
digests and counts, for the exact full-size parity test
(tests/test_gpu_fullsize_digests.py).

Only `oracle/` (the plain restatement of Alg. 1-3 and Ukkonen's banded DP)
and `synth/` (the seeded input generators) are called; nothing here comes
from the CUDA path.  Per workload it records:
  * the SHA-256 of the generated input (bytes, and offsets as little-endian
    int64), so that a different generator build is reported as such;
  * the derived parameters (Sigma, bits per code, q, N);
  * the partitions of Alg. 1-2: (sid, pos, len) rows in string order;
  * the candidate set C of Alg. 3 (after dedup): (i, j) rows, sorted;
  * min(ED, K + 1) of every candidate, in the order of C (banded DP with
    Ukkonen's cut-off, which returns the same values as the plain band);
  * the output: (i, j, ED) rows with ED <= K, sorted.
Rows are little-endian int64, row-major, hashed as one byte string.

    python tests/golden/make_fullsize_digests.py --config 2 [--roots N] [--threads T]

Each call adds or replaces one workload's entry.  Full-size runs take from a
minute (workload 2) to hours (workload 5) on a few cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "fullsize_digests.json")


def digest_rows(*cols) -> str:
    """SHA-256 of the rows (c0[t], c1[t], ...) as little-endian int64."""
    if not cols:
        return hashlib.sha256(b"").hexdigest()
    a = np.stack([np.asarray(c, dtype="<i8") for c in cols], axis=1) if len(cols) > 1 else \
        np.asarray(cols[0], dtype="<i8")
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def input_digest(s) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s.bytes, dtype=np.uint8).tobytes())
    h.update(np.ascontiguousarray(s.offsets, dtype="<i8").tobytes())
    return h.hexdigest()


def run(cfg: int, roots: int | None, threads: int | None) -> dict:
    t0 = time.time()
    s = synth.make_config(cfg, n_roots=roots)
    p = oracle.derive_params(s.bytes, s.offsets, K=s.K, T=s.T)
    t1 = time.time()
    parts = oracle.partition(s.bytes, s.offsets, p, threads=threads)
    t2 = time.time()
    C = oracle.candidates(s.bytes, s.offsets, s.K, parts)
    t3 = time.time()
    ed = oracle.ed_band_pairs(s.bytes, s.offsets, C, s.K, threads=threads, cutoff=True)
    t4 = time.time()
    keep = ed <= s.K
    return {
        "config": cfg,
        "roots": roots if roots is not None else synth.CONFIGS[cfg][3],
        "n_strings": s.n, "n_bytes": int(s.bytes.shape[0]), "K": s.K, "T": s.T,
        "input_sha256": input_digest(s),
        "derived": {"sigma": p.sigma, "bits": p.bits, "q": p.q, "N": p.N},
        "n_partitions": int(parts.sid.shape[0]),
        "partitions_sha256": digest_rows(parts.sid, parts.pos, parts.len),
        "n_candidates": int(C.shape[0]),
        "candidates_sha256": digest_rows(C[:, 0], C[:, 1]),
        "candidate_ed_sha256": digest_rows(ed),
        "n_output": int(keep.sum()),
        "output_sha256": digest_rows(C[keep, 0], C[keep, 1], ed[keep]),
        "oracle_seconds": {"generate": round(t1 - t0, 1), "partition": round(t2 - t1, 1),
                           "candidates": round(t3 - t2, 1), "verify": round(t4 - t3, 1)},
        "threads": threads or oracle.default_threads(),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, required=True)
    ap.add_argument("--roots", type=int, default=None, help="root families (default: the full workload)")
    ap.add_argument("--threads", type=int, default=None)
    args = ap.parse_args()
    oracle.build()
    entry = run(args.config, args.roots, args.threads)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data[str(args.config)] = entry
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        json.dump(dict(sorted(data.items())), f, indent=1)
        f.write("\n")
    os.replace(tmp, OUT)
    print(json.dumps(entry))


if __name__ == "__main__":
    main()
