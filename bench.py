#!/usr/bin/env python
"""Benchmark of the GB300 MinJoin edit-similarity join.

One step = one whole join (Alg. 3 of the MinJoin paper: parameters, partition,
hash join with both filters, dedup, banded verification, output compaction)
over a synthetic string set resident in HBM.  The metric is the join's
throughput in K-band DP cells per second of join wall time:
    value = sum over candidate pairs (a, b) of #{(i, j): 1 <= i <= |a|,
            1 <= j <= |b|, |i - j| <= K}, divided by the join time,
with the join time itself reported as ms_per_step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config C] [--impl native|reference]

Multi-GPU: N independent replicas (one process per GPU under torchrun), each
joining its own instance of the workload (different seed): weak scaling, no
collective on the data path; the barrier and the max over ranks of the step
time are the only communication.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "join wall time & verified DP cells/s; learned-band vs plain K-band, identical output"
UNIT = "cells/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# 32-bit integer ALU lanes per SM and clock by compute capability major
# (Blackwell SMs: 4 partitions x 16 lanes); the SM count and clock are read
# from the device and from the sampled clocks
INT_LANES_PER_SM = {10: 64, 12: 64, 9: 64}
ALU_OPS_PER_WORD_COLUMN = 16 # ops of one band word in one column of the bit-vector recurrence
RECORD_BYTES = 24            # one partition record written: sid, pos, len, string length (u32), key (u64)
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, a one-pass capture
# of the full-size launch) of the current kernel, keyed by (section, workload
# number); absent (reported as null) where no capture of the current kernel
# exists.  Text-like workload: verify_diag_kernel<3, 7> with three digit
# tables, code bytes and the per-chunk count of the top row's rises,
# 49.80 GB read + 3.82 GB written in one launch over 645 M candidates.
TRAFFIC_BYTES = {("verify_kernel", 5): 49.80e9 + 3.82e9}
# integer issue ceiling per SM and clock: the ALU pipe's 64 lanes plus the
# FMA pipe's 64 (integer multiply-adds run there)
ISSUE_LANES_PER_SM = 128


def replica_seed(cfg: int, rank: int) -> int:
    """Seed of the workload instance rank `rank` joins: the workload's own on
    rank 0, a distinct one on every other rank (weak scaling)."""
    return cfg if rank == 0 else cfg + 7919 * rank


def reduce_over_ranks(times_ms: list, cells: int, device) -> tuple:
    """The job's step times (max over ranks, element-wise) and its work (sum
    of the ranks' cells); the identity with one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in times_ms], float(cells)
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], float(c[0])


def band_cells(m: np.ndarray, n: np.ndarray, K: int) -> int:
    """K-band cells of pairs with lengths m >= n: sum over j = 1..n of
    min(m, j+K) - max(1, j-K) + 1, in closed form."""
    m = m.astype(np.int64)
    n = n.astype(np.int64)
    a = np.clip(m - K, 0, n)
    smin = a * (a + 1) // 2 + a * K + (n - a) * m
    b = np.minimum(K, n)
    smax = b + np.where(n > K, (n - K) * (n - K + 1) // 2, 0)
    return int(np.where(n > 0, smin - smax + n, 0).sum())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


def workload_name(cfg: int, s) -> str:
    import synth
    return f"config {cfg}: {synth.CONFIGS[cfg][0]}; K={s.K}, T={s.T}"


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(cfg: int, roots: int, threads: int | None = None) -> dict:
    """The oracle (as it stands) on a bounded sample of the workload: the
    same generator with fewer root families."""
    import oracle
    import synth
    s = synth.make_config(cfg, n_roots=roots)
    t0 = time.perf_counter()
    res = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T, threads=threads)
    dt = time.perf_counter() - t0
    L = s.lengths()
    a, b = res.candidates[:, 0], res.candidates[:, 1]
    cells = band_cells(np.maximum(L[a], L[b]), np.minimum(L[a], L[b]), s.K)
    return {"seconds": dt, "cells": cells, "value": cells / dt if dt > 0 else 0.0, "n_strings": s.n,
            "bytes": int(s.bytes.shape[0]), "candidates": int(res.candidates.shape[0]),
            "output": int(res.pairs.shape[0])}


def run_reference(args):
    """The CPU oracle timed as the reference arm (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    threads = os.cpu_count() or 1
    roots = args.ref_roots
    for _ in range(args.warmup):
        oracle_sample(args.config, roots, threads)
    runs = [oracle_sample(args.config, roots, threads) for _ in range(args.steps)]
    secs = sum(r["seconds"] for r in runs)
    cells = sum(r["cells"] for r in runs)
    value = cells / secs
    s_full = synth.CONFIGS[args.config]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": f"config {args.config}: {s_full[0]}; K={s_full[1]}, T={s_full[2]}",
                   "sample": f"{roots} root families x 10 copies per step ({runs[0]['n_strings']} strings, "
                             f"{runs[0]['bytes']} bytes)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{roots} of {s_full[3]} root families per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU

def run_native(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        from paper_1810_08833_gb300 import build
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1810_08833_gb300 as mj
    import synth

    cfg = args.config
    seed = replica_seed(cfg, rank)
    s = synth.make_config(cfg, seed=seed)
    data = torch.from_numpy(s.bytes).to(dev)
    off = torch.from_numpy(s.offsets).to(dev)
    ctx = mj.Context(local)
    plain = mj.params(s.K, T=s.T)
    learned = mj.params(s.K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED)
    stream = torch.cuda.Stream(dev)

    def sync_all():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        # the band network learns from a held-out instance of the workload
        # (different seed, a quarter of the families), outside the timed region
        t0 = time.perf_counter()
        tr = synth.make_config(cfg, seed=100 + seed, n_roots=max(10, synth.CONFIGS[cfg][3] // 4))
        tr_data = torch.from_numpy(tr.bytes).to(dev)
        tr_off = torch.from_numpy(tr.offsets).to(dev)
        ctx.join(tr_data, tr_off, mj.params(tr.K, T=tr.T, flags=mj.MJ_FLAG_FEATURES), stream=stream)
        x, ed, _, _ = ctx.features(stream=stream)
        ctx.band_init(seed=5)
        train_loss = ctx.band_train(x, ed, K=tr.K, steps=args.band_steps, batch=1024, lr=2e-3, tau=0.9, seed=13,
                                    stream=stream)
        train_s = time.perf_counter() - t0
        n_train = int(x.shape[0])
        del x, ed
        # learned mode keeps the network only where it was faster than plain
        # on the held-out instance (timed joins of both modes)
        calibration = ctx.band_calibrate(tr_data, tr_off, learned, stream=stream)
        del tr_data, tr_off

        def timed(p, steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            st = []
            e0.record(stream)
            for _ in range(steps):
                out = ctx.join(data, off, p, stream=stream)
                st.append(ctx.stats())
            e1.record(stream)
            sync_all()
            return e0.elapsed_time(e1) / steps, st, out

        def paired(steps):
            """Learned and plain joins alternating, each timed by its own
            events, so that neither mode gets the other's clock or cache
            state; medians per mode."""
            evs = {m: [] for m in ("learned", "plain")}
            st = {m: [] for m in evs}
            outs = {}
            for _ in range(steps):
                for mode, p in (("learned", learned), ("plain", plain)):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    outs[mode] = ctx.join(data, off, p, stream=stream)
                    e1.record(stream)
                    evs[mode].append((e0, e1))
                    st[mode].append(ctx.stats())
            sync_all()
            med = {m: statistics.median(a.elapsed_time(b) for a, b in evs[m]) for m in evs}
            return med, st, outs

        for _ in range(args.warmup):
            ctx.join(data, off, learned, stream=stream)
            ctx.join(data, off, plain, stream=stream)
        sync_all()
        clocks = Clocks(local)
        clocks.start()
        ms, stats, out_l = timed(learned, args.steps)
        pair_ms, pair_st, pair_out = paired(args.steps)
        clk = clocks.stop()
        ms_plain, stats_plain, out_p = pair_ms["plain"], pair_st["plain"], pair_out["plain"]
        identical = all(bool(torch.equal(a, b)) for a, b in zip(out_l, out_p)) and \
            all(bool(torch.equal(a, b)) for a, b in zip(pair_out["learned"], out_p))

        # end to end through host buffers: H2D of the inputs and D2H of the
        # output pairs inside every timed step
        h_data = torch.from_numpy(s.bytes).pin_memory()
        h_off = torch.from_numpy(s.offsets).pin_memory()
        n_out = stats[-1]["n_output"]
        h_out = [torch.empty(max(1, n_out) + 1024, dtype=torch.int32).pin_memory() for _ in range(3)]
        outs = tuple(o.numpy().view(np.uint32) for o in h_out)
        # (at least two calls: the verification stage's CUDA graph is
        # captured on the second call with new buffers)
        for _ in range(max(2, args.warmup)):
            ctx.join_host(h_data.numpy(), h_off.numpy(), learned, stream=stream, out=outs)
        sync_all()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            ctx.join_host(h_data.numpy(), h_off.numpy(), learned, stream=stream, out=outs)
        f1.record(stream)
        sync_all()
        ms_e2e = f0.elapsed_time(f1) / args.steps
        e2e_stats = ctx.stats()

        # batched verification: one persistent launch (default kernel) vs the
        # autotuned per-length-bucket plan, as one persistent launch per run
        # of buckets sharing a kernel (captured in a CUDA graph) or as one
        # launch per bucket
        batching = None
        if args.batching:
            ci, cj = ctx.candidates(data, off, plain, stream=stream)
            tune = ctx.autotune_verify(data, off, ci, cj, s.K, sample=args.tune_sample, stream=stream)
            batching = {"tuned": {str(b): {"pairs": v["pairs"], "kernel": v["kernel"], "lanes": v["lanes"],
                                           "ms": v["ms"]} for b, v in tune["buckets"].items()}}
            for name, cfgv in (("single_persistent", (mj.MJ_VERIFY_KERNEL_AUTO, 0, 0, 0)),
                               ("tuned_persistent_graph", (mj.MJ_VERIFY_KERNEL_TUNED, 0, 0, 1)),
                               ("tuned_per_bucket", (mj.MJ_VERIFY_KERNEL_TUNED, 0, 1, 0))):
                ctx.set_verify_config(*cfgv)
                for _ in range(2):
                    ctx.join(data, off, plain, stream=stream)
                sync_all()
                tms, tst, tout = timed(plain, args.steps)
                batching[name] = {"join_ms": tms,
                                  "verify_ms": statistics.median([x["ms_section"]["verify_kernel"] for x in tst]),
                                  "identical_output": all(bool(torch.equal(a, b)) for a, b in zip(tout, out_p))}
            ctx.set_verify_config(0, 0, 0, 0)

    last = stats[-1]
    cells = int(last["band_cells"])
    # ceiling of any first-pass gain: the band words x columns that pairs with
    # ED <= K take at band K (they run every column of the shorter string),
    # as a share of all the plain join's word-columns
    L = s.lengths().astype(np.int64)
    oi_h, oj_h = out_p[0].cpu().numpy().astype(np.int64), out_p[1].cpu().numpy().astype(np.int64)
    words_k = (s.K + 1 + 31) // 32
    true_wc = int((np.minimum(L[oi_h], L[oj_h]) * words_k).sum())
    true_share = true_wc / max(1, int(stats_plain[-1]["verify_word_columns"]))
    sec_ms = {k: statistics.median([st["ms_section"][k] for st in stats]) for k in mj.SECTIONS}
    launches = int(sum(st["n_launches"] for st in stats))

    (ms, ms_e2e, ms_plain), cells_all = reduce_over_ranks([ms, ms_e2e, ms_plain], cells, dev)

    if rank == 0:
        peaks = measured_peaks()
        hbm = peaks.get("hbm_gbs")
        hbm_src = "measured" if hbm else "fallback"
        hbm = hbm or FALLBACK_HBM_GBS
        sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
        props = torch.cuda.get_device_properties(dev)
        alu = {"sms": props.multi_processor_count, "lanes": INT_LANES_PER_SM.get(props.major, 64), "mhz": sm_mhz}
        nbytes = int(s.bytes.shape[0])
        # dominant kernel: the section with the largest share of the step
        dom = max(sec_ms, key=lambda k: sec_ms[k])
        roof = roofline(dom, sec_ms[dom], last, nbytes, hbm, hbm_src, alu, cfg)
        part_roof = partition_roofline(sec_ms, last, nbytes, hbm, hbm_src)
        line = {
            "metric": METRIC, "value": cells_all / (ms / 1000.0), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_name(cfg, s), "n_strings": s.n, "bytes": nbytes, "K": s.K, "T": s.T,
                       "verify_mode": "learned first-pass band, fallback to K", "parallelism": f"replicas x{world}",
                       "l2": f"inputs ({nbytes / 1e6:.0f} MB) larger than L2 (129 MB); no flush"},
            "join_ms": ms,
            "learned_vs_plain": {
                "learned_ms": pair_ms["learned"], "plain_ms": ms_plain, "speedup": ms_plain / pair_ms["learned"],
                "timing": "alternating learned and plain joins, median of each", "identical_output": identical,
                "learned_verify_word_columns": int(stats[-1]["verify_word_columns"]),
                "plain_verify_word_columns": int(stats_plain[-1]["verify_word_columns"]),
                "first_pass_settled": int(stats[-1]["first_pass_settled"]),
                "fallback_pairs": int(stats[-1]["fallback_pairs"]),
                "plain_sections_ms": {k: round(statistics.median([st["ms_section"][k] for st in stats_plain]), 4)
                                      for k in mj.SECTIONS},
                "band_training": {"samples": n_train, "steps": args.band_steps, "seconds": round(train_s, 2),
                                  "final_batch_loss": train_loss, "data": "held-out seed, a quarter of the families"},
                "calibration": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in calibration.items()},
                "network_runs": bool(calibration["enabled"]),
                "true_pair_word_column_share": round(true_share, 5),
            },
            "batching": batching,
            "cells_per_step": cells_all,
            "candidates": int(last["n_candidates"]), "raw_pairs": int(last["n_raw_pairs"]),
            "partitions": int(last["n_partitions"]), "output_pairs": int(last["n_output"]),
            "verify_word_columns": int(last["verify_word_columns"]),
            "sections_ms": {k: round(v, 4) for k, v in sec_ms.items()},
            "roofline": roof,
            "partition_roofline": part_roof,
            "e2e": {"value": cells_all / (ms_e2e / 1000.0), "unit": UNIT, "ms_per_step": ms_e2e,
                    "h2d_bytes_per_step": nbytes + 8 * (s.n + 1),
                    "d2h_bytes_per_step": 12 * int(e2e_stats["n_output"])},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            ob = oracle_sample(cfg, args.cpu_roots)
            line["cpu_baseline"] = {"value": ob["value"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"config {cfg} generator with {args.cpu_roots} root families "
                                              f"({ob['n_strings']} strings, {ob['bytes']} bytes, "
                                              f"{ob['candidates']} candidates), {ob['seconds']:.1f} s"}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def roofline(section: str, ms: float, st: dict, nbytes: int, hbm: float, hbm_src: str, alu: dict, cfg: int) -> dict:
    """Roofline entry of the dominant section, from its algorithmic work."""
    sec = ms / 1000.0
    traffic = TRAFFIC_BYTES.get((section, cfg))
    if section == "anchor_test":
        # reads every byte once, writes one anchor bit per byte
        work = nbytes + nbytes / 8
        ach = work / sec / 1e9
        return {"kernel": section, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic, "peak_source": hbm_src}
    if section in ("record_sort", "pair_dedup"):
        n = st["n_partitions"] if section == "record_sort" else st["n_raw_pairs"]
        per = 24 if section == "record_sort" else 16   # one read and one write of key (+ value)
        work = n * per
        ach = work / sec / 1e9
        return {"kernel": section, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic, "peak_source": hbm_src}
    # verification is integer-ALU work: the bit-vector recurrence costs 16
    # 32-bit operations per band word and column (ALU_OPS_PER_WORD_COLUMN),
    # counted over the word-columns the verifier actually advanced
    peak = alu["sms"] * alu["lanes"] * alu["mhz"] * 1e6 / 1e9   # Gop/s
    ops = st["verify_word_columns"] * ALU_OPS_PER_WORD_COLUMN
    ach = ops / sec / 1e9
    issue_peak = alu["sms"] * ISSUE_LANES_PER_SM * alu["mhz"] * 1e6 / 1e9
    return {"kernel": section, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gop/s", "frac": ach / peak,
            "traffic": traffic,
            "peak_source": f"{alu['sms']} SMs x {alu['lanes']} int32 lanes x {alu['mhz']:.0f} MHz (sampled)",
            "frac_of_issue_ceiling": ach / issue_peak}


def partition_roofline(sec_ms: dict, st: dict, nbytes: int, hbm: float, hbm_src: str) -> dict:
    """The partition stage (q-gram values, anchors, partition records) against
    HBM: every input byte read once plus one record written per partition."""
    ms = sec_ms["anchor_test"] + sec_ms["partition_records"]
    work = nbytes + RECORD_BYTES * st["n_partitions"]
    ach = work / (ms / 1000.0) / 1e9
    return {"sections": ["anchor_test", "partition_records"], "bound": "hbm", "achieved": ach, "peak": hbm,
            "unit": "GB/s", "frac": ach / hbm, "algorithmic_bytes": work, "ms": ms, "peak_source": hbm_src}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-roots", type=int, default=400)
    ap.add_argument("--ref-roots", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--band-steps", type=int, default=2000)
    ap.add_argument("--batching", type=int, default=-1, help="compare batched verification plans (default: config 3)")
    ap.add_argument("--tune-sample", type=int, default=2048)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.batching < 0:
        args.batching = 1 if args.config == 3 else 0
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
