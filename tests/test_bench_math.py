"""The benchmark's arithmetic on the CPU: the K-band cell count (the metric's
numerator) in closed form against brute force, and the roofline entries from
their definitions."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _cells_brute(m: int, n: int, K: int) -> int:
    # cells (i, j), 1 <= i <= m, 1 <= j <= n, |i - j| <= K
    return sum(max(0, min(m, j + K) - max(1, j - K) + 1) for j in range(1, n + 1))


def test_band_cells_closed_form():
    rng = np.random.default_rng(7)
    m = rng.integers(0, 300, size=400)
    n = rng.integers(0, 300, size=400)
    m, n = np.maximum(m, n), np.minimum(m, n)
    for K in (0, 1, 5, 40, 299, 1000):
        want = sum(_cells_brute(int(a), int(b), K) for a, b in zip(m, n))
        assert bench.band_cells(m, n, K) == want, K
    # edge cases: empty, equal lengths, a length difference beyond K
    for a, b, K in ((0, 0, 3), (5, 0, 3), (7, 7, 0), (7, 7, 10), (20, 3, 2), (1, 1, 0)):
        assert bench.band_cells(np.array([a]), np.array([b]), K) == _cells_brute(a, b, K)


def test_verify_roofline_from_definition():
    st = {"verify_word_columns": 2_000_000_000}
    alu = {"sms": 152, "lanes": 64, "mhz": 2070.0}
    r = bench.roofline("verify_kernel", 2.5, st, 250_000_000, 6669.2, "measured", alu, 2)
    ops = 2_000_000_000 * bench.ALU_OPS_PER_WORD_COLUMN
    assert r["bound"] == "alu" and r["unit"] == "Gop/s"
    assert abs(r["achieved"] - ops / 2.5e-3 / 1e9) < 1e-6
    assert abs(r["peak"] - 152 * 64 * 2070e6 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["traffic"] == bench.TRAFFIC_BYTES.get(("verify_kernel", 2))


def test_partition_roofline_from_definition():
    sec = {"anchor_test": 0.75, "partition_records": 0.25}
    st = {"n_partitions": 1_000_000}
    r = bench.partition_roofline(sec, st, 100_000_000, 6669.2, "measured")
    work = 100_000_000 + bench.RECORD_BYTES * 1_000_000
    assert r["algorithmic_bytes"] == work and r["ms"] == 1.0
    assert abs(r["achieved"] - work / 1e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6669.2) < 1e-12


def test_replica_seeds_are_distinct():
    seeds = [bench.replica_seed(4, r) for r in range(8)]
    assert seeds[0] == 4 and len(set(seeds)) == 8
