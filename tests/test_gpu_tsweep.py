"""The T sweep (the paper's study of T between K/5 and K) on the tiny DNA
workload: every output pair is a true pair, and recall does not fall as T
grows (more, shorter partitions give more chances to share one)."""
import pytest

pytestmark = pytest.mark.gpu


def test_t_sweep_tiny_dna():
    from paper_1810_08833_gb300 import t_sweep
    rows = t_sweep.main(["--config", "1", "--steps", "1"])
    assert [r["T"] for r in rows] == [2, 4, 6, 8, 10]
    assert all(r["precision"] == 1.0 for r in rows)
    assert all(0.0 < r["recall"] <= 1.0 for r in rows)
    assert rows[-1]["recall"] >= rows[0]["recall"]
    assert rows[-1]["candidates"] >= rows[0]["candidates"]
