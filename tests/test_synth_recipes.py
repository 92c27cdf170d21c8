"""The seeded stand-in workloads follow their stated recipes (CPU, reduced
family counts): determinism, size, alphabet, length bounds, K and T, and
families of ten related copies."""
import numpy as np
import pytest

import synth

ROOTS = {1: 20, 2: 8, 3: 4, 4: 40, 5: 6}


@pytest.mark.parametrize("cfg", sorted(ROOTS))
def test_recipe(cfg):
    r = ROOTS[cfg]
    s = synth.make_config(cfg, n_roots=r)
    again = synth.make_config(cfg, n_roots=r)
    other = synth.make_config(cfg, seed=cfg + 1000, n_roots=r)
    assert np.array_equal(s.bytes, again.bytes) and np.array_equal(s.offsets, again.offsets)
    assert not np.array_equal(s.bytes[: min(s.bytes.size, other.bytes.size)],
                              other.bytes[: min(s.bytes.size, other.bytes.size)])
    assert s.n == 10 * r
    assert np.array_equal(np.sort(np.bincount(s.family)), np.full(r, 10))   # 10 copies per root
    K, T = synth.CONFIGS[cfg][1], synth.CONFIGS[cfg][2]
    assert (s.K, s.T) == (K, T)
    L = s.lengths()
    alphabet = set(np.unique(s.bytes).tolist())
    if cfg == 1:
        assert np.all(L == 500) and alphabet <= set(b"ACGT")
    elif cfg == 2:
        assert alphabet <= set(b"ACGT") and 2800 <= L.min() and L.max() <= 7400
    elif cfg == 3:
        assert alphabet <= set(b"ACGT") and 1700 <= L.min() and L.max() <= 23500
    elif cfg == 4:
        assert alphabet <= set(synth.PROTEIN.tolist()) and 40 <= L.min() and L.max() <= 5600
    else:
        assert alphabet <= set(range(0x20, 0x7F)) and L.min() >= 100
        assert 900 <= np.median(L) <= 2100


def test_copies_are_near_their_root_family():
    """Copies of one root are closer to each other than to other families
    (per-copy rate at most 4% on config 2): share of equal 12-mers."""
    s = synth.make_config(2, n_roots=3)

    def kmers(i, step):
        x = s.string(i)
        return {x[p:p + 12] for p in range(0, len(x) - 11, step)}

    every = [kmers(j, 1) for j in range(s.n)]
    fam = s.family
    same, diff = [], []
    for i in range(s.n):
        a = kmers(i, 7)   # sampled 12-mers of i, looked up among all of j's
        for j in range(i + 1, s.n):
            share = len(a & every[j]) / max(1, len(a))
            (same if fam[i] == fam[j] else diff).append(share)
    assert min(same) > 0.2 and max(diff) < 0.05
