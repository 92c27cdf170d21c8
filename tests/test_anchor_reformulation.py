"""The GPU anchor test's reformulation of Alg. 2, checked on the CPU against
the definition (position i is an anchor iff h[i] < h[j] for every other j
within radius r), on random values with many ties and radii 1..90:

* only a minimum of i's aligned block of B = 2^floor(log2(r+1)) <= 16
  positions can be an anchor (the block lies inside i's window);
* for r < 15 a candidate is decided by its 2r neighbours;
* for r >= 15 the block is the whole 16-position run, the candidate must be
  its unique minimum, and the rest of the window is covered by a suffix
  minimum, whole-run minima and a prefix minimum of 16-position runs.

Runs start at multiples of 16 (the kernel's halo is a multiple of 32)."""
import numpy as np


def _anchor_def(h, o, r):
    w = np.concatenate([h[o - r:o], h[o + 1:o + r + 1]])
    return bool(np.all(h[o] < w))


def _anchor_runs(h, P, S, o0, j, r):
    o = o0 + j
    run = h[o0:o0 + 16]
    if r >= 15:
        eq = run == run.min()
        if eq.sum() != 1 or not eq[j]:
            return False
        m = np.iinfo(np.int64).max
        la = o - r
        if la < o0:
            m = S[la]
            for u in range((la >> 4) + 1, o0 >> 4):
                m = min(m, S[16 * u])
        rb = o + r
        for u in range((o0 >> 4) + 1, rb >> 4):
            m = min(m, S[16 * u])
        if rb >= o0 + 16:
            m = min(m, P[rb])
        return bool(P[o0 + 15] < m)
    B = 8 if r >= 7 else (4 if r >= 3 else 2)
    bs = o0 + (j & ~(B - 1))
    if h[o] != h[bs:bs + B].min():
        return False
    return bool(h[o] < min(h[o - r:o].min(), h[o + 1:o + r + 1].min()))


def test_block_candidates_equal_the_definition():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(400):
        r = int(rng.integers(1, 91))
        Hs = ((r + 31) // 32) * 32
        tile = 16 * int(rng.integers(2, 9))
        h = rng.integers(0, int(rng.choice([3, 40, 1 << 30])), size=tile + 2 * Hs).astype(np.int64)
        runs = h.reshape(-1, 16)
        P = np.minimum.accumulate(runs, axis=1).reshape(-1)
        S = np.minimum.accumulate(runs[:, ::-1], axis=1)[:, ::-1].reshape(-1)
        for v in range(tile // 16):
            o0 = Hs + 16 * v
            for j in range(16):
                assert _anchor_runs(h, P, S, o0, j, r) == _anchor_def(h, o0 + j, r), (r, v, j)
                checked += 1
    assert checked > 20000


def test_backward_roll_equals_forward_codes():
    """The packed q-gram code rolled backwards (each symbol entering the top
    field, the lowest leaving) equals the forward packing of q symbols."""
    rng = np.random.default_rng(12)
    for _ in range(500):
        b = int(rng.integers(1, 9))
        q = int(rng.integers(1, 64 // b + 1))
        mask = (1 << (32 if q * b <= 32 else 64)) - 1
        chunks = (q - 1 + 15) // 16
        sym = rng.integers(0, 1 << b, size=16 * (1 + chunks) + 1)
        top = b * (q - 1)
        code = 0
        for c in range(chunks, 0, -1):
            for j in range(15, -1, -1):
                code = ((code >> b) | (int(sym[16 * c + j]) << top)) & mask
        for j in range(15, -1, -1):
            code = ((code >> b) | (int(sym[j]) << top)) & mask
            want = 0
            for k in range(q):
                want = (want << b) | int(sym[j + k])
            assert code == want
