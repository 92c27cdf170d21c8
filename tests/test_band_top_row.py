"""The per-thread verifier keeps D of its band's top row (the anchor of the
early exit, Ukkonen's diagonal bound of Sec. 3's verification) without a
per-column update: along a diagonal D rises by 0 or 1 from one column to the
next, and it rises exactly when bit 0 of (Pv | Ph) & ~(Mv | Mh) is set, where
Pv / Mv are the vertical deltas entering the top row and Ph / Mh the
horizontal deltas leaving it.  This test runs the verifier's bit-vector
recurrence (Myers' step in the banded form the kernel uses: the state kept
one row down, the band sliding one row per column, virtual rows above row 1
starting with deltas of -1) on random strings, with arbitrary symbols in the
virtual rows and past the end of A, and checks at every column that the
one-bit rise equals the signed sum of the four deltas the step produces.
It also checks the identity against the plain DP: the top row's D, followed
along the band, matches the band-restricted DP wherever the top row lies
inside the matrix."""
import random

import numpy as np


def _band_dp(A, B, dlo, rows):
    """D over rows dlo .. len(A) and columns 0 .. len(B), restricted to the
    band of `rows` rows starting at row j + dlo in column j; virtual rows
    i <= 0 start at D[i][0] = -i, cells outside the band are infinite."""
    INF = 1 << 30
    m, n = len(A), len(B)
    D = {}
    for i in range(dlo, dlo + rows):
        D[(i, 0)] = -i if i <= 0 else i
    for j in range(1, n + 1):
        top = j + dlo
        for i in range(top, top + rows):
            best = INF
            if (i - 1, j) in D and i - 1 >= top:
                best = min(best, D[(i - 1, j)] + 1)
            if (i, j - 1) in D:
                best = min(best, D[(i, j - 1)] + 1)
            if (i - 1, j - 1) in D:
                a = A.get(i)
                best = min(best, D[(i - 1, j - 1)] + (0 if a == B[j - 1] else 1))
            D[(i, j)] = best
    return D


def _run(rng, W, sig, k, m, n):
    L = 32 * W
    d0 = m - n
    dlo = -((k - d0) >> 1)
    A = {}

    def a_at(row):   # A's symbol at 1-based row; outside 1..m arbitrary (virtual or past the end)
        if row not in A:
            A[row] = rng.randrange(sig + 1)
        return A[row]

    B = [rng.randrange(sig) for _ in range(n)]
    for i in range(1, m + 1):
        A[i] = B[min(i - 1, n - 1)] if rng.random() < 0.6 else rng.randrange(sig)
    mask = (1 << L) - 1
    nneg = 1 - dlo
    Mv = (1 << nneg) - 1 if nneg < L else mask
    Pv = mask & ~Mv
    Pv = (Pv >> 1) | (1 << (L - 1))   # the state is kept one row down
    Mv >>= 1
    score = -dlo                       # D[dlo][0]
    scores = [score]
    mismatches = 0
    for j in range(1, n + 1):
        Eq = 0
        for t in range(L):
            if a_at(j + dlo + t) == B[j - 1]:
                Eq |= 1 << t
        SUM = ((Eq & Pv) + Pv) & mask
        Xv = Eq | Mv
        Xh = (SUM ^ Pv) | Eq
        Ph = (Mv | ~(Xh | Pv)) & mask
        Mh = Pv & Xh
        step = (Pv & 1) - (Mv & 1) + (Ph & 1) - (Mh & 1)
        rise = ((Pv | Ph) & ~(Mv | Mh)) & 1
        mismatches += step != rise
        score += rise
        scores.append(score)
        xs = Xv >> 1
        Pv = (Mh | ~(xs | Ph)) & mask
        Mv = Ph & xs
        Pv |= 1 << (L - 1)
    return mismatches, scores, A, B, dlo, L


def test_top_row_rise_identity():
    rng = random.Random(11)
    cols = 0
    for trial in range(800):
        W = rng.choice([1, 2, 3])
        sig = rng.choice([2, 4, 20, 95])
        k = rng.randint(0, 32 * W - 2)
        m, n = rng.randint(1, 90), rng.randint(1, 90)
        if m < n:
            m, n = n, m
        d0 = m - n
        if d0 > k or d0 - (-((k - d0) >> 1)) >= 32 * W:
            continue
        bad, _, _, _, _, _ = _run(rng, W, sig, k, m, n)
        assert bad == 0, trial
        cols += n
    assert cols > 10000


def test_top_row_score_matches_band_dp():
    rng = random.Random(5)
    for trial in range(60):
        W = rng.choice([1, 2])
        sig = rng.choice([2, 4])
        k = rng.randint(0, 32 * W - 2)
        m, n = rng.randint(1, 40), rng.randint(1, 40)
        if m < n:
            m, n = n, m
        d0 = m - n
        if d0 > k or d0 - (-((k - d0) >> 1)) >= 32 * W:
            continue
        bad, scores, A, B, dlo, L = _run(rng, W, sig, k, m, n)
        assert bad == 0
        D = _band_dp(A, B, dlo, L)
        got = np.array(scores)
        want = np.array([D[(j + dlo, j)] for j in range(n + 1)])
        assert np.array_equal(got, want), trial
