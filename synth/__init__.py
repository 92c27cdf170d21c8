"""Seeded synthetic string sets shaped like the datasets of the MinJoin paper.

The paper measures on UNIREF, TREC and the GEN* genome sets (Sec. 4.1,
Table 5).  None of them is available here, so every input is generated from a
numpy PCG64 stream with the shape of one of those workloads: alphabet, length
distribution, and families of near-duplicates produced by random edits.

This module holds no arithmetic of the join itself (no q-gram hashing, no
anchors, no edit distance).  It is the one piece of code that both the CPU
oracle side and the CUDA side of the tests import.

Edit model (all configurations): every position of a root independently
undergoes an edit with probability `rate`; the edit is an insertion, a
deletion or a substitution with equal probability.  An insertion places a new
symbol before the position and keeps the original; a substitution replaces the
symbol by a new one drawn from the same symbol distribution (it may equal the
original).  The rate is drawn per copy.

A string set is a pair (bytes, offsets): `bytes` is the uint8 concatenation of
all strings and `offsets` (int64, n+1 entries) delimits them, string i being
bytes[offsets[i]:offsets[i+1]].
"""
from __future__ import annotations

import dataclasses

import numpy as np

DNA = np.frombuffer(b"ACGT", dtype=np.uint8).copy()
PROTEIN = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", dtype=np.uint8).copy()
PRINTABLE = np.arange(0x20, 0x7F, dtype=np.uint8)
LOWER = np.arange(ord("a"), ord("z") + 1, dtype=np.uint8)


@dataclasses.dataclass
class StringSet:
    """A concatenated string set plus the join parameters of its workload."""

    name: str
    bytes: np.ndarray      # uint8, concatenation of all strings
    offsets: np.ndarray    # int64, n+1 entries
    K: int                 # edit-distance threshold
    T: int                 # targeted number of partitions per string
    family: np.ndarray     # int64, root id of every string (ground truth only)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def string(self, i: int) -> bytes:
        return self.bytes[self.offsets[i]:self.offsets[i + 1]].tobytes()


def _concat(parts: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    lens = np.fromiter((p.shape[0] for p in parts), dtype=np.int64, count=len(parts))
    offsets = np.zeros(len(parts) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    data = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    return data.astype(np.uint8, copy=False), offsets


def _draw(rng: np.random.Generator, symbols: np.ndarray, probs, size: int) -> np.ndarray:
    if probs is None:
        return symbols[rng.integers(0, symbols.shape[0], size=size)]
    return symbols[rng.choice(symbols.shape[0], size=size, p=probs)]


def mutate(rng: np.random.Generator, src: np.ndarray, rate: float,
           symbols: np.ndarray, probs=None) -> np.ndarray:
    """One mutated copy of `src` under the edit model in the module docstring."""
    L = src.shape[0]
    edit = rng.random(L) < rate
    op = rng.integers(0, 3, size=L)            # 0 insertion, 1 deletion, 2 substitution
    ins = edit & (op == 0)
    keep = ~(edit & (op == 1))
    sub = edit & (op == 2)
    kept = src.copy()
    nsub = int(sub.sum())
    if nsub:
        kept[sub] = _draw(rng, symbols, probs, nsub)
    count = ins.astype(np.int64) + keep.astype(np.int64)
    start = np.cumsum(count) - count
    out = np.empty(int(count.sum()), dtype=np.uint8)
    nins = int(ins.sum())
    if nins:
        out[start[ins]] = _draw(rng, symbols, probs, nins)
    out[(start + ins)[keep]] = kept[keep]
    return out


def mutate_many(rng: np.random.Generator, srcs: np.ndarray, src_off: np.ndarray,
                rates: np.ndarray, symbols: np.ndarray, probs=None):
    """Mutated copies of many sources at once (same edit model as `mutate`).

    `srcs`/`src_off` is a concatenated source set; copy c is drawn from source c
    at rate rates[c].  The edited positions of a copy are a Bernoulli(rate)
    process, drawn as geometric gaps.  Returns (bytes, offsets) of the copies.
    """
    L = np.diff(src_off)
    pos_parts = []
    for c in range(L.shape[0]):
        Lc, rate = int(L[c]), float(rates[c])
        if Lc == 0 or rate <= 0.0:
            continue
        got = []
        last = -1
        while True:
            g = rng.geometric(rate, size=int(Lc * rate * 1.25) + 16)
            p = last + np.cumsum(g)
            got.append(p[p < Lc])
            if p[-1] >= Lc:
                break
            last = int(p[-1])
        pos_parts.append(np.concatenate(got) + int(src_off[c]))
    pos = np.concatenate(pos_parts) if pos_parts else np.zeros(0, np.int64)
    op = rng.integers(0, 3, size=pos.shape[0])    # 0 insertion, 1 deletion, 2 substitution
    ins_pos, del_pos, sub_pos = pos[op == 0], pos[op == 1], pos[op == 2]
    data = srcs.copy()
    if sub_pos.shape[0]:
        data[sub_pos] = _draw(rng, symbols, probs, sub_pos.shape[0])
    ins_val = _draw(rng, symbols, probs, ins_pos.shape[0])
    data = np.delete(data, del_pos)
    data = np.insert(data, ins_pos - np.searchsorted(del_pos, ins_pos), ins_val)
    # a copy's first symbol sits at its source offset, shifted by the edits before it
    off = src_off + np.searchsorted(ins_pos, src_off) - np.searchsorted(del_pos, src_off)
    return data.astype(np.uint8, copy=False), off


def _families(rng, roots: list[np.ndarray], copies: int, rate_lo: float, rate_hi: float,
              symbols, probs=None, fit_len: int | None = None, chunk: int = 1 << 25):
    root_data, root_off = _concat(roots)
    nroot = len(roots)
    rates = np.full(nroot * copies, rate_lo) if rate_hi == rate_lo else \
        rng.uniform(rate_lo, rate_hi, size=nroot * copies)
    owner = np.repeat(np.arange(nroot), copies)
    parts = []
    c0 = 0
    rl = np.diff(root_off)
    while c0 < owner.shape[0]:
        # copies [c0, c1) hold at most `chunk` source symbols
        c1 = c0 + 1
        acc = rl[owner[c0]]
        while c1 < owner.shape[0] and acc + rl[owner[c1]] <= chunk:
            acc += rl[owner[c1]]
            c1 += 1
        sel = owner[c0:c1]
        src_parts = [root_data[root_off[r]:root_off[r + 1]] for r in sel]
        srcs, soff = _concat(src_parts)
        out, off = mutate_many(rng, srcs, soff, rates[c0:c1], symbols, probs)
        for k in range(c1 - c0):
            parts.append(out[off[k]:off[k + 1]])
        c0 = c1
    if fit_len is not None:
        fitted = []
        for c in parts:
            if c.shape[0] > fit_len:
                c = c[:fit_len]
            elif c.shape[0] < fit_len:
                c = np.concatenate([c, _draw(rng, symbols, probs, fit_len - c.shape[0])])
            fitted.append(c)
        parts = fitted
    perm = rng.permutation(len(parts))
    parts = [parts[p] for p in perm]
    fam = owner[perm].astype(np.int64)
    data, offsets = _concat(parts)
    return data, offsets, fam


def _zipf_text_roots(rng, n_roots: int, vocab: int = 50_000, s: float = 1.1,
                     mean_len: float = 1500.0, sd_len: float = 200.0):
    """Roots of space-joined words: word ranks ~ Zipf(s) over `vocab` random
    lowercase words of length 2..12; each root is cut to L ~ N(mean, sd), L>=100."""
    wlen = rng.integers(2, 13, size=vocab)
    letters = LOWER[rng.integers(0, 26, size=int(wlen.sum()))]
    wstart = np.cumsum(wlen) - wlen
    p = np.arange(1, vocab + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    target = np.maximum(np.rint(rng.normal(mean_len, sd_len, size=n_roots)), 100).astype(np.int64)
    mean_word = float(((wlen + 1) * 1.0).mean())
    M = int(target.sum() / mean_word * 1.3) + 64 * n_roots + 1024
    ranks = rng.choice(vocab, size=M, p=p)
    wl = wlen[ranks] + 1                                  # word plus one space
    ends = np.cumsum(wl)
    starts = ends - wl
    total = int(ends[-1])
    widx = np.repeat(np.arange(M), wl)
    inword = np.arange(total) - starts[widx]
    stream = np.full(total, 0x20, dtype=np.uint8)
    letter = inword < wlen[ranks][widx]
    stream[letter] = letters[(wstart[ranks][widx] + inword)[letter]]
    roots, w = [], 0
    for L in target:
        # the root takes whole words from word w on until it holds >= L symbols
        base = starts[w]
        e = int(np.searchsorted(ends, base + L, side="left"))
        if e >= M:
            raise RuntimeError("word stream too short")
        roots.append(stream[base:base + L].copy())
        w = e + 1
    return roots


# name, K, T, roots, copies per root
CONFIGS = {
    1: ("tiny DNA: 1,000 x 500 over ACGT, 100 roots x 10 copies at 1%", 10, 10, 100),
    2: ("read-like DNA: 50,000 x N(5000,500) over ACGT, 5,000 roots x 10 at U[1%,4%]", 100, 100, 5000),
    3: ("long noisy DNA: 20,000 x loguniform[2k,20k], 2,000 roots x 10 at U[5%,15%]", 1000, 200, 2000),
    4: ("protein-like: 400,000 x lognormal(median 400), 20 letters Dirichlet(2), 40,000 roots x 10 at U[2%,10%]", 40, 40, 40000),
    5: ("text-like: 300,000 x ~1,500 bytes of Zipf(1.1) words, 30,000 roots x 10 at U[1%,8%]", 75, 75, 30000),
}


def make_config(cfg: int, seed: int | None = None, n_roots: int | None = None) -> StringSet:
    """Generate workload `cfg` (1..5) at `seed` (default: the config number).

    `n_roots` scales the workload down (same distributions, fewer families);
    every family has 10 mutated copies of one random root.
    """
    name, K, T, roots_default = CONFIGS[cfg]
    seed = cfg if seed is None else seed
    nr = roots_default if n_roots is None else n_roots
    rng = np.random.Generator(np.random.PCG64(seed))
    copies = 10
    if cfg == 1:
        roots = [_draw(rng, DNA, None, 500) for _ in range(nr)]
        data, off, fam = _families(rng, roots, copies, 0.01, 0.01, DNA, fit_len=500)
    elif cfg == 2:
        lens = np.clip(np.rint(rng.normal(5000, 500, size=nr)), 3000, 7000).astype(np.int64)
        roots = [_draw(rng, DNA, None, int(L)) for L in lens]
        data, off, fam = _families(rng, roots, copies, 0.01, 0.04, DNA)
    elif cfg == 3:
        lens = np.rint(np.exp(rng.uniform(np.log(2000), np.log(20000), size=nr))).astype(np.int64)
        roots = [_draw(rng, DNA, None, int(L)) for L in lens]
        data, off, fam = _families(rng, roots, copies, 0.05, 0.15, DNA)
    elif cfg == 4:
        freq = rng.dirichlet(np.full(PROTEIN.shape[0], 2.0))
        lens = np.clip(np.rint(np.exp(rng.normal(np.log(400), 0.462, size=nr))), 50, 5000).astype(np.int64)
        roots = [_draw(rng, PROTEIN, freq, int(L)) for L in lens]
        data, off, fam = _families(rng, roots, copies, 0.02, 0.10, PROTEIN, freq)
    elif cfg == 5:
        roots = _zipf_text_roots(rng, nr)
        data, off, fam = _families(rng, roots, copies, 0.01, 0.08, PRINTABLE)
    else:
        raise ValueError(f"unknown configuration {cfg}")
    return StringSet(name=name, bytes=data, offsets=off, K=K, T=T, family=fam)


def random_set(seed: int, n: int, min_len: int, max_len: int, symbols: np.ndarray = DNA,
               K: int = 4, T: int = 4, families: int = 0, rate: float = 0.05) -> StringSet:
    """Small mixed set for edge-case tests: `families` groups of near copies plus
    independent random strings with uniform lengths in [min_len, max_len]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts, fam = [], []
    f = 0
    while len(parts) < n:
        L = int(rng.integers(min_len, max_len + 1))
        root = _draw(rng, symbols, None, L)
        if families and f < families:
            for _ in range(min(10, n - len(parts))):
                parts.append(mutate(rng, root, rate, symbols))
                fam.append(f)
            f += 1
        else:
            parts.append(root)
            fam.append(f)
            f += 1
    data, off = _concat(parts)
    return StringSet(name=f"random seed={seed}", bytes=data, offsets=off, K=K, T=T,
                     family=np.asarray(fam, np.int64))


def from_strings(strings: list[bytes], K: int, T: int, name: str = "explicit") -> StringSet:
    parts = [np.frombuffer(s, dtype=np.uint8).copy() for s in strings]
    data, off = _concat(parts)
    return StringSet(name=name, bytes=data, offsets=off, K=K, T=T,
                     family=np.arange(len(strings), dtype=np.int64))
