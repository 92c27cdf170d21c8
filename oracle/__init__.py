"""CPU oracle for the MinJoin edit-similarity join (test infrastructure only).

Plain restatement of the paper's algorithms (Alg. 1-3, Ukkonen's banded DP of
Sec. 3) in `minjoin_oracle.cpp`, driven from here through ctypes.  Only the
tests, the smoke check of the entry module and the CPU-baseline leg of the
benchmark may import this package; the product path never does.

Threading: partitioning (per string) and verification (per pair) are split
into chunks run on a thread pool; ctypes releases the GIL during each call.
The hash join of Alg. 3 runs sequentially, as in the paper.

Parallel repetition (Sec. 2.2, Thm 1) is the union of the partitions made
under R independent random functions Pi; `partition_repeated` builds it from
R calls of `partition`.  It is pinned by properties, not by printed values:
R = 1 is the plain partition, every repetition tiles every string, and the
candidates and the recall never shrink as R grows.
"""
from __future__ import annotations

import contextlib
import ctypes
import dataclasses
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "minjoin_oracle.cpp")
_LIB = os.path.join(_HERE, "libminjoin_oracle.so")
_lock = threading.Lock()
_lib = None

I64P = ctypes.POINTER(ctypes.c_int64)
U8P = ctypes.POINTER(ctypes.c_uint8)
U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no GPU involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.mjo_q_rule.restype = ctypes.c_uint32
    lib.mjo_q_rule.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
    lib.mjo_radius.restype = ctypes.c_int64
    lib.mjo_radius.argtypes = [ctypes.c_int64] * 4
    lib.mjo_hash_qgrams.restype = None
    lib.mjo_hash_qgrams.argtypes = [U8P, ctypes.c_int64, ctypes.c_int32, U8P, ctypes.c_int32,
                                    ctypes.c_uint64, U64P, U64P]
    lib.mjo_find_anchors.restype = ctypes.c_int64
    lib.mjo_find_anchors.argtypes = [U64P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, I64P]
    lib.mjo_partition_range.restype = ctypes.c_int64
    lib.mjo_partition_range.argtypes = [U8P, I64P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.c_int64, U8P, ctypes.c_int32,
                                        ctypes.c_uint64, U64P, I64P, I64P, I64P, ctypes.c_int64, I64P]
    lib.mjo_candidates.restype = ctypes.c_int64
    lib.mjo_candidates.argtypes = [U8P, I64P, ctypes.c_int64, ctypes.c_int64, I64P, I64P, I64P,
                                   ctypes.c_int64, ctypes.POINTER(I64P)]
    lib.mjo_free.restype = None
    lib.mjo_free.argtypes = [ctypes.c_void_p]
    lib.mjo_ed_full.restype = ctypes.c_int64
    lib.mjo_ed_full.argtypes = [U8P, ctypes.c_int64, U8P, ctypes.c_int64]
    lib.mjo_ed_band.restype = ctypes.c_int64
    lib.mjo_ed_band.argtypes = [U8P, ctypes.c_int64, U8P, ctypes.c_int64, ctypes.c_int64]
    lib.mjo_ed_band_pairs.restype = None
    lib.mjo_ed_band_pairs.argtypes = [U8P, I64P, I64P, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int64, I64P]
    lib.mjo_ed_band_cutoff.restype = ctypes.c_int64
    lib.mjo_ed_band_cutoff.argtypes = [U8P, ctypes.c_int64, U8P, ctypes.c_int64, ctypes.c_int64]
    lib.mjo_ed_band_cutoff_pairs.restype = None
    lib.mjo_ed_band_cutoff_pairs.argtypes = [U8P, I64P, I64P, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, I64P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


@contextlib.contextmanager
def using(path: str):
    """Run the wrapper functions against another build of the oracle source
    (the tests use this to show that the pins reject a planted mistake)."""
    global _lib
    prev = _load()
    with _lock:
        _lib = _bind(path)
    try:
        yield
    finally:
        with _lock:
            _lib = prev


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- parameters

@dataclasses.dataclass
class Params:
    """Parameters of one join (Sec. 2.1-2.2, Alg. 2-3)."""
    K: int
    T: int
    q: int
    r_min: int
    seed: int
    sigma: int
    bits: int
    rank: np.ndarray        # uint8[256]: rank code of every byte value present
    N: int


def alphabet(data: np.ndarray) -> tuple[np.ndarray, int, int]:
    """Sigma = the distinct byte values present, ranked ascending (codes
    0..|Sigma|-1), with bits = max(1, ceil(log2 |Sigma|)) per code."""
    present = np.zeros(256, dtype=bool)
    if data.shape[0]:
        present[np.unique(data)] = True
    rank = np.zeros(256, dtype=np.uint8)
    vals = np.nonzero(present)[0]
    rank[vals] = np.arange(vals.shape[0], dtype=np.uint8) if vals.shape[0] <= 256 else 0
    sigma = int(vals.shape[0])
    bits = 1
    while (1 << bits) < sigma:
        bits += 1
    return rank, sigma, bits


def q_rule(N: int, T: int, sigma: int) -> int:
    return int(_load().mjo_q_rule(N, T, sigma))


def radius(slen: int, q: int, T: int, r_min: int) -> int:
    return int(_load().mjo_radius(slen, q, T, r_min))


def derive_params(data: np.ndarray, offsets: np.ndarray, K: int, T: int = 0, q: int = 0,
                  r_min: int = 1, seed: int = 0x5EED) -> Params:
    """Sec. 2.2: Sigma from the bytes present, N = max length, T = K unless
    given, q = the rounded-up rule of mjo_q_rule unless given, then capped so
    that a packed q-gram fits 64 bits."""
    rank, sigma, bits = alphabet(data)
    lens = np.diff(offsets)
    N = int(lens.max()) if lens.shape[0] else 0
    T = K if T == 0 else T
    if q == 0:
        q = q_rule(N, T, sigma)
    q = max(1, min(q, 64 // bits))
    return Params(K=K, T=T, q=q, r_min=r_min, seed=seed, sigma=sigma, bits=bits, rank=rank, N=N)


# ---------------------------------------------------------------- partitions

def hash_qgrams(s: bytes, p: Params, table: np.ndarray | None = None) -> np.ndarray:
    lib = _load()
    a = _u8(s)
    m = max(0, a.shape[0] - p.q + 1)
    h = np.zeros(max(m, 1), dtype=np.uint64)
    tab = None if table is None else np.ascontiguousarray(table, dtype=np.uint64)
    if m:
        lib.mjo_hash_qgrams(_p(a, U8P), a.shape[0], p.q, _p(p.rank, U8P), p.bits, p.seed,
                            None if tab is None else _p(tab, U64P), _p(h, U64P))
    return h[:m]


def find_anchors(h: np.ndarray, slen: int, r: int) -> np.ndarray:
    lib = _load()
    h = np.ascontiguousarray(h, dtype=np.uint64)
    out = np.zeros(h.shape[0] + 2, dtype=np.int64)
    hp = _p(h, U64P) if h.shape[0] else None
    k = lib.mjo_find_anchors(hp, h.shape[0], slen, r, _p(out, I64P))
    return out[:k]


@dataclasses.dataclass
class Partitions:
    sid: np.ndarray
    pos: np.ndarray
    len: np.ndarray
    n_anchor: np.ndarray    # anchors per string (partitions + 1, or 1 for an empty string)


def partition(data: np.ndarray, offsets: np.ndarray, p: Params, table: np.ndarray | None = None,
              threads: int | None = None, lo: int = 0, hi: int | None = None) -> Partitions:
    """Alg. 1 on strings [lo, hi) (all by default), chunked over threads."""
    lib = _load()
    data = _u8(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = offsets.shape[0] - 1
    hi = n if hi is None else hi
    tab = None if table is None else np.ascontiguousarray(table, dtype=np.uint64)
    threads = threads or default_threads()
    bounds = np.linspace(lo, hi, num=min(max(1, (hi - lo) // 64), threads * 8) + 1).astype(np.int64)
    bounds = np.unique(bounds)

    def run(a, b):
        nbytes = int(offsets[b] - offsets[a])
        cap = nbytes + 2 * (b - a) + 16
        sid = np.empty(cap, np.int64)
        pos = np.empty(cap, np.int64)
        ln = np.empty(cap, np.int64)
        na = np.empty(max(b - a, 1), np.int64)
        k = lib.mjo_partition_range(_p(data, U8P) if data.shape[0] else None, _p(offsets, I64P), a, b, p.q,
                                    p.T, p.r_min, _p(p.rank, U8P), p.bits, p.seed,
                                    None if tab is None else _p(tab, U64P), _p(sid, I64P), _p(pos, I64P),
                                    _p(ln, I64P), cap, _p(na, I64P))
        if k < 0:
            raise RuntimeError("partition capacity exceeded")
        return sid[:k], pos[:k], ln[:k], na[:b - a]

    if bounds.shape[0] < 2:
        z = np.zeros(0, np.int64)
        return Partitions(z, z, z, z)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda ab: run(*ab), zip(bounds[:-1], bounds[1:])))
    return Partitions(np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res]),
                      np.concatenate([r[2] for r in res]), np.concatenate([r[3] for r in res]))


REPETITION_STEP = 0x9E3779B97F4A7C15   # Weyl step between the seeds of repeated Pi functions


def repetition_seed(seed: int, k: int) -> int:
    """Seed of Pi_k under parallel repetition: seed + k * 0x9E3779B97F4A7C15
    modulo 2^64 (k = 0 is the base seed; the partition key keeps it)."""
    return (seed + k * REPETITION_STEP) % (1 << 64)


def partition_repeated(data: np.ndarray, offsets: np.ndarray, p: Params, repeats: int,
                       threads: int | None = None) -> Partitions:
    """Sec. 2.2's parallel repetition: the union of the partitions of every
    string under Pi_0 .. Pi_{R-1}, ordered by string, then repetition, then
    position.  n_anchor sums the anchors of the R partitionings."""
    parts = [partition(data, offsets, dataclasses.replace(p, seed=repetition_seed(p.seed, k)), threads=threads)
             for k in range(repeats)]
    sid = np.concatenate([q.sid for q in parts])
    order = np.argsort(sid, kind="stable")
    return Partitions(sid[order], np.concatenate([q.pos for q in parts])[order],
                      np.concatenate([q.len for q in parts])[order], sum(q.n_anchor for q in parts))


# ---------------------------------------------------------------- join

def candidates(data: np.ndarray, offsets: np.ndarray, K: int, parts: Partitions) -> np.ndarray:
    """Alg. 3's hash join (sort, both filters, eviction, dedup), sequential.
    Returns an (m, 2) int64 array of distinct pairs i < j, sorted."""
    lib = _load()
    data = _u8(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = offsets.shape[0] - 1
    outp = I64P()
    sid = np.ascontiguousarray(parts.sid, np.int64)
    pos = np.ascontiguousarray(parts.pos, np.int64)
    ln = np.ascontiguousarray(parts.len, np.int64)
    z = np.zeros(1, np.int64)
    k = lib.mjo_candidates(_p(data, U8P) if data.shape[0] else None, _p(offsets, I64P), n, K,
                           _p(sid if sid.shape[0] else z, I64P), _p(pos if pos.shape[0] else z, I64P),
                           _p(ln if ln.shape[0] else z, I64P), sid.shape[0], ctypes.byref(outp))
    try:
        arr = np.ctypeslib.as_array(outp, shape=(max(k, 1) * 2,))[:2 * k].copy()
    finally:
        lib.mjo_free(outp)
    return arr.reshape(k, 2)


def ed_full(a: bytes, b: bytes) -> int:
    lib = _load()
    x, y = _u8(a), _u8(b)
    return int(lib.mjo_ed_full(_p(x, U8P) if x.shape[0] else None, x.shape[0],
                               _p(y, U8P) if y.shape[0] else None, y.shape[0]))


def ed_band(a: bytes, b: bytes, k: int) -> int:
    lib = _load()
    x, y = _u8(a), _u8(b)
    return int(lib.mjo_ed_band(_p(x, U8P) if x.shape[0] else None, x.shape[0],
                               _p(y, U8P) if y.shape[0] else None, y.shape[0], k))


def ed_band_cutoff(a: bytes, b: bytes, k: int) -> int:
    """ed_band with Ukkonen's cut-off (stops once a whole band row exceeds k)."""
    lib = _load()
    x, y = _u8(a), _u8(b)
    return int(lib.mjo_ed_band_cutoff(_p(x, U8P) if x.shape[0] else None, x.shape[0],
                                      _p(y, U8P) if y.shape[0] else None, y.shape[0], k))


def ed_band_pairs(data: np.ndarray, offsets: np.ndarray, pairs: np.ndarray, k: int,
                  threads: int | None = None, cutoff: bool = False) -> np.ndarray:
    """min(ED, k+1) of every pair (banded DP), chunked over threads; with
    cutoff=True each DP stops once a whole band row exceeds k (same values)."""
    lib = _load()
    data = _u8(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    m = pairs.shape[0]
    out = np.zeros(max(m, 1), np.int64)
    if m == 0:
        return out[:0]
    threads = threads or default_threads()
    bounds = np.unique(np.linspace(0, m, num=min(m, threads * 16) + 1).astype(np.int64))
    dp = _p(data, U8P) if data.shape[0] else None

    fn = lib.mjo_ed_band_cutoff_pairs if cutoff else lib.mjo_ed_band_pairs

    def run(a, b):
        fn(dp, _p(offsets, I64P), _p(pairs, I64P), a, b, k, _p(out, I64P))

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda ab: run(*ab), zip(bounds[:-1], bounds[1:])))
    return out[:m]


@dataclasses.dataclass
class JoinResult:
    pairs: np.ndarray        # (r, 2) int64, i < j, sorted
    ed: np.ndarray           # (r,) int64, each <= K
    candidates: np.ndarray   # (c, 2) int64, the deduplicated candidate set C
    cand_ed: np.ndarray      # (c,) int64, min(ED, K+1) of every candidate
    parts: Partitions
    params: Params


def minjoin(data: np.ndarray, offsets: np.ndarray, K: int, T: int = 0, q: int = 0, r_min: int = 1,
            seed: int = 0x5EED, table: np.ndarray | None = None, threads: int | None = None,
            repeats: int = 1) -> JoinResult:
    """Alg. 3 end to end: partition every string (Alg. 1-2; with repeats > 1
    the union under independent Pi functions, Sec. 2.2), hash join with the
    length and position filters, dedup, then verify every candidate with
    Ukkonen's banded DP and keep the pairs with ED <= K."""
    data = _u8(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    p = derive_params(data, offsets, K, T, q, r_min, seed)
    if repeats > 1:
        if table is not None:
            raise ValueError("an explicit Pi table allows no repetition")
        parts = partition_repeated(data, offsets, p, repeats, threads=threads)
    else:
        parts = partition(data, offsets, p, table=table, threads=threads)
    C = candidates(data, offsets, K, parts)
    ed = ed_band_pairs(data, offsets, C, K, threads=threads)
    keep = ed <= K
    return JoinResult(pairs=C[keep], ed=ed[keep], candidates=C, cand_ed=ed, parts=parts, params=p)
