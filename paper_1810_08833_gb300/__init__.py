"""Python binding of the GB300 MinJoin library (include/minjoin.h).

Argument marshalling only: every step of the join runs in the CUDA kernels of
libminjoin.so.  PyTorch supplies device memory and the current stream.  There
is no CPU fallback: if the library is missing or no GPU is present, the calls
raise.

Functions mirror the C entry points:
    derive      mj_derive       step a1 (Sec. 2.2 parameters)
    partition   mj_partition    steps a2-a4 (Alg. 1-2)
    candidates  mj_candidates   steps a2-a7 (Alg. 3's hash join)
    verify      mj_verify       step a8 (Ukkonen band, Sec. 3)
    join        mj_join         the whole path (Alg. 3)
    join_host   mj_join_host    the whole path from/to host memory
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libminjoin.so")

MJ_VERIFY_PLAIN = 0
MJ_VERIFY_LEARNED = 1


class MinJoinError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_uint32), ("T", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("r_min", ctypes.c_int32), ("seed", ctypes.c_uint64), ("verify_mode", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("repeats", ctypes.c_uint32)]


class Derived(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_uint32), ("bits", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("T", ctypes.c_uint32), ("K", ctypes.c_uint32), ("r_max", ctypes.c_int32),
                ("N", ctypes.c_uint64), ("rank", ctypes.c_uint8 * 256), ("input_max_len", ctypes.c_uint64),
                ("present", ctypes.c_uint8 * 256)]


class BandTrainParams(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("batch", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("tau", ctypes.c_float), ("seed", ctypes.c_uint64)]


class BandCalibration(ctypes.Structure):
    _fields_ = [("plain_ms", ctypes.c_float), ("learned_ms", ctypes.c_float),
                ("plain_word_columns", ctypes.c_uint64), ("learned_word_columns", ctypes.c_uint64),
                ("first_pass_settled", ctypes.c_uint64), ("enabled", ctypes.c_uint32)]


MJ_FLAG_KEY_CHECK = 1
MJ_FLAG_FEATURES = 16
MJ_FLAG_FIRST_PASS = 32
MJ_FLAG_DEDUP_SORT = 64
MJ_FLAG_DEDUP_BITMAP = 128
BAND_FEATURES = 8
BAND_PARAMS = 4801


class VerifyConfig(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_uint32), ("lanes", ctypes.c_uint32), ("batching", ctypes.c_uint32),
                ("graph", ctypes.c_uint32)]


class AutotuneReport(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint32 * 32), ("kernel", ctypes.c_uint32 * 32), ("lanes", ctypes.c_uint32 * 32),
                ("ms", (ctypes.c_float * 6) * 32), ("cand_kernel", ctypes.c_uint32 * 6),
                ("cand_lanes", ctypes.c_uint32 * 6), ("n_candidates", ctypes.c_uint32)]


MJ_VERIFY_KERNEL_AUTO = 0
MJ_VERIFY_KERNEL_DIAGONAL = 1
MJ_VERIFY_KERNEL_WAVEFRONT = 2
MJ_VERIFY_KERNEL_TUNED = 3


class Stats(ctypes.Structure):
    _fields_ = [("n_strings", ctypes.c_uint64), ("n_bytes", ctypes.c_uint64), ("n_partitions", ctypes.c_uint64),
                ("n_raw_pairs", ctypes.c_uint64), ("n_candidates", ctypes.c_uint64),
                ("n_output", ctypes.c_uint64), ("key_collisions", ctypes.c_uint64),
                ("band_cells", ctypes.c_uint64), ("first_pass_settled", ctypes.c_uint64),
                ("fallback_pairs", ctypes.c_uint64), ("device_flags", ctypes.c_uint32),
                ("ms_derive", ctypes.c_float), ("ms_partition", ctypes.c_float),
                ("ms_join_filter", ctypes.c_float), ("ms_verify", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("n_launches", ctypes.c_uint64), ("ms_section", ctypes.c_float * 9),
                ("verify_word_columns", ctypes.c_uint64)]

SECTIONS = ("anchor_test", "partition_records", "record_sort", "pair_emission", "pair_dedup", "eq_planes",
            "verify_kernel", "output_compaction", "verify_order")


VP = ctypes.c_void_p
U64 = ctypes.c_uint64
U32 = ctypes.c_uint32

_SIGS = {
    "mj_params_default": (None, [ctypes.POINTER(Params), U32]),
    "mj_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mj_create": (ctypes.c_int, [ctypes.POINTER(VP), ctypes.c_int]),
    "mj_destroy": (None, [VP]),
    "mj_get_stats": (ctypes.c_int, [VP, ctypes.POINTER(Stats)]),
    "mj_set_verify_config": (ctypes.c_int, [VP, ctypes.POINTER(VerifyConfig)]),
    "mj_autotune_verify": (ctypes.c_int, [VP, VP, VP, U32, VP, VP, U64, U32, U32, VP, ctypes.POINTER(AutotuneReport)]),
    "mj_derive": (ctypes.c_int, [VP, VP, VP, U32, ctypes.POINTER(Params), VP, ctypes.POINTER(Derived)]),
    "mj_partition": (ctypes.c_int, [VP, VP, VP, U32, ctypes.POINTER(Params), VP, VP, ctypes.POINTER(U64)]),
    "mj_partition_copy": (ctypes.c_int, [VP, VP, VP, VP, VP, VP]),
    "mj_candidates": (ctypes.c_int, [VP, VP, VP, U32, ctypes.POINTER(Params), VP, VP, ctypes.POINTER(U64)]),
    "mj_candidates_copy": (ctypes.c_int, [VP, VP, VP, VP]),
    "mj_verify": (ctypes.c_int, [VP, VP, VP, U32, VP, VP, VP, U64, U32, VP, VP]),
    "mj_verify_static": (ctypes.c_int, [VP, VP, U32, VP, VP, U64, U32, VP, VP]),
    "mj_device_flags": (ctypes.c_int, [VP, VP, ctypes.POINTER(U32)]),
    "mj_verify_static_flags": (ctypes.c_int, [VP, ctypes.POINTER(U32)]),
    "mj_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int64]),
    "mj_set_alphabet": (ctypes.c_int, [VP, VP, U64]),
    "mj_candidates_records": (ctypes.c_int, [VP, VP, VP, VP, VP, VP, U64, U32, ctypes.POINTER(Params), VP,
                                             ctypes.POINTER(U64)]),
    "mj_pairs_unique": (ctypes.c_int, [VP, VP, VP, U64, U32, VP, ctypes.POINTER(U64)]),
    "mj_band_calibrate": (ctypes.c_int, [VP, VP, VP, U32, ctypes.POINTER(Params), VP,
                                         ctypes.POINTER(BandCalibration)]),
    "mj_join": (ctypes.c_int, [VP, VP, VP, U32, ctypes.POINTER(Params), VP, ctypes.POINTER(U64)]),
    "mj_result_copy": (ctypes.c_int, [VP, VP, VP, VP, VP]),
    "mj_join_host": (ctypes.c_int, [VP, VP, VP, U32, ctypes.POINTER(Params), VP, ctypes.POINTER(U64)]),
    "mj_result_copy_host": (ctypes.c_int, [VP, VP, VP, VP, VP]),
    "mj_features_copy": (ctypes.c_int, [VP, VP, VP, VP, VP, ctypes.POINTER(U64), VP]),
    "mj_band_init": (ctypes.c_int, [VP, U64, U32, U32]),
    "mj_band_train": (ctypes.c_int, [VP, VP, VP, U64, U32, ctypes.POINTER(BandTrainParams), VP,
                                     ctypes.POINTER(ctypes.c_float)]),
    "mj_band_forward": (ctypes.c_int, [VP, VP, U64, VP, VP]),
    "mj_band_grad": (ctypes.c_int, [VP, VP, VP, U64, ctypes.c_float, VP, VP, ctypes.POINTER(ctypes.c_float)]),
    "mj_band_get_weights": (ctypes.c_int, [VP, VP, U64]),
    "mj_band_set_weights": (ctypes.c_int, [VP, VP, U64]),
    "mj_band_save": (ctypes.c_int, [VP, ctypes.c_char_p]),
    "mj_band_load": (ctypes.c_int, [VP, ctypes.c_char_p]),
}

_lib = None


def library(path: str | None = None) -> ctypes.CDLL:
    """Load libminjoin.so (built by paper_1810_08833_gb300.build.build())."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"MinJoin CUDA library not built: {p} is missing "
                               "(run paper_1810_08833_gb300.build.build())")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(status: int, where: str):
    if status != 0:
        raise MinJoinError(status, where, library().mj_strerror(status).decode())


def params(K: int, T: int = 0, q: int = 0, r_min: int = 1, seed: int = 0x5EED,
           verify_mode: int = MJ_VERIFY_PLAIN, flags: int = 0, repeats: int = 1) -> Params:
    p = Params()
    library().mj_params_default(ctypes.byref(p), K)
    p.T, p.q, p.r_min, p.seed, p.verify_mode, p.flags = T, q, r_min, seed, verify_mode, flags
    p.repeats = repeats
    return p


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr() if t.numel() else None


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check_inputs(data, offsets):
    import torch
    if not (data.is_cuda and offsets.is_cuda):
        raise ValueError("bytes and offsets must be CUDA tensors")
    if data.dtype != torch.uint8 or offsets.dtype != torch.int64:
        raise ValueError("bytes must be uint8 and offsets int64")
    if not (data.is_contiguous() and offsets.is_contiguous()):
        raise ValueError("bytes and offsets must be contiguous")
    return offsets.numel() - 1


class Context:
    """One mj_ctx on a CUDA device (not thread-safe)."""

    def __init__(self, device: int = 0):
        self._lib = library()
        h = VP()
        _check(self._lib.mj_create(ctypes.byref(h), device), "mj_create")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.mj_get_stats(self._h, ctypes.byref(s)), "mj_get_stats")
        out = {name: getattr(s, name) for name, _ in Stats._fields_ if name != "ms_section"}
        out["ms_section"] = dict(zip(SECTIONS, list(s.ms_section)))
        return out

    def set_verify_config(self, kernel: int = MJ_VERIFY_KERNEL_AUTO, lanes: int = 0, batching: int = 0,
                          graph: int = 0):
        cfg = VerifyConfig(kernel, lanes, batching, graph)
        _check(self._lib.mj_set_verify_config(self._h, ctypes.byref(cfg)), "mj_set_verify_config")

    def autotune_verify(self, data, offsets, i, j, K: int, sample: int = 4096, stream=None) -> dict:
        n = _check_inputs(data, offsets)
        rep = AutotuneReport()
        _check(self._lib.mj_autotune_verify(self._h, _ptr(data), _ptr(offsets), n, _ptr(i), _ptr(j), i.numel(), K,
                                            sample, _stream(stream), ctypes.byref(rep)), "mj_autotune_verify")
        cands = [(rep.cand_kernel[k], rep.cand_lanes[k]) for k in range(rep.n_candidates)]
        buckets = {}
        for b in range(32):
            if rep.count[b]:
                buckets[b] = {"pairs": rep.count[b], "kernel": rep.kernel[b], "lanes": rep.lanes[b],
                              "ms": {f"{k}/{l}": round(rep.ms[b][c], 4) for c, (k, l) in enumerate(cands)}}
        return {"candidates": cands, "buckets": buckets}

    def derive(self, data, offsets, p: Params, stream=None) -> dict:
        n = _check_inputs(data, offsets)
        d = Derived()
        _check(self._lib.mj_derive(self._h, _ptr(data), _ptr(offsets), n, ctypes.byref(p), _stream(stream),
                                   ctypes.byref(d)), "mj_derive")
        return {"sigma": d.sigma, "bits": d.bits, "q": d.q, "T": d.T, "K": d.K, "r_max": d.r_max, "N": d.N,
                "rank": np.frombuffer(bytes(d.rank), dtype=np.uint8).copy(), "input_max_len": d.input_max_len,
                "present": np.frombuffer(bytes(d.present), dtype=np.uint8).astype(bool)}

    def partition(self, data, offsets, p: Params, table=None, stream=None):
        import torch
        n = _check_inputs(data, offsets)
        cnt = U64()
        _check(self._lib.mj_partition(self._h, _ptr(data), _ptr(offsets), n, ctypes.byref(p), _ptr(table),
                                      _stream(stream), ctypes.byref(cnt)), "mj_partition")
        m = cnt.value
        dev = data.device
        sid = torch.empty(m, dtype=torch.int32, device=dev)
        pos = torch.empty(m, dtype=torch.int32, device=dev)
        ln = torch.empty(m, dtype=torch.int32, device=dev)
        key = torch.empty(m, dtype=torch.int64, device=dev)
        _check(self._lib.mj_partition_copy(self._h, _ptr(sid), _ptr(pos), _ptr(ln), _ptr(key), _stream(stream)),
               "mj_partition_copy")
        return sid, pos, ln, key

    def candidates(self, data, offsets, p: Params, table=None, stream=None):
        import torch
        n = _check_inputs(data, offsets)
        cnt = U64()
        _check(self._lib.mj_candidates(self._h, _ptr(data), _ptr(offsets), n, ctypes.byref(p), _ptr(table),
                                       _stream(stream), ctypes.byref(cnt)), "mj_candidates")
        m = cnt.value
        ci = torch.empty(m, dtype=torch.int32, device=data.device)
        cj = torch.empty(m, dtype=torch.int32, device=data.device)
        _check(self._lib.mj_candidates_copy(self._h, _ptr(ci), _ptr(cj), _stream(stream)), "mj_candidates_copy")
        return ci, cj

    def set_alphabet(self, present=None, N: int = 0):
        """Fix Sigma (256 presence flags) and the longest length N for later
        calls (a sharded join's global values); None reverts."""
        if present is None:
            _check(self._lib.mj_set_alphabet(self._h, None, 0), "mj_set_alphabet")
            return
        buf = (ctypes.c_uint8 * 256)(*[1 if x else 0 for x in np.asarray(present).tolist()])
        _check(self._lib.mj_set_alphabet(self._h, ctypes.cast(buf, VP), int(N)), "mj_set_alphabet")

    def _copy_candidates(self, m: int, device):
        import torch
        ci = torch.empty(m, dtype=torch.int32, device=device)
        cj = torch.empty(m, dtype=torch.int32, device=device)
        _check(self._lib.mj_candidates_copy(self._h, _ptr(ci), _ptr(cj), None), "mj_candidates_copy")
        return ci, cj

    def candidates_records(self, sid, pos, ln, key, slen, n_strings: int, p: Params, stream=None):
        """Candidate pairs (i < j, sorted) from partition records (int32 sid,
        pos, len, slen; int64 key), all CUDA tensors of one size."""
        import torch
        m = sid.numel()
        for t, dt in ((sid, torch.int32), (pos, torch.int32), (ln, torch.int32), (key, torch.int64),
                      (slen, torch.int32)):
            if not t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.numel() != m:
                raise ValueError("records must be contiguous CUDA tensors (int32; key int64) of one size")
        cnt = U64()
        _check(self._lib.mj_candidates_records(self._h, _ptr(sid), _ptr(pos), _ptr(ln), _ptr(key), _ptr(slen), m,
                                               int(n_strings), ctypes.byref(p), _stream(stream), ctypes.byref(cnt)),
               "mj_candidates_records")
        return self._copy_candidates(cnt.value, sid.device)

    def pairs_unique(self, i, j, n_strings: int, stream=None):
        """The distinct pairs (min, max) among (i[t], j[t]), sorted."""
        import torch
        m = i.numel()
        for t in (i, j):
            if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous() or t.numel() != m:
                raise ValueError("pair tensors must be contiguous int32 CUDA tensors of one size")
        cnt = U64()
        _check(self._lib.mj_pairs_unique(self._h, _ptr(i), _ptr(j), m, int(n_strings), _stream(stream),
                                         ctypes.byref(cnt)), "mj_pairs_unique")
        return self._copy_candidates(cnt.value, i.device)

    def verify(self, data, offsets, i, j, K: int, k=None, stream=None):
        import torch
        n = _check_inputs(data, offsets)
        m = i.numel()
        for t in (i, j) + ((k,) if k is not None else ()):
            if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous() or t.numel() != m:
                raise ValueError("pair index and band tensors must be contiguous int32 CUDA tensors of equal size")
        ed = torch.empty(m, dtype=torch.int32, device=data.device)
        _check(self._lib.mj_verify(self._h, _ptr(data), _ptr(offsets), n, _ptr(i), _ptr(j), _ptr(k), m, K,
                                   _stream(stream), _ptr(ed)), "mj_verify")
        return ed

    def device_flags(self, stream=None) -> int:
        f = U32()
        _check(self._lib.mj_device_flags(self._h, _stream(stream), ctypes.byref(f)), "mj_device_flags")
        return f.value

    def join(self, data, offsets, p: Params, stream=None):
        import torch
        n = _check_inputs(data, offsets)
        cnt = U64()
        _check(self._lib.mj_join(self._h, _ptr(data), _ptr(offsets), n, ctypes.byref(p), _stream(stream),
                                 ctypes.byref(cnt)), "mj_join")
        m = cnt.value
        oi = torch.empty(m, dtype=torch.int32, device=data.device)
        oj = torch.empty(m, dtype=torch.int32, device=data.device)
        oe = torch.empty(m, dtype=torch.int32, device=data.device)
        _check(self._lib.mj_result_copy(self._h, _ptr(oi), _ptr(oj), _ptr(oe), _stream(stream)), "mj_result_copy")
        return oi, oj, oe

    # ---- learned first-pass band
    def features(self, stream=None):
        """Features, band-K results and pairs of every candidate of the last
        join run with MJ_FLAG_FEATURES (or in learned mode)."""
        import torch
        cnt = U64()
        _check(self._lib.mj_features_copy(self._h, None, None, None, None, ctypes.byref(cnt), _stream(stream)),
               "mj_features_copy")
        m = cnt.value
        x = torch.empty((m, BAND_FEATURES), dtype=torch.float32, device="cuda")
        ed = torch.empty(m, dtype=torch.int32, device="cuda")
        ci = torch.empty(m, dtype=torch.int32, device="cuda")
        cj = torch.empty(m, dtype=torch.int32, device="cuda")
        _check(self._lib.mj_features_copy(self._h, _ptr(x), _ptr(ed), _ptr(ci), _ptr(cj), None, _stream(stream)),
               "mj_features_copy")
        return x, ed, ci, cj

    def band_init(self, seed: int = 1, margin: int = 0, min_multiplicity: int = 0):
        _check(self._lib.mj_band_init(self._h, seed, margin, min_multiplicity), "mj_band_init")

    def band_train(self, x, ed, K: int, steps: int = 2000, batch: int = 1024, lr: float = 1e-3, tau: float = 0.9,
                   seed: int = 1, stream=None) -> float:
        tp = BandTrainParams(steps, batch, lr, tau, seed)
        loss = ctypes.c_float()
        _check(self._lib.mj_band_train(self._h, _ptr(x), _ptr(ed), x.shape[0], K, ctypes.byref(tp), _stream(stream),
                                       ctypes.byref(loss)), "mj_band_train")
        return loss.value

    def band_forward(self, x, stream=None):
        import torch
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(self._lib.mj_band_forward(self._h, _ptr(x), x.shape[0], _stream(stream), _ptr(out)), "mj_band_forward")
        return out

    def band_grad(self, x, y, tau: float = 0.0, stream=None):
        import torch
        g = torch.empty(BAND_PARAMS, dtype=torch.float32, device=x.device)
        loss = ctypes.c_float()
        _check(self._lib.mj_band_grad(self._h, _ptr(x), _ptr(y), x.shape[0], tau, _stream(stream), _ptr(g),
                                      ctypes.byref(loss)), "mj_band_grad")
        return g, loss.value

    def band_calibrate(self, data, offsets, p: Params, stream=None) -> dict:
        """Times plain and learned joins on a held-out instance and keeps
        learned mode's network on only if it was faster (mj_band_calibrate)."""
        n = _check_inputs(data, offsets)
        r = BandCalibration()
        _check(self._lib.mj_band_calibrate(self._h, _ptr(data), _ptr(offsets), n, ctypes.byref(p), _stream(stream),
                                           ctypes.byref(r)), "mj_band_calibrate")
        return {f: getattr(r, f) for f, _ in BandCalibration._fields_}

    def band_weights(self) -> np.ndarray:
        w = np.empty(BAND_PARAMS, dtype=np.float32)
        _check(self._lib.mj_band_get_weights(self._h, w.ctypes.data, BAND_PARAMS), "mj_band_get_weights")
        return w

    def band_set_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(self._lib.mj_band_set_weights(self._h, w.ctypes.data, w.shape[0]), "mj_band_set_weights")

    def band_save(self, path: str):
        _check(self._lib.mj_band_save(self._h, path.encode()), "mj_band_save")

    def band_load(self, path: str):
        _check(self._lib.mj_band_load(self._h, path.encode()), "mj_band_load")

    def join_host(self, data: np.ndarray, offsets: np.ndarray, p: Params, stream=None, out=None):
        """Host buffers in, host arrays out (pinned buffers avoid staging copies)."""
        n = offsets.shape[0] - 1
        data = np.ascontiguousarray(data, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        cnt = U64()
        _check(self._lib.mj_join_host(self._h, data.ctypes.data if data.size else None, offsets.ctypes.data, n,
                                      ctypes.byref(p), _stream(stream), ctypes.byref(cnt)), "mj_join_host")
        m = cnt.value
        if out is None:
            out = tuple(np.empty(m, dtype=np.uint32) for _ in range(3))
        oi, oj, oe = (o[:m] for o in out)
        _check(self._lib.mj_result_copy_host(self._h, oi.ctypes.data if m else None, oj.ctypes.data if m else None,
                                             oe.ctypes.data if m else None, _stream(stream)), "mj_result_copy_host")
        return oi, oj, oe
