"""mj_verify_static, the verification entry point that allocates nothing.

It serves callers that may not call cudaMalloc (a plug-in whose host
application owns all device memory, a latency-critical path that must avoid
allocation, a fixed device-memory budget): its scratch is a file-scope device
array of the library.  Here it is called through the C ABI and must give the
same distances as mj_verify and as the oracle's banded DP, on two calls in a
row with different inputs and bands (the second call must not see anything
left over from the first), without changing the device's free memory; an
input beyond the array's size is rejected without writing the output, and an
out-of-range pair id is reported by mj_verify_static_flags.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _pairs(seed, K, count):
    rng = np.random.Generator(np.random.PCG64(seed))
    strs, pairs = [], []
    for t in range(count):
        L = int(rng.integers(0, 4 * K + 60))
        a = synth.DNA[rng.integers(0, 4, size=L)]
        b = synth.mutate(rng, a, float(rng.uniform(0.0, 2.5 * K / max(L, 1))), synth.DNA)
        strs += [a.tobytes(), b.tobytes()]
        pairs.append((2 * t, 2 * t + 1))
    strs.append(b"")
    pairs += [(2 * count, 0), (1, 1)]
    return synth.from_strings(strs, K=K, T=K), np.asarray(pairs, dtype=np.int64)


def test_static_verify_matches_mj_verify_on_two_calls():
    import torch
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build
    build.build()
    lib = mj.library()
    cases = []
    for seed, K in ((11, 40), (12, 100), (14, 255)):
        s, pairs = _pairs(seed, K, 400 if K < 255 else 120)
        data, off = to_device(s)
        i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
        j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
        ed = torch.full((pairs.shape[0],), -1, dtype=torch.int32, device="cuda")
        cases.append((s, pairs, K, data, off, i, j, ed))
    stream = torch.cuda.current_stream().cuda_stream
    with mj.Context(0) as ctx:
        wants = [ctx.verify(data, off, i, j, K) for (s, pairs, K, data, off, i, j, ed) in cases]
        torch.cuda.synchronize()
        # warm-up calls (the first call on a device looks up the array's
        # address, and the driver loads each band width's kernel on its first
        # launch), then the free device memory must not move
        for s, pairs, K, data, off, i, j, ed in cases:
            assert lib.mj_verify_static(data.data_ptr(), off.data_ptr(), s.n, i.data_ptr(), j.data_ptr(),
                                        pairs.shape[0], K, stream, ed.data_ptr()) == 0
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for (s, pairs, K, data, off, i, j, ed), want in zip(cases, wants):
            ed.fill_(-1)
            st = lib.mj_verify_static(data.data_ptr(), off.data_ptr(), s.n, i.data_ptr(), j.data_ptr(),
                                      pairs.shape[0], K, stream, ed.data_ptr())
            assert st == 0, lib.mj_strerror(st)
            torch.cuda.synchronize()
            got = ed.cpu().numpy()
            assert np.array_equal(got, want.cpu().numpy()), K
            assert np.array_equal(got.astype(np.int64), oracle.ed_band_pairs(s.bytes, s.offsets, pairs, K)), K
        assert torch.cuda.mem_get_info()[0] == free_before
        f = ctypes.c_uint32(99)
        assert lib.mj_verify_static_flags(stream, ctypes.byref(f)) == 0 and f.value == 0


def test_static_verify_reports_out_of_range_ids():
    import torch
    import paper_1810_08833_gb300 as mj
    lib = mj.library()
    s, pairs = _pairs(15, 20, 10)
    data, off = to_device(s)
    i = torch.tensor([0, s.n + 3], dtype=torch.int32, device="cuda")
    j = torch.tensor([1, 1], dtype=torch.int32, device="cuda")
    ed = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.mj_verify_static(data.data_ptr(), off.data_ptr(), s.n, i.data_ptr(), j.data_ptr(), 2, 20, stream,
                                ed.data_ptr()) == 0
    f = ctypes.c_uint32(0)
    assert lib.mj_verify_static_flags(stream, ctypes.byref(f)) == 0
    assert f.value & 1
    got = ed.cpu().tolist()
    assert got[1] == 21 and got[0] == oracle.ed_band(s.string(0), s.string(1), 20)


def test_static_verify_rejects_input_beyond_the_array():
    import torch
    import paper_1810_08833_gb300 as mj
    lib = mj.library()
    big = np.frombuffer(b"ACGT", np.uint8)[np.random.Generator(np.random.PCG64(3)).integers(0, 4, 17 << 20)]
    data = torch.from_numpy(big).cuda()
    off = torch.tensor([0, 1 << 20, big.shape[0]], dtype=torch.int64, device="cuda")
    i = torch.tensor([0], dtype=torch.int32, device="cuda")
    j = torch.tensor([1], dtype=torch.int32, device="cuda")
    ed = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = lib.mj_verify_static(data.data_ptr(), off.data_ptr(), 2, i.data_ptr(), j.data_ptr(), 1, 10,
                              torch.cuda.current_stream().cuda_stream, ed.data_ptr())
    assert st == -5                      # MJ_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert ed.cpu().tolist() == [-1]


def test_static_verify_rejects_out_of_range_band():
    import torch
    import paper_1810_08833_gb300 as mj
    lib = mj.library()
    s, pairs = _pairs(13, 10, 4)
    data, off = to_device(s)
    i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
    j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
    ed = torch.full((pairs.shape[0],), -1, dtype=torch.int32, device="cuda")
    st = lib.mj_verify_static(data.data_ptr(), off.data_ptr(), s.n, i.data_ptr(), j.data_ptr(), pairs.shape[0],
                              256, torch.cuda.current_stream().cuda_stream, ed.data_ptr())
    assert st == -5                      # MJ_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert (ed.cpu().numpy() == -1).all()
