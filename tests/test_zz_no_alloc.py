"""mj_verify_static, the verification entry point that allocates nothing.

It serves callers that may not call cudaMalloc (a plug-in whose host
application owns all device memory, a latency-critical path that must avoid
allocation, a fixed device-memory budget): its scratch is a file-scope device
array of the library.  Here it is called through the C ABI and must give the
same distances as mj_verify, on two calls in a row with different inputs and
bands (the second call must not see anything left over from the first).
"""
import ctypes

import numpy as np
import pytest

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
    with mj.Context(0) as ctx:
        for seed, K in ((11, 40), (12, 100)):
            s, pairs = _pairs(seed, K, 400)
            data, off = to_device(s)
            i = torch.from_numpy(pairs[:, 0].astype(np.int32)).cuda()
            j = torch.from_numpy(pairs[:, 1].astype(np.int32)).cuda()
            ed = torch.full((pairs.shape[0],), -1, dtype=torch.int32, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            st = lib.mj_verify_static(data.data_ptr(), off.data_ptr(), s.n, i.data_ptr(), j.data_ptr(),
                                      pairs.shape[0], K, stream, ed.data_ptr())
            assert st == 0, lib.mj_strerror(st)
            want = ctx.verify(data, off, i, j, K)
            torch.cuda.synchronize()
            assert np.array_equal(ed.cpu().numpy(), want.cpu().numpy()), (seed, K)


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
