"""Error paths without a GPU fault: a device allocation made to fail on the
host (mj_inject_alloc_failure) surfaces as MJ_ERR_OOM, the context stays
usable and gives the oracle's result on the next call, and destroying the
contexts returns the device's free memory to where it was."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu

OOM = -3


def _join_status(ctx, mj, data, off, p):
    """Status of mj_join (and the output on success)."""
    try:
        return 0, ctx.join(data, off, p)
    except mj.MinJoinError as e:
        return e.status, None


def _rows(out):
    return np.stack([t.cpu().numpy() for t in out], axis=1).astype(np.int64)


def test_injected_allocation_failures():
    import torch
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build
    build.build()
    lib = mj.library()
    s = synth.make_config(1, n_roots=20)
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
    want = np.concatenate([ref.pairs, ref.ed[:, None]], axis=1)
    data, off = to_device(s)
    with mj.Context(0) as warm:          # loads the kernels once
        warm.join(data, off, mj.params(s.K, T=s.T))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    statuses = []
    try:
        for nth in range(1, 41):
            for flags in (0, mj.MJ_FLAG_DEDUP_SORT):
                p = mj.params(s.K, T=s.T, flags=flags)
                with mj.Context(0) as ctx:
                    assert lib.mj_inject_alloc_failure(nth) == 0
                    st, out = _join_status(ctx, mj, data, off, p)
                    assert lib.mj_inject_alloc_failure(0) == 0
                    statuses.append(st)
                    assert st in (0, OOM), st
                    if st == 0:
                        assert np.array_equal(_rows(out), want)
                    # the same context, with allocations working again
                    assert np.array_equal(_rows(ctx.join(data, off, p)), want), (nth, flags)
                    assert ctx.stats()["device_flags"] == 0
    finally:
        lib.mj_inject_alloc_failure(0)
    assert OOM in statuses and 0 in statuses   # both failing and untouched joins were seen
    torch.cuda.synchronize()
    leaked = free0 - torch.cuda.mem_get_info()[0]
    assert leaked <= (2 << 20), leaked


def test_injected_failure_in_verify_and_candidates():
    import torch
    import paper_1810_08833_gb300 as mj
    lib = mj.library()
    s = synth.make_config(4, n_roots=50)
    parts = oracle.partition(s.bytes, s.offsets, oracle.derive_params(s.bytes, s.offsets, K=s.K, T=s.T))
    want_c = oracle.candidates(s.bytes, s.offsets, s.K, parts)
    data, off = to_device(s)
    seen_oom = False
    try:
        for nth in range(1, 16):
            with mj.Context(0) as ctx:
                lib.mj_inject_alloc_failure(nth)
                try:
                    ctx.candidates(data, off, mj.params(s.K, T=s.T))
                except mj.MinJoinError as e:
                    assert e.status == OOM
                    seen_oom = True
                lib.mj_inject_alloc_failure(0)
                ci, cj = ctx.candidates(data, off, mj.params(s.K, T=s.T))
                got = np.stack([ci.cpu().numpy(), cj.cpu().numpy()], 1).astype(np.int64)
                assert np.array_equal(got, want_c)
                lib.mj_inject_alloc_failure(1)
                try:
                    ctx.verify(data, off, ci, cj, s.K)
                    torch.cuda.synchronize()
                except mj.MinJoinError as e:
                    assert e.status == OOM
                lib.mj_inject_alloc_failure(0)
                ed = ctx.verify(data, off, ci, cj, s.K).cpu().numpy().astype(np.int64)
                assert np.array_equal(ed, oracle.ed_band_pairs(s.bytes, s.offsets, want_c, s.K))
    finally:
        lib.mj_inject_alloc_failure(0)
    assert seen_oom
