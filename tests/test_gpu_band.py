"""The learned first-pass band on the GPU: the network's forward pass and
gradients against the CPU reference, the candidate features, training, and
the learned join's output (identical to the plain join) with its gain."""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1810_08833_gb300 as mj
    from paper_1810_08833_gb300 import build
    build.build()
    c = mj.Context(0)
    yield c
    c.close()


def _random_net(seed, m=512):
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.normal(0, 0.3, size=mlp.NPARAM).astype(np.float32)
    X = rng.uniform(0, 1, size=(m, mlp.F)).astype(np.float32)
    y = rng.uniform(0, 1.1, size=m).astype(np.float32)
    return w, X, y


def test_forward_matches_cpu_reference(ctx):
    import torch
    w, X, _ = _random_net(1)
    ctx.band_set_weights(w)
    got = ctx.band_forward(torch.from_numpy(X).cuda()).cpu().numpy()
    want = mlp.forward(w.astype(np.float64), X.astype(np.float64))
    assert np.allclose(got, want, rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("tau", [0.0, 0.9])
def test_gradient_matches_cpu_reference(ctx, tau):
    import torch
    w, X, y = _random_net(2)
    ctx.band_set_weights(w)
    g, loss = ctx.band_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), tau=tau)
    g = g.cpu().numpy().astype(np.float64)
    L, want = mlp.grad(w.astype(np.float64), X.astype(np.float64), y.astype(np.float64), tau=tau)
    assert abs(loss - L) <= 1e-3 * max(1.0, abs(L))
    rel = np.linalg.norm(g - want) / np.linalg.norm(want)
    assert rel < 1e-3, rel
    big = np.abs(want) > 1e-3 * np.abs(want).max()
    assert np.allclose(g[big], want[big], rtol=1e-3, atol=1e-6)


def test_training_lowers_the_loss(ctx):
    import torch
    rng = np.random.Generator(np.random.PCG64(3))
    X = rng.uniform(0, 1, size=(4096, mlp.F)).astype(np.float32)
    ed = np.clip(np.rint(40 * (0.2 + 0.6 * X[:, 1] + 0.2 * X[:, 5] * X[:, 2])), 0, 41).astype(np.int32)
    x_t = torch.from_numpy(X).cuda()
    ed_t = torch.from_numpy(ed).cuda()
    ctx.band_init(seed=7)
    y = torch.from_numpy(np.minimum(ed, 41).astype(np.float32) / 40.0).cuda()
    _, before = ctx.band_grad(x_t, y, tau=0.0)
    ctx.band_train(x_t, ed_t, K=40, steps=1500, batch=512, lr=3e-3, tau=0.0, seed=11)
    _, after = ctx.band_grad(x_t, y, tau=0.0)
    assert after < 0.2 * before, (before, after)


def _multiplicities(s, K, parts):
    """Matched partition pairs behind every candidate: identical partition
    substrings in two different strings passing both filters of Alg. 3."""
    L = s.lengths()
    groups = {}
    for sid, pos, ln in zip(parts.sid.tolist(), parts.pos.tolist(), parts.len.tolist()):
        groups.setdefault(s.string(sid)[pos:pos + ln], []).append((sid, pos))
    count = {}
    for members in groups.values():
        for x in range(len(members)):
            for y in range(x + 1, len(members)):
                (i, pi), (j, pj) = members[x], members[y]
                if i == j or abs(L[i] - L[j]) > K:
                    continue
                if abs(pi - pj) + abs((L[i] - pi) - (L[j] - pj)) <= K:
                    key = (min(i, j), max(i, j))
                    count[key] = count.get(key, 0) + 1
    return count


def test_features_match_their_definition(ctx):
    import paper_1810_08833_gb300 as mj
    s = synth.random_set(41, n=250, min_len=60, max_len=400, K=8, T=8, families=15, rate=0.02)
    p = oracle.derive_params(s.bytes, s.offsets, K=8, T=8)
    parts = oracle.partition(s.bytes, s.offsets, p)
    data, off = to_device(s)
    ctx.join(data, off, mj.params(8, T=8, flags=mj.MJ_FLAG_FEATURES))
    x, ed, ci, cj = ctx.features()
    x, ed, ci, cj = (t.cpu().numpy() for t in (x, ed, ci, cj))
    mult = _multiplicities(s, 8, parts)
    L = s.lengths()
    npart = np.bincount(parts.sid, minlength=s.n)
    assert len(mult) == ci.shape[0]
    for u in range(ci.shape[0]):
        i, j = int(ci[u]), int(cj[u])
        c = mult[(i, j)]
        n = min(L[i], L[j])
        want = [np.log2(1 + n) / 16, abs(L[i] - L[j]) / 8, c / 9, npart[i] / 9, npart[j] / 9,
                c / max(1, min(npart[i], npart[j])), np.log2(1 + c) / 8, 8 / 108]
        assert np.allclose(x[u], want, rtol=1e-5, atol=1e-6), (u, x[u], want)
    want_ed = oracle.ed_band_pairs(s.bytes, s.offsets, np.stack([ci, cj], 1).astype(np.int64), 8)
    assert np.array_equal(ed.astype(np.int64), want_ed)


def test_save_load_roundtrip(ctx, tmp_path):
    w, _, _ = _random_net(4)
    ctx.band_set_weights(w)
    path = str(tmp_path / "band.bin")
    ctx.band_save(path)
    ctx.band_init(seed=99)
    ctx.band_load(path)
    assert np.array_equal(ctx.band_weights(), w)


def train_band(ctx, cfg, roots, seed, steps=1500):
    """Train the band network on a held-out instance of a workload."""
    import paper_1810_08833_gb300 as mj
    s = synth.make_config(cfg, seed=seed, n_roots=roots)
    data, off = to_device(s)
    ctx.join(data, off, mj.params(s.K, T=s.T, flags=mj.MJ_FLAG_FEATURES))
    x, ed, _, _ = ctx.features()
    ctx.band_init(seed=5)
    ctx.band_train(x, ed, K=s.K, steps=steps, batch=1024, lr=2e-3, tau=0.9, seed=13)
    return x.shape[0]


@pytest.mark.parametrize("cfg,roots", [(4, 400), (5, 150), (2, 30)])
def test_learned_join_equals_plain_and_gains(ctx, cfg, roots):
    """Same output as the plain K band on every pair; the first pass settles
    pairs with fewer band words, so the verifier advances fewer words."""
    import paper_1810_08833_gb300 as mj
    train_band(ctx, cfg, roots, seed=100 + cfg)
    s = synth.make_config(cfg, n_roots=roots)
    data, off = to_device(s)
    pi, pj, pe = ctx.join(data, off, mj.params(s.K, T=s.T))
    plain = ctx.stats()
    li, lj, le = ctx.join(data, off, mj.params(s.K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED,
                                                flags=mj.MJ_FLAG_FIRST_PASS))
    learned = ctx.stats()
    for a, b in ((pi, li), (pj, lj), (pe, le)):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    ref = oracle.minjoin(s.bytes, s.offsets, K=s.K, T=s.T)
    assert np.array_equal(np.stack([li.cpu().numpy(), lj.cpu().numpy()], 1).astype(np.int64), ref.pairs)
    if cfg != 2:   # K = 100: pairs within K are rare in this workload
        assert learned["first_pass_settled"] > 0
        assert learned["verify_word_columns"] < plain["verify_word_columns"], (learned, plain)


def test_calibration_gates_learned_mode(ctx):
    """mj_band_calibrate times both modes on a held-out instance and keeps the
    network only if learned mode was faster; either way the learned join
    returns the plain output, and forcing the first passes still runs them."""
    import paper_1810_08833_gb300 as mj
    train_band(ctx, 4, 300, seed=104, steps=500)
    cal_set = synth.make_config(4, seed=204, n_roots=300)
    cd, co = to_device(cal_set)
    rep = ctx.band_calibrate(cd, co, mj.params(cal_set.K, T=cal_set.T))
    assert rep["enabled"] == (1 if rep["learned_ms"] < rep["plain_ms"] else 0)
    assert rep["plain_ms"] > 0 and rep["learned_ms"] > 0
    assert rep["learned_word_columns"] <= rep["plain_word_columns"] + rep["plain_word_columns"] // 2
    s = synth.make_config(4, n_roots=300)
    data, off = to_device(s)
    want = [t.cpu().numpy() for t in ctx.join(data, off, mj.params(s.K, T=s.T))]
    got = [t.cpu().numpy() for t in ctx.join(data, off, mj.params(s.K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED))]
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    if not rep["enabled"]:
        assert ctx.stats()["first_pass_settled"] == 0   # the plain path ran
    forced = [t.cpu().numpy() for t in ctx.join(data, off, mj.params(s.K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED,
                                                                      flags=mj.MJ_FLAG_FIRST_PASS))]
    assert ctx.stats()["first_pass_settled"] > 0
    for a, b in zip(want, forced):
        assert np.array_equal(a, b)
    # a new model clears the calibration: the network runs again
    ctx.band_set_weights(ctx.band_weights())
    ctx.join(data, off, mj.params(s.K, T=s.T, verify_mode=mj.MJ_VERIFY_LEARNED, flags=mj.MJ_FLAG_FIRST_PASS))
    assert ctx.stats()["first_pass_settled"] > 0
