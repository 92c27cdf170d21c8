"""The CPU reference of the band network: backpropagation pinned by central
finite differences (no GPU)."""
import numpy as np

from oracle import mlp


def _data(seed, m=96):
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.normal(0, 0.4, size=mlp.NPARAM)
    X = rng.uniform(0, 1, size=(m, mlp.F))
    y = rng.uniform(0, 1.2, size=m)
    return w, X, y


def test_backprop_matches_finite_differences_mse():
    w, X, y = _data(1)
    L, g = mlp.grad(w, X, y)
    assert abs(L - mlp.loss(w, X, y)) < 1e-12
    rng = np.random.Generator(np.random.PCG64(2))
    idx = np.concatenate([rng.choice(mlp.NPARAM, 300, replace=False), [mlp.NPARAM - 1, 0, 512, 4800 - 64]])
    num = mlp.numeric_grad(w, X, y, idx)
    assert np.allclose(g[idx], num, rtol=1e-5, atol=1e-8)


def test_backprop_matches_finite_differences_pinball():
    w, X, y = _data(3)
    L, g = mlp.grad(w, X, y, tau=0.9)
    rng = np.random.Generator(np.random.PCG64(4))
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    num = mlp.numeric_grad(w, X, y, idx, tau=0.9, eps=1e-7)
    assert np.allclose(g[idx], num, rtol=1e-4, atol=1e-7)


def test_planted_backprop_mistake_is_caught():
    # a gradient that drops the ReLU mask of the second layer disagrees with
    # the finite differences
    w, X, y = _data(5)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    dy = -2.0 * (y - (h2 @ W3 + b3)) / X.shape[0]
    wrong_gW2 = (np.outer(dy, W3)).T @ h1          # mask (z2 > 0) dropped
    idx = np.arange(576, 576 + 4096)
    num = mlp.numeric_grad(w, X, y, idx[:256])
    assert not np.allclose(wrong_gW2.ravel()[:256], num, rtol=1e-5, atol=1e-8)
