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


# ------------------------------------------------------------ hand-worked pins

import importlib.util  # noqa: E402

import pytest  # noqa: E402

import mlp_pins  # noqa: E402

MLP_SRC = mlp.__file__


@pytest.mark.parametrize("name,fn", mlp_pins.ALL_MLP_PINS, ids=[n for n, _ in mlp_pins.ALL_MLP_PINS])
def test_mlp_pin(name, fn):
    fn(mlp)


def test_parameter_count_matches_header():
    assert mlp.NPARAM == mlp_pins.NPARAM == 4801


# Plausible mistakes planted in a copy of oracle/mlp.py; every occurrence of
# the text is replaced, so a mistake shared by the forward pass, the loss and
# the backpropagation (which the finite-difference tests cannot see) is what
# is planted.  The hand-worked pins must reject each one.
MLP_MUTANTS = [
    ("pinball_tau_swapped", "np.where(r > 0, tau * r, (tau - 1.0) * r)", "np.where(r > 0, (1.0 - tau) * r, -tau * r)"),
    ("pinball_grad_and_loss_swapped",
     "np.where(r > 0, -tau, 1.0 - tau)", "np.where(r > 0, tau - 1.0, tau)"),
    ("relu1_dropped", "h1 = np.maximum(X @ W1.T + b1, 0.0)", "h1 = X @ W1.T + b1"),
    ("relu2_dropped", "h2 = np.maximum(h1 @ W2.T + b2, 0.0)", "h2 = h1 @ W2.T + b2"),
    ("w2_transposed", "h1 @ W2.T + b2", "h1 @ W2 + b2"),
    ("w1_column_major", "w[o:o + H * F].reshape(H, F)", "w[o:o + H * F].reshape(F, H).T"),
    ("unpack_b1_before_w1", "W1 = w[o:o + H * F].reshape(H, F); o += H * F\n    b1 = w[o:o + H]; o += H",
     "b1 = w[o:o + H]; o += H\n    W1 = w[o:o + H * F].reshape(H, F); o += H * F"),
    ("unpack_w3_b2_swapped", "b2 = w[o:o + H]; o += H\n    W3 = w[o:o + H]; o += H",
     "W3 = w[o:o + H]; o += H\n    b2 = w[o:o + H]; o += H"),
    ("output_bias_dropped", "return h2 @ W3 + b3", "return h2 @ W3"),
    ("mse_halved", "np.mean(r * r)", "0.5 * np.mean(r * r)"),
]


def _load_mutant(tmp_path, name, old, new):
    src = open(MLP_SRC).read()
    assert old in src, f"mutation {name} does not apply"
    path = tmp_path / f"mlp_{name}.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"mlp_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", MLP_MUTANTS, ids=[m[0] for m in MLP_MUTANTS])
def test_mlp_pins_reject_mutant(tmp_path, name, old, new):
    mod = _load_mutant(tmp_path, name, old, new)
    failed = []
    for pin_name, fn in mlp_pins.ALL_MLP_PINS:
        try:
            fn(mod)
        except AssertionError:
            failed.append(pin_name)
    assert failed, f"no pin rejects the mutant {name}"
