"""CPU reference of the learned band's network (test infrastructure only).

The network is not part of the MinJoin paper: it predicts a candidate's edit
distance (as a fraction of K) to choose a narrower first verification band.
This module restates it plainly in float64 numpy so the GPU kernels' forward
pass and gradients can be checked: x (8) -> Linear(8, 64) -> ReLU ->
Linear(64, 64) -> ReLU -> Linear(64, 1).  Parameters are one flat vector in
the order W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.  Loss: mean
squared error (tau == 0) or the pinball loss at quantile tau.

Pinned by a hand-worked network (outputs, both losses and gradient entries
computed by hand, with the parameter layout checked one weight per block) and
by central finite differences of `loss`, which share nothing with the explicit
backpropagation below (tests/mlp_pins.py, tests/test_oracle_mlp.py).
"""
import numpy as np

F, H = 8, 64
NPARAM = H * F + H + H * H + H + H + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H * F].reshape(H, F); o += H * F
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def forward(w, X):
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3 + b3


def loss(w, X, y, tau=0.0):
    r = np.asarray(y, dtype=np.float64) - forward(w, X)
    if tau == 0.0:
        return float(np.mean(r * r))
    return float(np.mean(np.where(r > 0, tau * r, (tau - 1.0) * r)))


def grad(w, X, y, tau=0.0):
    """Loss and d loss / d w by the chain rule, layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = X.shape[0]
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    yhat = h2 @ W3 + b3
    r = y - yhat
    if tau == 0.0:
        L = np.mean(r * r)
        dy = -2.0 * r / m
    else:
        L = np.mean(np.where(r > 0, tau * r, (tau - 1.0) * r))
        dy = np.where(r > 0, -tau, 1.0 - tau) / m
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return float(L), g


def numeric_grad(w, X, y, idx, tau=0.0, eps=1e-6):
    """Central differences of `loss` at the parameters `idx`."""
    w = np.asarray(w, dtype=np.float64).copy()
    out = []
    for i in idx:
        old = w[i]
        w[i] = old + eps
        lp = loss(w, X, y, tau)
        w[i] = old - eps
        lm = loss(w, X, y, tau)
        w[i] = old
        out.append((lp - lm) / (2 * eps))
    return np.array(out)
