"""Pins of the band network's CPU reference (oracle/mlp.py) by hand-worked
values: a network with a few non-zero weights placed by the parameter layout
that include/minjoin.h states (W1[64][8], b1[64], W2[64][64], b2[64], W3[64],
b3, each matrix row-major with the output unit first), whose outputs, losses
and a few gradients were computed by hand.  Each pin takes the module under
test, so tests/test_oracle_mlp.py can run them on deliberately broken copies
of oracle/mlp.py as well as on the shipped one.
"""
from __future__ import annotations

import numpy as np

F, H = 8, 64
NPARAM = H * F + H + H * H + H + H + 1     # 4801, as stated in the header


def idx_w1(h, f):
    return h * F + f


def idx_b1(h):
    return H * F + h


def idx_w2(o, i):
    return H * F + H + o * H + i


def idx_b2(h):
    return H * F + H + H * H + h


def idx_w3(h):
    return H * F + H + H * H + H + h


IDX_B3 = NPARAM - 1


def hand_net() -> np.ndarray:
    """The hand-worked network: every weight not set here is zero."""
    w = np.zeros(NPARAM)
    w[idx_w1(0, 0)] = 1.0
    w[idx_w1(1, 1)] = -2.0
    w[idx_w1(5, 7)] = 0.5
    w[idx_b1(0)] = -0.5
    w[idx_b1(1)] = 1.0
    w[idx_w2(0, 0)] = 2.0
    w[idx_w2(2, 0)] = -1.0
    w[idx_w2(3, 1)] = 1.5
    w[idx_w2(4, 5)] = 4.0
    w[idx_b2(2)] = 0.25
    w[idx_w3(0)] = 1.0
    w[idx_w3(2)] = 10.0
    w[idx_w3(3)] = -1.0
    w[idx_w3(4)] = 0.5
    w[IDX_B3] = 0.125
    return w


# x1 = (1.5, 0.25, 0, 0, 0, 0, 0, 2):
#   first layer  z1[0] = 1.5 - 0.5 = 1, z1[1] = -2 * 0.25 + 1 = 0.5, z1[5] = 0.5 * 2 = 1
#   second layer z2[0] = 2 * 1 = 2, z2[2] = -1 * 1 + 0.25 = -0.75 -> ReLU 0,
#                z2[3] = 1.5 * 0.5 = 0.75, z2[4] = 4 * 1 = 4
#   output       1 * 2 + 10 * 0 - 1 * 0.75 + 0.5 * 4 + 0.125 = 3.375
# x2 = (0.25, 1, 0, 0, 0, 0, 0, -4):
#   first layer  z1[0] = -0.25, z1[1] = -1, z1[5] = -2: all cut by the ReLU
#   second layer only z2[2] = 0.25 survives (its bias)
#   output       10 * 0.25 + 0.125 = 2.625
X_HAND = np.array([[1.5, 0.25, 0, 0, 0, 0, 0, 2.0],
                   [0.25, 1.0, 0, 0, 0, 0, 0, -4.0]])
Y_HAND = np.array([3.375, 2.625])


def pin_forward_hand(m):
    got = np.asarray(m.forward(hand_net(), X_HAND), dtype=np.float64)
    assert got.shape == (2,), got.shape
    assert np.allclose(got, Y_HAND, rtol=0, atol=1e-12), got


def pin_layout_one_weight_per_block(m):
    """One non-zero parameter per block, each read back through the output:
    with x = e_3, W1[7][3] = 2 and W2[9][7] = 3 route 2 * 3 = 6 to hidden unit
    9 of the second layer, and W3[9] = 0.5 gives 3; the biases b1[7], b2[9]
    and b3 each shift the output by a known amount."""
    w = np.zeros(NPARAM)
    w[idx_w1(7, 3)] = 2.0
    w[idx_w2(9, 7)] = 3.0
    w[idx_w3(9)] = 0.5
    x = np.zeros((1, F))
    x[0, 3] = 1.0
    assert np.allclose(m.forward(w, x), [3.0], atol=1e-12)
    w[idx_b1(7)] = 1.0          # z1[7] = 3 -> 9 at unit 9 -> 4.5
    assert np.allclose(m.forward(w, x), [4.5], atol=1e-12)
    w[idx_b2(9)] = -1.0         # z2[9] = 8 -> 4
    assert np.allclose(m.forward(w, x), [4.0], atol=1e-12)
    w[IDX_B3] = -0.75
    assert np.allclose(m.forward(w, x), [3.25], atol=1e-12)
    # the same weights one slot off do nothing for this input
    v = np.zeros(NPARAM)
    v[idx_w1(7, 4)] = 2.0
    v[idx_w2(9, 7)] = 3.0
    v[idx_w3(9)] = 0.5
    assert np.allclose(m.forward(v, x), [0.0], atol=1e-12)


def pin_loss_hand(m):
    """Residuals y - yhat of +0.5 and -1 on the two hand inputs: mean squared
    error (0.25 + 1) / 2 = 0.625; pinball loss at tau = 0.9: a positive
    residual costs tau * r = 0.45, a negative one (tau - 1) * r = 0.1, mean
    0.275.  At residuals exactly +1 and -1 the pinball loss is tau and
    1 - tau."""
    w = hand_net()
    y = Y_HAND + np.array([0.5, -1.0])
    assert abs(m.loss(w, X_HAND, y) - 0.625) < 1e-12
    assert abs(m.loss(w, X_HAND, y, tau=0.9) - 0.275) < 1e-12
    assert abs(m.loss(w, X_HAND[:1], Y_HAND[:1] + 1.0, tau=0.9) - 0.9) < 1e-12
    assert abs(m.loss(w, X_HAND[:1], Y_HAND[:1] - 1.0, tau=0.9) - 0.1) < 1e-12
    assert abs(m.loss(w, X_HAND[1:], Y_HAND[1:] + 1.0, tau=0.25) - 0.25) < 1e-12
    assert abs(m.loss(w, X_HAND[1:], Y_HAND[1:] - 1.0, tau=0.25) - 0.75) < 1e-12


def pin_grad_hand(m):
    """Hand-worked gradients at the hand network with residuals +0.5 and -1.
    MSE: d/dyhat = -2 r / 2 = (-0.5, +1) per sample, so
      d/db3 = 0.5, d/dW3[0] = -0.5 * 2 + 1 * 0 = -1, d/dW3[2] = 1 * 0.25 = 0.25,
      d/dW3[4] = -0.5 * 4 = -2,
      d/db2[0] = -0.5 * W3[0] = -0.5 (unit 0 is active on x1 only),
      d/dW2[0][0] = -0.5 * 1 * h1[0] = -0.5,
      d/dW1[0][0] = -0.5 * W3[0] * W2[0][0] * x1[0] = -1.5  (unit 2 of layer 2
      is cut on x1, so W2[2][0] adds nothing there), d/db1[0] = -1.
    Pinball at tau = 0.9: d/dyhat = (-tau, 1 - tau) / 2 = (-0.45, 0.05):
      d/db3 = -0.4, d/dW3[2] = 0.05 * 0.25 = 0.0125, d/db2[2] = 0.05 * 10 = 0.5."""
    w = hand_net()
    y = Y_HAND + np.array([0.5, -1.0])
    L, g = m.grad(w, X_HAND, y)
    assert abs(L - 0.625) < 1e-12
    want = {IDX_B3: 0.5, idx_w3(0): -1.0, idx_w3(2): 0.25, idx_w3(4): -2.0, idx_b2(0): -0.5,
            idx_w2(0, 0): -0.5, idx_w1(0, 0): -1.5, idx_b1(0): -1.0}
    for k, v in want.items():
        assert abs(g[k] - v) < 1e-12, (k, g[k], v)
    L, g = m.grad(w, X_HAND, y, tau=0.9)
    assert abs(L - 0.275) < 1e-12
    for k, v in {IDX_B3: -0.4, idx_w3(2): 0.0125, idx_b2(2): 0.5}.items():
        assert abs(g[k] - v) < 1e-12, (k, g[k], v)


ALL_MLP_PINS = [
    ("forward_hand", pin_forward_hand),
    ("layout_one_weight_per_block", pin_layout_one_weight_per_block),
    ("loss_hand", pin_loss_hand),
    ("grad_hand", pin_grad_hand),
]
