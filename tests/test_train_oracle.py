"""Pins of the training oracle (oracle/train.py), no GPU.

The backpropagated gradients are checked against central finite differences
of the loss in FP64 on entries of every gate block of W_x and U, of W_fc and
of h_0; the unrolled forward against the single-step cell that the golden
fixture pins; the loss and Adam against closed forms.
"""

import numpy as np
import pytest

from oracle import gru, train


def problem(T=4, P=5, n_in=7, H=6, n_out=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (T, P, n_in))
    h0 = rng.uniform(-0.5, 0.5, (P, H))
    Y = rng.normal(0, 0.3, (T, P, n_out))
    Wx = rng.normal(0, 0.4, (3 * H, n_in))
    Uh = rng.normal(0, 0.4, (3 * H, H))
    Wfc = rng.normal(0, 0.4, (n_out, H))
    return X, h0, Y, Wx, Uh, Wfc


def test_unrolled_forward_equals_repeated_cell():
    X, h0, Y, Wx, Uh, Wfc = problem()
    D, cache = train.seq_forward(X, h0, Wx, Uh, Wfc)
    h = h0
    for t in range(X.shape[0]):
        h, d = gru.gru_step(X[t], h, Wx, Uh, Wfc)
        assert np.array_equal(d, D[t])
        assert np.array_equal(h, cache["hs"][t + 1])


def test_loss_closed_form():
    X, h0, Y, Wx, Uh, Wfc = problem(T=2, P=4)
    D = Y + 0.5                               # every entry off by 1/2
    n_out = Y.shape[2]
    assert train.loss(D, Y, Wx, Uh, Wfc, alpha=0.0) == pytest.approx(2 * n_out * 0.25)
    reg = 1e-4 * (np.sum(Wx ** 2) + np.sum(Uh ** 2) + np.sum(Wfc ** 2))
    assert train.loss(Y, Y, Wx, Uh, Wfc) == pytest.approx(reg)


@pytest.mark.parametrize("alpha", [0.0, 1e-4])
def test_bptt_gradient_matches_finite_differences(alpha):
    X, h0, Y, Wx, Uh, Wfc = problem()
    H = Uh.shape[1]
    L, gWx, gUh, gWfc, gh0 = train.loss_and_grads(X, h0, Y, Wx, Uh, Wfc, alpha)

    def f(Wx_, Uh_, Wfc_, h0_):
        D, _ = train.seq_forward(X, h0_, Wx_, Uh_, Wfc_)
        return train.loss(D, Y, Wx_, Uh_, Wfc_, alpha)

    eps = 1e-6
    rng = np.random.default_rng(1)
    checks = []
    # entries of each gate block (z, r, h) of W_x and U, of W_fc, and of h_0
    for which, shape in (("Wx", Wx.shape), ("Uh", Uh.shape), ("Wfc", Wfc.shape), ("h0", h0.shape)):
        blocks = [(0, H), (H, 2 * H), (2 * H, 3 * H)] if which in ("Wx", "Uh") else [(0, shape[0])]
        for lo, hi in blocks:
            for _ in range(3):
                checks.append((which, (int(rng.integers(lo, hi)), int(rng.integers(0, shape[1])))))
    grads = {"Wx": gWx, "Uh": gUh, "Wfc": gWfc, "h0": gh0}
    for which, idx in checks:
        args = {"Wx": Wx.copy(), "Uh": Uh.copy(), "Wfc": Wfc.copy(), "h0": h0.copy()}
        args[which][idx] += eps
        fp = f(args["Wx"], args["Uh"], args["Wfc"], args["h0"])
        args[which][idx] -= 2 * eps
        fm = f(args["Wx"], args["Uh"], args["Wfc"], args["h0"])
        fd = (fp - fm) / (2 * eps)
        g = grads[which][idx]
        assert abs(fd - g) <= 1e-7 * max(1.0, abs(fd)), (which, idx, fd, g)


def test_gradient_of_a_single_step_by_hand():
    # T = 1, H = 1, n_in = 1, n_out = 1, h0 = 0: h = (1 - z) c with
    # z = sigma(a x), c = tanh(b x), d = w h; dL/dw = 2 (d - y) h (P = 1)
    a, b, w, x, y = 0.3, -0.7, 1.9, 0.8, 0.25
    Wx = np.array([[a], [0.0], [b]])
    Uh = np.zeros((3, 1))
    Wfc = np.array([[w]])
    z = 1 / (1 + np.exp(-a * x))
    c = np.tanh(b * x)
    h = (1 - z) * c
    L, gWx, gUh, gWfc, gh0 = train.loss_and_grads(np.array([[[x]]]), np.zeros((1, 1)), np.array([[[y]]]),
                                                   Wx, Uh, Wfc, alpha=0.0)
    e = 2 * (w * h - y)
    assert L == pytest.approx((w * h - y) ** 2, rel=1e-14)
    assert gWfc[0, 0] == pytest.approx(e * h, rel=1e-14)
    assert gWx[0, 0] == pytest.approx(e * w * (-c) * z * (1 - z) * x, rel=1e-14)   # through z
    assert gWx[2, 0] == pytest.approx(e * w * (1 - z) * (1 - c * c) * x, rel=1e-14)  # through c
    assert gWx[1, 0] == 0.0                      # r multiplies h0 = 0
    assert np.all(gUh == 0.0)                    # every U term multiplies h0 = 0


def test_adam_closed_forms():
    rng = np.random.default_rng(2)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    m, v = np.zeros(50), np.zeros(50)
    lr, eps = 1e-2, 1e-8
    # with bias correction the first step is lr g / (|g| + eps): a signed step of lr
    p1, m, v = train.adam_step(p, g, m, v, 1, lr=lr, eps=eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # a constant gradient keeps m_hat = g and v_hat = g^2: the same step again
    p2, m, v = train.adam_step(p1, g, m, v, 2, lr=lr, eps=eps)
    assert np.allclose(p2 - p1, p1 - p, rtol=0, atol=1e-14)
