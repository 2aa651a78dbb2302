"""Pins of the oracle's surrogate MLP (3 -> 32 -> 32 -> 2, ReLU): hand-built
forward values, backpropagation against central finite differences, Adam's
first-step closed form."""
import numpy as np
import pytest

H = 32


def split(w):
    o = 0
    W1 = w[o:o + H * 3].reshape(H, 3); o += H * 3
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = w[o:o + 2]
    return W1, b1, W2, b2, W3, b3


def test_layout_size(orc):
    assert orc.MLP_NW == 1250


def test_forward_hand_built(orc):
    # hidden 1 = relu(u_q) and relu(-u_q); layer 2 identity; output = (u0 - u1, 2 u2 + 0.5)
    w = np.zeros(orc.MLP_NW)
    W1, b1, W2, b2, W3, b3 = split(w)
    for q in range(3):
        W1[q, q] = 1.0
        W1[3 + q, q] = -1.0
    W2[:, :] = np.eye(H)
    W3[0, 0], W3[0, 3], W3[0, 1], W3[0, 4] = 1.0, -1.0, -1.0, 1.0
    W3[1, 2], W3[1, 5] = 2.0, -2.0
    b3[1] = 0.5
    for u in ([0.3, -0.7, 1.1], [-2.0, 0.5, -0.25]):
        y = orc.mlp_forward(w, np.array(u))[0]
        assert y[0] == pytest.approx(u[0] - u[1], abs=1e-15)
        assert y[1] == pytest.approx(2 * u[2] + 0.5, abs=1e-15)


def test_backprop_matches_finite_differences(orc):
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.4, orc.MLP_NW)
    u = rng.normal(0, 1, (17, 3))
    t = rng.normal(0, 1, (17, 2))
    loss, g = orc.mlp_loss_grad(w, u, t)
    assert loss > 0
    eps = 1e-6
    for k in list(range(0, orc.MLP_NW, 7)) + [orc.MLP_NW - 1, orc.MLP_NW - 2]:
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (orc.mlp_loss_grad(wp, u, t)[0] - orc.mlp_loss_grad(wm, u, t)[0]) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=2e-6, abs=1e-9)


def test_loss_is_half_mean_square(orc):
    rng = np.random.default_rng(3)
    w = rng.normal(0, 0.3, orc.MLP_NW)
    u = rng.normal(0, 1, (5, 3))
    t = rng.normal(0, 1, (5, 2))
    y = orc.mlp_forward(w, u)
    assert orc.mlp_loss_grad(w, u, t)[0] == pytest.approx(0.5 * np.mean(np.sum((y - t) ** 2, 1)), rel=1e-14)


def test_adam_first_step_closed_form(orc):
    # first step from zero moments: w -= lr g / (|g| + eps)
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    m1, m2 = np.zeros(3), np.zeros(3)
    orc.adam_step(w, g, m1, m2, 1e-2, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(w, [1.0 - 1e-2 * 0.3 / (0.3 + 1e-8), -2.0 + 1e-2 * 1e-3 / (1e-3 + 1e-8), 0.5], rtol=1e-13)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(m2, 0.001 * g * g, rtol=1e-13)
