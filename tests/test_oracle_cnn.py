"""Pins for the float64 reference network of the warm-start predictor: the convolution
against scipy's correlate, its backward pass against finite differences, the whole network's
gradients against finite differences, and one Adam step against the update written out."""

import numpy as np
import pytest

from oracle import cnn

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv_same_is_cross_correlation():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = cnn.conv_same(x, w, b)
    for bb in range(2):
        for co in range(4):
            want = b[co] + sum(scipy_signal.correlate(x[bb, ci], w[co, ci], mode="same")
                               for ci in range(3))
            np.testing.assert_allclose(got[bb, co], want, atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 2, 5, 6))
    w = rng.normal(size=(3, 2, 3, 3))
    gout = rng.normal(size=(1, 3, 5, 6))
    gx, gw, gb = cnn.conv_same_backward(x, w, gout)
    f = lambda xx, ww, bb: float(np.sum(gout * cnn.conv_same(xx, ww, bb)))
    b = np.zeros(3)
    eps = 1e-6
    for idx in [(0, 1, 0, 0), (0, 0, 2, 3), (0, 1, 4, 5)]:
        d = np.zeros_like(x); d[idx] = eps
        np.testing.assert_allclose((f(x + d, w, b) - f(x - d, w, b)) / (2 * eps), gx[idx], rtol=1e-6)
    for idx in [(0, 0, 0, 0), (2, 1, 1, 2), (1, 0, 2, 1)]:
        d = np.zeros_like(w); d[idx] = eps
        np.testing.assert_allclose((f(x, w + d, b) - f(x, w - d, b)) / (2 * eps), gw[idx], rtol=1e-6)
    np.testing.assert_allclose(gb, gout.sum(axis=(0, 2, 3)))


def test_network_gradients_finite_differences():
    rng = np.random.default_rng(3)
    chans = [2, 4, 4, 1]
    params = [(rng.normal(size=(co, ci, 3, 3)) * 0.4, rng.normal(size=co) * 0.1)
              for ci, co in zip(chans[:-1], chans[1:])]
    x = rng.normal(size=(2, 2, 6, 5))
    t = rng.normal(size=(2, 1, 6, 5))
    mask = np.ones((6, 5)); mask[0, :] = mask[-1, :] = 0.0
    loss, grads = cnn.loss_and_grads(params, x, t, mask)
    eps = 1e-6
    for li, idx in [(0, (1, 0, 1, 1)), (1, (2, 3, 0, 2)), (2, (0, 1, 2, 2))]:
        def L(delta):
            p2 = [(w.copy(), b.copy()) for w, b in params]
            p2[li][0][idx] += delta
            return cnn.loss_and_grads(p2, x, t, mask)[0]
        np.testing.assert_allclose((L(eps) - L(-eps)) / (2 * eps), grads[li][0][idx], rtol=1e-5)
    # bias of the first layer
    def Lb(delta):
        p2 = [(w.copy(), b.copy()) for w, b in params]
        p2[0][1][1] += delta
        return cnn.loss_and_grads(p2, x, t, mask)[0]
    np.testing.assert_allclose((Lb(eps) - Lb(-eps)) / (2 * eps), grads[0][1][1], rtol=1e-5)


def test_adam_step_written_out():
    p = np.array([1.0, -2.0]); g = np.array([0.5, -0.25])
    m = np.zeros(2); v = np.zeros(2)
    p1, m1, v1 = cnn.adam_step(p, g, m, v, 1, 0.01)
    # first step: mhat = g, vhat = g^2, so the move is lr * g / (|g| + eps) = lr * sign(g)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8))
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2 at every
    step (m_t = (1 - beta1^t) g, v_t = (1 - beta2^t) g^2), so step t moves p by
    lr g / (|g| + eps).  A bias correction without its power t (1 - beta instead of
    1 - beta^t) moves 1.34 lr at t = 2 and fails here."""
    g = np.array([0.5, -0.25, 3.0])
    p = np.array([1.0, -2.0, 0.5])
    m = np.zeros(3)
    v = np.zeros(3)
    lr = 0.01
    for t in range(1, 6):
        p_new, m, v = cnn.adam_step(p, g, m, v, t, lr)
        np.testing.assert_allclose(p - p_new, lr * g / (np.abs(g) + 1e-8), rtol=1e-12)
        p = p_new


def test_adam_three_steps_worked_example():
    """Three steps with gradients 1/2, -3/10, 1/5 from p = 1, lr = 0.01, computed by hand
    in exact fractions: m = 1/20, 3/200, 67/2000; v = 1/4000, 1359/4000000,
    1517641/4000000000; bias-corrected at t = 2: m^ = (3/200)/(19/100) = 3/38,
    v^ = (1359/4000000)/(1999/1000000) = 1359/7996."""
    p = np.array([1.0])
    m = np.zeros(1)
    v = np.zeros(1)
    want_m = [0.05, 0.015, 0.0335]
    want_v = [0.00025, 0.00033975, 0.00037941025]
    want_p = [1.0 - 0.01 * 0.5 / (0.5 + 1e-8),
              1.0 - 0.01 * 0.5 / (0.5 + 1e-8) - 0.01 * (3.0 / 38.0) / ((1359.0 / 7996.0) ** 0.5 + 1e-8),
              0.9846107430790882]
    for t, g in enumerate([0.5, -0.3, 0.2], start=1):
        p, m, v = cnn.adam_step(p, np.array([g]), m, v, t, 0.01)
        np.testing.assert_allclose(m, want_m[t - 1], rtol=1e-14)
        np.testing.assert_allclose(v, want_v[t - 1], rtol=1e-14)
        np.testing.assert_allclose(p, want_p[t - 1], rtol=1e-14)
