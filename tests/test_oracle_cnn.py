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
