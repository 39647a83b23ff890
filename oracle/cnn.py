"""Plain float64 reference of the small convolutional network that predicts MFWH warm starts
(oracle; test infrastructure only, never called by the library).

The network: L layers of 3 x 3 "same" convolutions (zero padding) with bias, ReLU after every
layer but the last, on images of shape [C, H, W].  Weights w[l] have shape [Cout, Cin, 3, 3]
and act as a cross-correlation:  out[co, y, x] = b[co] + sum_{ci, dy, dx} w[co, ci, dy, dx] *
in[ci, y + dy - 1, x + dx - 1].  Training minimises the mean squared error over a mask with
Adam (Kingma and Ba's update with bias correction).
"""

import numpy as np


def conv_same(x, w, b=None):
    """x: [B, Cin, H, W]; w: [Cout, Cin, 3, 3]; returns [B, Cout, H, W]."""
    B, Cin, H, W = x.shape
    Cout = w.shape[0]
    xp = np.zeros((B, Cin, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, Cout, H, W))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + W]               # in[ci, y + dy - 1, x + dx - 1]
            out += np.einsum("oc,bchw->bohw", w[:, :, dy, dx], patch)
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv_same_backward(x, w, gout):
    """Gradients of sum(gout * conv_same(x, w, b)) w.r.t. x, w and b."""
    B, Cin, H, W = x.shape
    xp = np.zeros((B, Cin, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + W]
            gw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gout, patch)
            gxp[:, :, dy:dy + H, dx:dx + W] += np.einsum("oc,bohw->bchw", w[:, :, dy, dx], gout)
    gb = gout.sum(axis=(0, 2, 3))
    return gxp[:, :, 1:-1, 1:-1], gw, gb


def forward(params, x):
    """params: list of (w, b).  Returns the output and the per-layer inputs (for backward)."""
    acts = [x]
    h = x
    for i, (w, b) in enumerate(params):
        h = conv_same(h, w, b)
        if i + 1 < len(params):
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def loss_and_grads(params, x, target, mask):
    """Mean squared error over the masked points and its gradients (list of (gw, gb))."""
    out, acts = forward(params, x)
    count = float(np.sum(mask)) * x.shape[0]
    diff = (out - target) * mask
    loss = float(np.sum(diff * diff) / count)
    g = 2.0 * diff / count
    grads = [None] * len(params)
    for i in reversed(range(len(params))):
        w, b = params[i]
        gx, gw, gb = conv_same_backward(acts[i], w, g)
        grads[i] = (gw, gb)
        if i > 0:
            g = gx * (acts[i] > 0.0)                          # ReLU of the previous layer
    return loss, grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of parameter array p (returns new p, m, v); t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
