"""GPU parity of the warm-start network (BF16 tensor-core convolutions, FP32 accumulation
and Adam) against the float64 reference network in oracle/cnn.py.  The reference runs on
the same BF16-rounded weights and inputs; the GPU also rounds each layer's activations to
BF16, so agreement is to BF16 precision: 2e-2 relative (max norm) for outputs, 5e-2 for
gradients (Frobenius, per layer)."""

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build
from oracle import cnn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load()


def bf16(a):
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(flat, chans):
    params, o = [], 0
    for ci, co in zip(chans[:-1], chans[1:]):
        w = flat[o:o + co * ci * 9].reshape(co, ci, 3, 3); o += co * ci * 9
        b = flat[o:o + co]; o += co
        params.append((w.astype(np.float64), b.astype(np.float64)))
    return params


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("layers,channels,H,W", [(3, 8, 20, 21), (5, 32, 17, 40)])
def test_cnn_forward_and_gradients(layers, channels, H, W):
    chans = [2] + [channels] * (layers - 1) + [1]
    net = M.CNN(layers=layers, channels=channels, in_channels=2, seed=3)
    rng = np.random.default_rng(5)
    flat = np.concatenate([np.concatenate([rng.normal(size=co * ci * 9) * np.sqrt(2 / (9 * ci)),
                                           rng.normal(size=co) * 0.05])
                           for ci, co in zip(chans[:-1], chans[1:])]).astype(np.float32)
    assert flat.size == net.n_params
    net.set_params(flat)
    B = 2
    x = rng.normal(size=(B, 2, H, W)).astype(np.float32)
    t = rng.normal(size=(B, 1, H, W)).astype(np.float32)
    mask = np.ones((H, W), dtype=np.float32); mask[0, :] = mask[-1, :] = 0; mask[:, 0] = mask[:, -1] = 0
    params = [(bf16(w), b) for w, b in unflatten(flat, chans)]
    want, _ = cnn.forward(params, bf16(x))
    y = torch.empty((B, 1, H, W), dtype=torch.float32, device="cuda")
    net.forward(dev32(x), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 2e-2 * np.max(np.abs(want))
    # one training step: loss, gradients and the first Adam move
    lr = 1e-3
    loss = net.train_step(dev32(x), dev32(t), dev32(mask), lr)
    want_loss, want_grads = cnn.loss_and_grads(params, bf16(x), t.astype(np.float64), mask)
    assert abs(loss - want_loss) <= 2e-2 * want_loss
    p1, g = net.get_params(grads=True)
    for (gw, gb), (ow, ob) in zip(unflatten(g, chans), want_grads):
        assert np.linalg.norm(gw - ow) <= 5e-2 * np.linalg.norm(ow)
        assert np.linalg.norm(gb - ob) <= 5e-2 * max(np.linalg.norm(ob), 1e-12)
    # Adam's first step moves every parameter by lr * g / (|g| + eps)
    step = flat - p1
    np.testing.assert_allclose(step, lr * g / (np.abs(g) + 1e-8), rtol=1e-3, atol=1e-9)


def test_cnn_training_reduces_the_loss_and_rejects_bad_arguments():
    net = M.CNN(layers=3, channels=8, in_channels=2, seed=1)
    rng = np.random.default_rng(9)
    H = W = 24
    x = rng.normal(size=(4, 2, H, W)).astype(np.float32)
    t = (0.5 * x[:, :1] - 0.25 * x[:, 1:]).astype(np.float32)     # a linear target
    mask = np.ones((H, W), dtype=np.float32)
    xd, td, md = dev32(x), dev32(t), dev32(mask)
    losses = [net.train_step(xd, td, md, 3e-3) for _ in range(150)]
    assert losses[-1] < 0.2 * losses[0]
    with pytest.raises(_lib.MfwhError):
        M.CNN(layers=1)
    with pytest.raises(_lib.MfwhError):
        net.set_params(np.zeros(3, dtype=np.float32))


def test_warm_start_features_targets_and_prediction():
    """mfwh_warm_start_data builds x = (f_m / max|f_m|, omega_m / scale) and t = V_m omega_m^2 /
    max|f_m|; mfwh_warm_start maps the network output back, keeping it only if it lowers the
    Helmholtz residual of every frequency (else V^0 = 0)."""
    from paper_2507_23613_gb300 import inputs
    wl = inputs.gaussian_workload("ws", (40, 36), 3, [16.0, 24.0, 33.0], 300.0, 7,
                                  sources_per_freq=2)
    wl.n_p = 2
    s = M.Solver(wl.n, wl.length, wl.omega, torch.from_numpy(wl.forcing).cuda(), n_p=2)
    H, W = wl.n[1] + 1, wl.n[0] + 1
    v = torch.from_numpy(np.random.default_rng(3).normal(size=wl.forcing.shape)).cuda()
    x = torch.empty((wl.nf, 2, H, W), dtype=torch.float32, device="cuda")
    t = torch.empty((wl.nf, 1, H, W), dtype=torch.float32, device="cuda")
    s.warm_start_data(v, x, t, omega_scale=45.0)
    f = wl.forcing
    sc = np.max(np.abs(f.reshape(wl.nf, -1)), axis=1)
    np.testing.assert_allclose(x[:, 0].cpu().numpy(), f / sc[:, None, None], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(x[:, 1].cpu().numpy(),
                               np.broadcast_to((wl.omega / 45.0)[:, None, None], (wl.nf, H, W)),
                               rtol=1e-6)
    vn = v.cpu().numpy()
    want_t = vn / np.max(np.abs(vn.reshape(wl.nf, -1)), axis=1)[:, None, None]
    np.testing.assert_allclose(t[:, 0].cpu().numpy(), want_t, rtol=1e-6, atol=1e-7)
    net = M.CNN(layers=3, channels=8, in_channels=2, seed=4)
    y = torch.empty((wl.nf, 1, H, W), dtype=torch.float32, device="cuda")
    net.forward(x, y)
    torch.cuda.synchronize()
    shape = y[:, 0].cpu().numpy().astype(np.float64)
    shape[:, [0, -1], :] = 0.0
    shape[:, :, [0, -1]] = 0.0
    # the amplitude that minimises the L2 Helmholtz residual, from the oracle's operator
    from oracle import wave as Wv
    g = Wv.Grid(wl.n, wl.length)
    inner = g.interior()
    alpha = []
    for m in range(wl.nf):
        Aphi = Wv.laplacian(shape[m], g, 1.0) + wl.omega[m] ** 2 * shape[m]
        Aphi[[0, -1], :] = 0.0                      # interior points only
        Aphi[:, [0, -1]] = 0.0
        alpha.append(np.sum(Aphi * f[m]) / np.sum(Aphi * Aphi))
    pred = shape * np.array(alpha)[:, None, None]
    v0 = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    kept, ratio = s.warm_start(net, v0, omega_scale=45.0)
    got = v0.cpu().numpy()
    # the kept/rejected decision follows ||b - (v - S v)|| / ||b|| of the prediction
    b = torch.empty_like(v0)
    s.apply_Pi(torch.zeros_like(v0), b, forced=True)
    pv = torch.from_numpy(pred).cuda()
    spv = torch.empty_like(v0)
    s.apply_Pi(pv, spv, forced=False)
    want_ratio = float(torch.linalg.norm(b - (pv - spv)) / torch.linalg.norm(b))
    assert kept == (want_ratio < 1.0)
    if kept:
        np.testing.assert_allclose(got, pred, rtol=1e-5, atol=1e-6 * np.max(np.abs(pred)))
        assert ratio == pytest.approx(want_ratio, rel=1e-6)
    else:
        assert not np.any(got) and ratio == 1.0
    # the fitted amplitude never raises the L2 residual above that of the zero start
    for m in range(wl.nf):
        Aphi = Wv.laplacian(pred[m], g, 1.0) + wl.omega[m] ** 2 * pred[m]
        assert np.linalg.norm((f[m] - Aphi)[inner]) <= np.linalg.norm(f[m][inner]) * (1 + 1e-12)
