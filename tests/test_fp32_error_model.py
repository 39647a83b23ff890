"""Where the FP32 path's parity tolerance comes from (CPU only).

The FP32 wave path (precision MFWH_PREC_FP32_KAHAN) advances the leapfrog scheme (eq.
WaveSchemeA, first step eq. implicitFirstStep) in increment form with FP32 wave levels,
D^{n+1} = D^n + kappa (c^2 Delta_h W^n - F^n), W^{n+1} = W^n + D^{n+1}, accumulates the
filter sums (eq. pDefQ) as Kahan pairs (or, in its blocked form, as plain float32 partial
sums over each launch folded into the Kahan pairs), and solves B V = q in FP64.  This test writes that
arithmetic out in numpy float32, operation by operation in the kernels' order (coefficients
and weights rounded to float32 on the host; a fused multiply-add as the float32 rounding of
its exact float64 value), and measures how far one map Pi lands from the FP64 oracle per
frequency, e_m = max |V_32 - V_64| / max |V_64|.  The GPU tests allow e_m <= 2e-5 for one
map on these grids; the model must stay at least four times below that, so the tolerance
covers the arithmetic with a margin for the GPU's different but equally accurate rounding
order, and is not fitted to a measurement.
"""

import numpy as np
import pytest

from oracle import filters as F
from oracle import wave as W
from paper_2507_23613_gb300 import inputs

TOL_PI32 = 2e-5           # the GPU tests' bound for one FP32 map (tests/test_gpu_fp32.py)
f32 = np.float32


def _fma32(a, b, c):
    """float32 fused multiply-add: the exact a b + c (float64 holds a float32 product exactly)
    rounded once to float32 (the rare double rounding through float64 is immaterial here)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(f32)


def _pi_fp32(p, V, forced, block=0):
    """One map Pi (or S for forced=False) in the FP32 path's arithmetic.  block = 0: Kahan
    update at every step (MFWH_PREC_FP32_KAHAN); block = T: plain float32 partial sums over
    each launch of T steps, folded into the Kahan pair at the launch's end
    (MFWH_PREC_FP32_BLOCKSUM)."""
    s = p.setup
    g = p.grid
    inner = g.interior()
    dim = g.dim
    c2 = np.asarray(p.c2, dtype=np.float64)
    W0 = np.zeros(g.shape)
    W0[inner] = np.sum(V, axis=0)[inner]
    w = W0.astype(f32)                                   # W^0 = fl32(sum_m V_m)
    D = np.zeros(g.shape, f32)
    wq = s.w.astype(f32)
    qs = np.stack([(wq[0, m] * w).astype(f32) for m in range(p.nf)])
    qc = np.zeros_like(qs)
    part = np.zeros_like(qs)
    ff = p.forcing.astype(f32)
    inv_h2 = [1.0 / (h * h) for h in g.h]                # h listed x first; array axes reversed
    for n in range(s.n_t):
        kappa = 0.5 * s.dt ** 2 if n == 0 else s.dt ** 2
        # per-axis coefficients kappa c^2 / h_i^2 rounded to float32 (one per c^2 value)
        coef = [(kappa * c2 * ih).astype(f32) if c2.ndim else f32(kappa * float(c2) * ih)
                for ih in inv_h2]
        fc = [f32(kappa * np.cos(s.omega_t[m] * n * s.dt)) for m in range(p.nf)]
        wc = w[inner]
        diffs = []
        for axis_x in range(dim):                        # axis_x = 0 is x, the last array axis
            ax = dim - 1 - axis_x
            plus = [slice(1, -1)] * dim
            minus = [slice(1, -1)] * dim
            plus[ax] = slice(2, None)
            minus[ax] = slice(0, -2)
            diffs.append(((w[tuple(plus)] - wc) + (w[tuple(minus)] - wc)).astype(f32))
        cf = [c[inner] if np.ndim(c) else c for c in coef]
        # inc = Ay dyy, then fma(Az, dzz, inc), fma(Ax, dxx, inc), fma(-fc_m, f_m, inc)
        inc = (cf[1] * diffs[1]).astype(f32)
        if dim == 3:
            inc = _fma32(cf[2], diffs[2], inc)
        inc = _fma32(cf[0], diffs[0], inc)
        if forced:
            for m in range(p.nf):
                inc = _fma32(-fc[m], ff[m][inner], inc)
        dn = (D[inner] + inc).astype(f32)
        wn = (wc + dn).astype(f32)
        D[inner] = dn
        w = w.copy()
        w[inner] = wn
        for m in range(p.nf):
            if block:                                    # partial sum of the launch
                part[m][inner] = _fma32(wq[n + 1, m], wn, part[m][inner])
                if (n + 1) % block == 0 or n + 1 == s.n_t:     # fold at the launch's end
                    sm, cm, x = qs[m][inner], qc[m][inner], part[m][inner]
                    y = (x - cm).astype(f32)
                    t = (sm + y).astype(f32)
                    qc[m][inner] = ((t - sm) - y).astype(f32)
                    qs[m][inner] = t
                    part[m][inner] = 0.0
                continue
            sm, cm = qs[m][inner], qc[m][inner]          # Kahan update with w_{n+1,m}
            y = _fma32(wq[n + 1, m], wn, -cm)
            t = (sm + y).astype(f32)
            qc[m][inner] = ((t - sm) - y).astype(f32)
            qs[m][inner] = t
    q = qs.astype(np.float64) - qc.astype(np.float64)
    out = np.linalg.solve(s.B, q.reshape(p.nf, -1)).reshape(q.shape)
    for m in range(p.nf):
        W.zero_boundary(out[m], g)
    return out


def _rel_err(got, want):
    got = got.reshape(got.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return np.max(np.abs(got - want), axis=1) / np.max(np.abs(want), axis=1)


def _random_v(wl, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=wl.forcing.shape) * 0.01
    g = W.Grid(wl.n, wl.length)
    for m in range(v.shape[0]):
        W.zero_boundary(v[m], g)
    return v


def _cases():
    sq = inputs.square_small()
    rag = inputs.gaussian_workload("ragged", (70, 45), 8,
                                   lambda r: inputs.draw_frequencies(r, 8, 10.0, 60.0), 400.0, 77,
                                   length=(1.3, 0.9))
    cube = inputs.gaussian_workload("cube", (20, 18, 16), 3, [6.1, 9.7, 15.2], 300.0, 5)
    zc = np.zeros((17, 19, 21))                          # [z][y][x]
    zc[:8] = 1.0
    zc[8:] = 2.25                                        # c = 1 below z = 0.5, 1.5 from it on
    return [("square65_nf2", sq, 1, 1.0), ("ragged70x45_nf8", rag, 2, 1.0),
            ("cube20x18x16_two_layer", cube, 1, zc)]


@pytest.mark.parametrize("name,wl,n_p,c2", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_fp32_arithmetic_stays_well_inside_the_gpu_tolerance(name, wl, n_p, c2):
    g = W.Grid(wl.n, wl.length)
    p = W.make_problem(g, wl.omega, wl.forcing, c2=c2, n_p=n_p,
                       filter_mode=F.FILTER_TRADITIONAL)
    v = _random_v(wl, 3)
    blocks = (0, 16) if g.dim == 2 else (0, 4)           # the blocked FP32 kernels' depths
    for forced in (True, False):
        want = W.apply_Pi(p, v, forced=forced)
        for block in blocks:
            err = _rel_err(_pi_fp32(p, v, forced, block), want)
            assert np.all(err <= TOL_PI32 / 4), (name, forced, block, err)
            assert np.all(err > 1e-9), (name, forced, block, err)   # the model does round
