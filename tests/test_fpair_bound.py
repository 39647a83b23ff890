"""The error bound that the GPU parity tests take for the FP64 kernels' filter sums.

Those kernels keep each filter sum q_m = sum_n w_{n,m} W^n (eq. pDefQ) as an unevaluated
pair of floats updated by two-product/two-sum (Dekker's product via FMA, Knuth's two-sum,
a final fast renormalisation).  The parity tests allow a map an absolute error of
N_t 2^-46 of its output.  This test runs the same update sequence in numpy float32 (round to
nearest, FMA emulated exactly through float64 products of float32 operands) on sums of the
bench workload's length and checks the accumulated error against that bound, in the worst
case of no cancellation and in the oscillating case of real filter sums.  CPU only."""

import numpy as np

F32 = np.float32


def _split(v):
    hi = v.astype(F32)
    lo = (v - hi.astype(np.float64)).astype(F32)
    return hi, lo


def _fma32(a, b, c):
    # a * b is exact in float64 for float32 a, b; one rounding of the sum to float32 stands
    # in for the fused operation (the double rounding this can add is far below the bound)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def _pair_update(qh, ql, wh, wl, xh, xl):
    ph = (wh * xh).astype(F32)
    pe = _fma32(wh, xh, -ph)
    pe = _fma32(wh, xl, pe)
    pe = _fma32(wl, xh, pe)
    s = (qh + ph).astype(F32)
    bv = (s - qh).astype(F32)
    e = ((qh - (s - bv)) + (ph - bv)).astype(F32)
    e = (e + (ql + pe)).astype(F32)
    hi = (s + e).astype(F32)
    lo = (e - (hi - s)).astype(F32)
    return hi, lo


def _accumulate(w, x):
    """Pair sums of w[n] * x[n, :] over n; returns (pair value in float64, exact reference,
    largest partial-sum magnitude per column)."""
    qh = np.zeros(x.shape[1], F32)
    ql = np.zeros(x.shape[1], F32)
    ref = np.zeros(x.shape[1])
    comp = np.zeros(x.shape[1])
    peak = np.zeros(x.shape[1])
    for n in range(x.shape[0]):
        wh, wl = _split(np.full(1, w[n]))
        xh, xl = _split(x[n])
        qh, ql = _pair_update(qh, ql, wh, wl, xh, xl)
        # reference: Kahan-compensated float64 sum of float64 products
        y = w[n] * x[n] - comp
        t = ref + y
        comp = (t - ref) - y
        ref = t
        peak = np.maximum(peak, np.abs(ref))
    return qh.astype(np.float64) + ql.astype(np.float64), ref, peak


def test_pair_sum_error_within_parity_bound():
    n_t = 2761                                   # N_t of the 1025^2, N_f = 8 bench workload
    rng = np.random.default_rng(7)
    t = np.arange(n_t) / n_t
    w = (2.0 / n_t) * np.cos(37.0 * t) * (0.75 + 0.25 * np.cos(2 * np.pi * t))
    cols = 512
    # oscillating wave levels (cancelling sums) and same-sign levels (no cancellation)
    phase = rng.uniform(0, 2 * np.pi, size=cols)
    x_osc = np.cos(np.outer(41.0 * t, np.ones(cols)) + phase) * rng.uniform(0.1, 10.0, cols)
    x_pos = rng.uniform(0.5, 1.5, size=(n_t, cols)) * np.sign(w)[:, None]
    bound = n_t * 2.0 ** -46
    for x in (x_osc, x_pos):
        got, ref, peak = _accumulate(w, x)
        err = np.abs(got - ref) / peak
        assert np.max(err) < bound, (np.max(err), bound)
        # and far above FP32 sums: a plain float32 accumulation errs by ~1e-7 here
        assert np.max(err) < 1e-12


def test_pair_renormalisation_invariant():
    """After every update |lo| <= ulp(hi) / 2, so hi alone is the float nearest the sum."""
    rng = np.random.default_rng(3)
    qh = np.zeros(4096, F32)
    ql = np.zeros(4096, F32)
    for _ in range(200):
        wh, wl = _split(rng.normal(size=4096) * 1e-3)
        xh, xl = _split(rng.normal(size=4096))
        qh, ql = _pair_update(qh, ql, wh, wl, xh, xl)
        half_ulp = np.spacing(np.abs(qh)) / 2
        assert np.all(np.abs(ql) <= half_ulp)
