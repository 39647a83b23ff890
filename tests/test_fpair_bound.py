"""The error bound that the GPU parity tests take for the FP64 kernels' filter sums.

Those kernels keep each filter sum q_m = sum_n w_{n,m} W^n (eq. pDefQ) as an unevaluated
pair of floats updated by two-product/two-sum (Dekker's product via FMA, Knuth's two-sum,
a final fast renormalisation); each new wave value enters as a pair split off its bit
pattern (fpair_split) and each weight as the host's round-to-nearest pair.  The parity
tests allow a map an absolute error of N_t 2^-46 of its output.  This test runs the same update sequence in numpy float32 (round to
nearest, FMA emulated exactly through float64 products of float32 operands) on sums of the
bench workload's length and checks the accumulated error against that bound, in the worst
case of no cancellation and in the oscillating case of real filter sums.  CPU only."""

import numpy as np

F32 = np.float32


def _split(v):
    hi = v.astype(F32)
    lo = (v - hi.astype(np.float64)).astype(F32)
    return hi, lo


def _split_bits(v):
    """The step kernels' pair of a double formed on the bit pattern (fpair_split): |v| rounded
    to 24 significant bits (ties away from zero) by integer arithmetic, the remainder as an
    integer count of units 2^(e - 1075) converted to float and scaled by powers of two."""
    with np.errstate(over="ignore", invalid="ignore"):
        return _split_bits_raw(np.asarray(v, dtype=np.float64))


def _split_bits_raw(v):
    bits = v.view(np.uint64)
    a = bits & np.uint64(0x7FFFFFFFFFFFFFFF)
    h = (a + np.uint64(1 << 28)) & ~np.uint64((1 << 29) - 1)
    eh = (h >> np.uint64(52)).astype(np.int64)
    ev = (a >> np.uint64(52)).astype(np.int64)
    neg = (bits >> np.uint64(63)).astype(bool)
    hi_mag = h.view(np.float64).astype(F32)                 # exact: 24 significant bits
    d = (a.astype(np.int64) - h.astype(np.int64))           # |d| <= 2^28
    # d 2^k with k = ev - 1075, as (d 2^kk) 2^(k - kk) in float32 (kk = k + 64 when 2^k is not
    # a normal float): the first product is exact, the second rounds only to a subnormal
    k = ev - 1075
    low = k < -126
    kk = np.clip(np.where(low, k + 64, k), -126, 127)
    s1 = np.ldexp(np.ones(k.shape), kk).astype(F32)
    s2 = np.where(low, F32(2.0 ** -64), F32(1.0)).astype(F32)
    lo_mag = ((d.astype(F32) * s1).astype(F32) * s2).astype(F32)
    small = eh < 897
    hi = np.where(neg, -hi_mag, hi_mag).astype(F32)
    lo = np.where(neg, -lo_mag, lo_mag).astype(F32)
    hi[small] = 0.0
    lo[small] = 0.0
    big = eh > 1138                                         # |v| >= 2^116, inf, NaN
    hi[big] = np.where(np.isnan(v[big]), np.float32(np.nan),
                       np.where(neg[big], -np.inf, np.inf)).astype(F32)
    lo[big] = 0.0
    return hi, lo


def test_bit_split_is_a_pair_of_the_double():
    """hi + lo = v to 2^-48 |v| across magnitudes 2^-100 .. 2^110 (below about 2^-101 lo is a
    subnormal float and the pair keeps 2^-150 absolute) and both signs; it matches the
    round-to-nearest split except on exact ties of the rounding bit; zero and values below
    2^-126 give (0, 0); from 2^116 on hi is infinite, and NaN stays NaN."""
    rng = np.random.default_rng(5)
    v = rng.uniform(1.0, 2.0, 200000) * np.exp2(rng.integers(-100, 110, 200000))
    v *= np.where(rng.random(200000) < 0.5, -1.0, 1.0)
    hi, lo = _split_bits(v)
    err = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - v) / np.abs(v)
    assert np.max(err) <= 2.0 ** -48, np.max(err)
    rh, rl = _split(v)
    same = (hi == rh) & (lo == rl)
    assert np.mean(same) > 0.9999
    # a value with the rounding bit set and nothing below it: ties go away from zero
    tie = np.array([1.0 + 2.0 ** -24, -(1.0 + 3 * 2.0 ** -24)])
    th, tl = _split_bits(tie)
    assert th[0] == np.float32(1.0 + 2.0 ** -23) and tl[0] == np.float32(-(2.0 ** -24))
    assert th[1] == np.float32(-(1.0 + 2.0 ** -22)) and tl[1] == np.float32(2.0 ** -24)
    # a rounding carry into the next binade keeps the remainder exact
    c = np.array([2.0 - 2.0 ** -30])
    ch, cl = _split_bits(c)
    assert ch[0] == 2.0 and cl[0] == np.float32(-(2.0 ** -30))
    zh, zl = _split_bits(np.array([0.0, -0.0, 1e-39, 3e-300]))
    assert np.all(zh == 0) and np.all(zl == 0)
    tiny = np.array([3.1e-35, -7.7e-38])       # subnormal lo: 2^-150 absolute
    yh, yl = _split_bits(tiny)
    assert np.all(np.abs(yh.astype(np.float64) + yl.astype(np.float64) - tiny) <= 2.0 ** -149)
    sh, sl = _split_bits(np.array([np.inf, -np.inf, np.nan, 1e36, -2.0 ** 120]))
    assert sh[0] == np.inf and sh[1] == -np.inf and np.isnan(sh[2])
    assert sh[3] == np.inf and sh[4] == -np.inf and np.all(sl == 0)   # saturate from 2^116


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
        xh, xl = _split_bits(x[n])
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
