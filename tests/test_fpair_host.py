"""The float-pair arithmetic of the FP64 step kernels (csrc/fpair.cuh), compiled for the host
and checked against exact arithmetic (CPU only).

fpair.cuh holds the pair form of the filter sums q_m (eq. pDefQ): fpair_split (the pair of
a new wave value, formed on its bit pattern with integer and FP32 operations), fpair_fma (q +
w x with Dekker's two-product and Knuth's two-sum) and fpair_from / small_int_to_float.  Its
functions use only IEEE float and integer operations with round to nearest, fused
multiply-adds written out as fmaf, and no flush of subnormals, so the host can evaluate
them operation for operation (the host build passes -ffp-contract=off, so that it performs
exactly the operations written; on the GPU the error of whole maps is checked by the
parity tests).  So the header itself, not a re-implementation, is compiled here with a few
bit-cast intrinsics supplied for the host, and its results are compared with exact rational
arithmetic and with the numpy model the parity bound rests on.
"""

import ctypes as C
import os
import shutil
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_23613_gb300", "csrc")
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_fpair_bound import _split_bits  # noqa: E402  (the numpy model of fpair_split)

SHIM = r"""
#include <cstring>
#include <cstdint>
#include <cmath>
// Host versions of the bit casts and the conversion fpair.cuh calls.
static inline long long __double_as_longlong(double v) { long long r; std::memcpy(&r, &v, 8); return r; }
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline float __uint_as_float(unsigned i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned i; std::memcpy(&i, &f, 4); return i; }
static inline float __double2float_rn(double v) { return (float)v; }
#include "fpair.cuh"
extern "C" {
void split_many(const double* v, float* hi, float* lo, long n) {
  for (long i = 0; i < n; ++i) { float2 p = mfwh::fpair_split(v[i]); hi[i] = p.x; lo[i] = p.y; }
}
void from_many(const double* v, float* hi, float* lo, long n) {
  for (long i = 0; i < n; ++i) { float2 p = mfwh::fpair_from(v[i]); hi[i] = p.x; lo[i] = p.y; }
}
void fma_many(const float* wh, const float* wl, const float* xh, const float* xl, float* qh,
              float* ql, long n) {
  for (long i = 0; i < n; ++i) {
    float2 q = mfwh::fpair_fma(wh[i], wl[i], xh[i], xl[i], make_float2(qh[i], ql[i]));
    qh[i] = q.x; ql[i] = q.y;
  }
}
long small_int_mismatches(void) {   // every |i| < 2^22
  long bad = 0;
  for (int i = -(1 << 22) + 1; i < (1 << 22); ++i)
    if (mfwh::small_int_to_float(i) != (float)i) ++bad;
  return bad;
}
}
"""


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def fp(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("fpair")
    src, so = d / "fpair_host.cpp", d / "libfpair_host.so"
    src.write_text(SHIM)
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                    "-I", inc, "-I", CSRC, str(src), "-o", str(so)], check=True,
                   capture_output=True)
    lib = C.CDLL(str(so))
    fptr, dptr = C.POINTER(C.c_float), C.POINTER(C.c_double)
    lib.split_many.argtypes = [dptr, fptr, fptr, C.c_long]
    lib.from_many.argtypes = [dptr, fptr, fptr, C.c_long]
    lib.fma_many.argtypes = [fptr] * 6 + [C.c_long]
    lib.small_int_mismatches.restype = C.c_long
    return lib


def _pairs(fn, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    hi = np.zeros(v.size, np.float32)
    lo = np.zeros(v.size, np.float32)
    p = lambda a, t: a.ctypes.data_as(C.POINTER(t))  # noqa: E731
    fn(p(v, C.c_double), p(hi, C.c_float), p(lo, C.c_float), v.size)
    return hi, lo


def _random_doubles(rng, n, emin, emax):
    e = rng.integers(emin, emax, n)
    m = rng.uniform(1.0, 2.0, n)
    s = rng.choice([-1.0, 1.0], n)
    return s * np.ldexp(m, e)


def test_small_int_to_float_is_exact(fp):
    assert fp.small_int_mismatches() == 0


def test_split_is_the_double_to_2_pow_minus_48(fp):
    """hi + lo = v to within 2^-48 |v| over the normal range of the pair, with hi the float of
    v's 24 leading bits; the error v - hi - lo is computed exactly in float64."""
    rng = np.random.default_rng(5)
    v = _random_doubles(rng, 200000, -100, 116)
    hi, lo = _pairs(fp.split_many, v)
    err = (v - hi.astype(np.float64)) - lo.astype(np.float64)   # exact: both steps are exact
    assert np.all(np.abs(err) <= np.ldexp(np.abs(v), -48))
    assert np.all(np.abs(v - hi.astype(np.float64)) <= np.ldexp(np.abs(v), -24))
    # the kernels' split equals round-to-nearest (fpair_from) except on exact ties
    fh, fl = _pairs(fp.from_many, v)
    same = (fh == hi) & (fl == lo)
    assert same.mean() > 0.999


def test_split_matches_its_numpy_model_bit_for_bit(fp):
    """The numpy model of fpair_split that the parity bound is derived with returns exactly the
    pairs the kernel source computes, across the range, at the edges and for non-finite v."""
    rng = np.random.default_rng(6)
    v = np.concatenate([
        _random_doubles(rng, 100000, -140, 130),
        [0.0, -0.0, 1.0, -1.0, 1.0 - 2.0 ** -30, 2.0 ** 116, -(2.0 ** 116), 2.0 ** 116 * (1 - 2.0 ** -30),
         2.0 ** -126, 2.0 ** -127, 2.0 ** -101, 2.0 ** -100 * 1.5, 5e-324, np.inf, -np.inf, np.nan,
         np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -25]])
    hi, lo = _pairs(fp.split_many, v)
    mh, ml = _split_bits(v)
    same_hi = (hi.view(np.uint32) == mh.view(np.uint32)) | (np.isnan(hi) & np.isnan(mh))
    same_lo = lo.view(np.uint32) == ml.view(np.uint32)
    # a zero's sign is not part of the pair's value
    same_lo |= (lo == 0.0) & (ml == 0.0)
    same_hi |= (hi == 0.0) & (mh == 0.0)
    bad = np.flatnonzero(~(same_hi & same_lo))
    assert bad.size == 0, [(v[i], hi[i], lo[i], mh[i], ml[i]) for i in bad[:5]]


def test_split_edges(fp):
    v = np.array([0.0, 1e-300, 2.0 ** -127, 2.0 ** 116, -(2.0 ** 117), np.inf, -np.inf, np.nan,
                  1.0 - 2.0 ** -30])
    hi, lo = _pairs(fp.split_many, v)
    assert hi[0] == 0 and lo[0] == 0 and hi[1] == 0 and lo[1] == 0 and hi[2] == 0 and lo[2] == 0
    assert np.isposinf(hi[3]) and np.isneginf(hi[4]) and np.isposinf(hi[5]) and np.isneginf(hi[6])
    assert np.isnan(hi[7])
    assert hi[8] == 1.0 and lo[8] == np.float32(-(2.0 ** -30))   # rounding carries into the binade


def test_pair_fma_against_exact_arithmetic(fp):
    """q + (wh + wl)(xh + xl) within 4 * 2^-48 (|q| + |w x|) of the exact value, computed in
    rational arithmetic, with the result renormalised (|lo| <= ulp(hi) / 2)."""
    rng = np.random.default_rng(7)
    n = 4000
    w = _random_doubles(rng, n, -12, 4)
    x = _random_doubles(rng, n, -20, 20)
    q = _random_doubles(rng, n, -20, 30) * rng.choice([0.0, 1.0], n, p=[0.05, 0.95])
    wh, wl = _pairs(fp.from_many, w)
    xh, xl = _pairs(fp.split_many, x)
    qh, ql = _pairs(fp.from_many, q)
    rh, rl = qh.copy(), ql.copy()
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))  # noqa: E731
    fp.fma_many(p(wh), p(wl), p(xh), p(xl), p(rh), p(rl), n)
    F = lambda f: Fraction(float(f))  # noqa: E731
    for i in range(n):
        wx = (F(wh[i]) + F(wl[i])) * (F(xh[i]) + F(xl[i]))
        exact = F(qh[i]) + F(ql[i]) + wx
        got = F(rh[i]) + F(rl[i])
        scale = abs(F(qh[i]) + F(ql[i])) + abs(wx)
        assert abs(got - exact) <= 4 * scale / 2 ** 48, i
        if rh[i] != 0:
            ulp = float(np.spacing(np.float32(abs(rh[i]))))   # float ulp of hi
            assert abs(float(rl[i])) <= 0.5 * ulp, i
