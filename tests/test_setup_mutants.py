"""The host set-up's comparison with the oracle catches plausible mistakes in the library's
set-up code (CPU only).

The library's set-up (paper_2507_23613_gb300/csrc/setup.cpp: time step, adjusted
frequencies, period counts, quadrature weights, Algorithm 2, filter weights, B) is plain
C++.  Each mutant below rewrites one line of it, as a slip in writing it from the paper
would.  The mutated file is compiled with the host compiler together with a small shim that
exports the planner, into a test-only shared object, and its set-up of five problems is
compared with the oracle's: every mutant must disagree.  The unmutated build must agree,
and must return exactly what libmfwh.so's mfwh_plan returns.
"""

import concurrent.futures as cf
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build
from oracle import filters as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_23613_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

# name: (text of setup.cpp, replacement, what it corrupts)
MUTANTS = {
    "trapezoid_overshoot_as_fraction": (
        "double beta = (dt * (k + 1) - t_fm[m]) / dt;", "double beta = (t_fm[m] - dt * k) / dt;",
        "overshoot 1 - r of the partial panel, eq. DefNI"),
    "trapezoid_end_weight": (
        "0.5 * dt * (2.0 - beta * beta) : 0.5 * dt;", "0.5 * dt * (1.0 - beta * beta) : 0.5 * dt;",
        "weight at t_k, eq. DefNI"),
    "trapezoid_after_end_weight": (
        "0.5 * dt * (1.0 - beta) * (1.0 - beta);", "0.5 * dt * (1.0 - beta);",
        "weight at t_{k+1}, eq. DefNI"),
    "optimiser_period_without_n_p": (
        "n_pm[m] = period_count(n_p, omega[m], omega[0]);",
        "n_pm[m] = period_count(1, omega[m], omega[0]);", "N_{p,m} = floor(N_p T_1 / T_m), eq. TbarDef"),
    # (a slip in one of period_count's two correction loops is corrected by the other)
    "period_count_rounded_quotient": (
        "  return (int)k;\n}", "  return (int)std::floor(n_p * (omega_m / omega_1));\n}",
        "N_{p,m} from the rounded quotient (the library's earlier form), eq. TbarDef"),
    "period_count_rounded_products": (
        "while (k > 0 && (long double)k * (long double)omega_1 > num) --k;",
        "while (k > 0 && (long double)(k * omega_1) > num) --k;",
        "exact comparison for the floor of N_p omega_m / omega_1, eq. TbarDef"),
    "optimiser_sine_sign": (
        "fs[m].g[n] = wgt * std::sin(omega[m] * t);", "fs[m].g[n] = -wgt * std::sin(omega[m] * t);",
        "sine component function, eq. compFuncs"),
    "constraint_slope_as_value": (
        "H[(nf + i) * nf + j] = fa[j].slope(omega[i]);", "H[(nf + i) * nf + j] = fa[j].value(omega[i]);",
        "zero-slope constraint rows of H, eq. constraintsVec"),
    # (flipping the sign of every slope would be no mistake: the slopes enter only the
    # homogeneous zero-slope rows of the constraints)
    "cosine_sum_slope_factor": (
        "s -= g[n] * t * std::sin(lam * t);", "s -= g[n] * std::sin(lam * t);",
        "factor t of d/dlambda cos(lambda t) = -t sin(lambda t)"),
    "lambda_range": (
        "const double lam_max = omega[nf - 1] + c_delta * nf * delta;",
        "const double lam_max = omega[nf - 1] + c_delta * delta;", "right end of Lambda, eq. LambdaRange"),
    "lambda_nodes": (
        "double lam = (k + 0.5) * lam_max / n_lambda;", "double lam = (k + 1.0) * lam_max / n_lambda;",
        "midpoint nodes of Algorithm 2"),
    "parameters_c_s_exchanged": (
        "params[3 * m + 1] = y[m];\n    params[3 * m + 2] = y[nf + m];",
        "params[3 * m + 1] = y[nf + m];\n    params[3 * m + 2] = y[m];", "order (a, c, s), eq. yOpt"),
    "lstsq_back_substitution_sign": (
        "for (int j = c + 1; j < cols; ++j) s -= M[c * cols + j] * x[j];",
        "for (int j = c + 1; j < cols; ++j) s += M[c * cols + j] * x[j];",
        "back substitution of the least-squares solve"),
    "lstsq_rhs_reflection": (
        "for (int r = c; r < rows; ++r) d += v[r - c] * b[r];\n    d = 2.0 * d / vnorm2;",
        "for (int r = c; r < rows; ++r) d += v[r - c] * b[r];\n    d = d / vnorm2;",
        "Householder reflection of the right-hand side"),
    "lu_back_substitution_sign": (
        "for (int i = c + 1; i < n; ++i) s -= A[c * n + i] * Bm[i * k + j];",
        "for (int i = c + 1; i < n; ++i) s += A[c * n + i] * Bm[i * k + j];",
        "back substitution of the LU solves (G, B)"),
    "implicit_time_step": (
        "const double x2 = (1.0 - std::cos(theta)) / (0.5 * std::cos(theta));",
        "const double x2 = (1.0 - std::cos(theta)) / std::cos(theta);",
        "implicit dt from omega~_1 dt = theta"),
    "fourth_order_limit": (
        "(P.order == 4 ? std::sqrt(3.0) / 2.0 : 1.0)", "(P.order == 4 ? 0.5 : 1.0)",
        "time-step limit of the fourth-order operator"),
    "time_step_unadjusted": (
        "s.dt = 2.0 * std::sin(kPi * p->n_p / n_t) / p->omega[0];",
        "s.dt = 2.0 * kPi * p->n_p / n_t / p->omega[0];", "dt with omega~_1 N_t dt = 2 pi N_p"),
    "two_layer_c_max": (
        "P.c_max = std::max(p->c_lo, p->c_hi);", "P.c_max = p->c_lo;",
        "c_max of a two-layer medium in the time step"),
    "adjusted_frequency_factor": (
        "double c = (1.0 - 0.5 * beta * x * x) / (1.0 + alpha * x * x);",
        "double c = (1.0 - beta * x * x) / (1.0 + alpha * x * x);", "eq. omegaImplicit"),
    "period_counts_unadjusted": (
        "s.n_pm[m] = period_count(p->n_p, s.omega_tilde[m], s.omega_tilde[0]);",
        "s.n_pm[m] = period_count(p->n_p, p->omega[m], p->omega[0]);",
        "N_{p,m} from omega~, eq. TbarDef"),
    "period_length_unadjusted": (
        "s.t_fm[m] = s.n_pm[m] * (2.0 * kPi / s.omega_tilde[m]);",
        "s.t_fm[m] = s.n_pm[m] * (2.0 * kPi / p->omega[m]);", "T~_{f,m} from omega~, eq. TbarDef"),
    "traditional_factor": (
        "-std::tan(0.5 * wd) / (2.0 * std::tan(wd));", "-std::tan(0.5 * wd) / std::tan(wd);",
        "eq. origParamAdjust"),
    "optimiser_unadjusted_omega": (
        "optimise_parameters(nf, s.omega_tilde, p->n_p", "optimise_parameters(nf, p->omega, p->n_p",
        "Algorithm 2 with inputs omega~"),
    "weights_scale": (
        "P.w[(size_t)n * nf + m] = 2.0 / s.t_fm[m] * sigma", "P.w[(size_t)n * nf + m] = 1.0 / s.t_fm[m] * sigma",
        "factor 2 / T~_{f,m}, eq. pDefQ"),
    "kernel_sine_sign": (
        "prm[3 * m + 1] * std::cos(ph) + prm[3 * m + 2] * std::sin(ph);",
        "prm[3 * m + 1] * std::cos(ph) - prm[3 * m + 2] * std::sin(ph);", "eq. newFilterKernel"),
    "filter_matrix_transposed": (
        "acc += P.w[(size_t)n * nf + m] * P.cosf[(size_t)n * nf + j];",
        "acc += P.w[(size_t)n * nf + j] * P.cosf[(size_t)n * nf + m];", "B_{mj}, eq. filterA"),
}

SHIM = r"""
#include <cstring>
#include <string>
#include "internal.h"
namespace mfwh { void set_error(const std::string&) {} }
extern "C" int shim_plan(const mfwh_problem* p, mfwh_setup* out, double* w, long long cap) {
  mfwh::Plan P;
  const mfwh_status st = mfwh::plan_problem(p, &P, 0.0);
  if (st != MFWH_OK) return (int)st;
  *out = P.s;
  if ((long long)P.w.size() > cap) return -1;
  std::memcpy(w, P.w.data(), sizeof(double) * P.w.size());
  return 0;
}
extern "C" int shim_opt(int nf, const double* omega, int n_p, int n_t, double* params,
                        double* lam_max, int* n_lambda) {
  return (int)mfwh::optimise_parameters(nf, omega, n_p, n_t, 20, 2.0, params, lam_max, n_lambda);
}
"""

# (grid cells, lengths, omega, N_p, c_hi, order, time stepping, filter mode)
CASES = [
    ((64, 64), (1.0, 1.0), [5.5, 9.3], 1, None, 2, "explicit", F.FILTER_OPTIMIZED),
    ((64, 64), (1.0, 1.0), [5.5, 9.3], 1, None, 2, "explicit", F.FILTER_TRADITIONAL),
    ((12, 10, 8), (1.0, 1.0, 1.0), [6.1, 9.7, 15.2], 1, 1.5, 2, "explicit", F.FILTER_OPTIMIZED),
    ((32, 32), (1.0, 1.0), [3.0, 6.0, 12.0], 1, None, 2, "implicit", F.FILTER_OPTIMIZED),
    ((40, 33), (1.3, 0.9), [5.1, 10.1, 15.1], 2, None, 4, "explicit", F.FILTER_OPTIMIZED),
]
_MODE = {F.FILTER_OPTIMIZED: _lib.FILTER_OPTIMIZED, F.FILTER_TRADITIONAL: _lib.FILTER_TRADITIONAL}


def _problem(case):
    n, length, omega, n_p, c_hi, order, ts, mode = case
    kw = dict(n_p=n_p, order=order, time_stepping=ts, filter_mode=_MODE[mode])
    if c_hi is not None:
        kw.update(c_lo=1.0, c_hi=c_hi, interface=0.5, layer_axis=len(n) - 1)
    return M.make_problem(n, length, omega, **kw)


def _oracle(case):
    n, length, omega, n_p, c_hi, order, ts, mode = case
    h = [L / k for L, k in zip(length, n)]
    return F.make_setup(omega, h, 1.0 if c_hi is None else max(1.0, c_hi), 0.5, n_p, mode,
                        order=order, time_stepping=ts)


# Algorithm 2 alone (optimise_parameters) on frequencies given as they are: the second case
# sits at a rounding corner of eq. TbarDef, where omega_3 is the largest double below
# 3 omega_1, so the floating-point quotient omega_3 / omega_1 rounds to 3 while the exact
# ratio, and so N_{p,3} = floor(N_p omega_3 / omega_1) for N_p = 1, stays below (N_{p,3} = 2).
_B, _A = 9.677471780157282, 29.032415340471843
OPT_CASES = [([5.5, 9.3, 14.2], 2, 300), ([_B, 1.7 * _B, _A], 1, 200)]


def _plan(lib, case):
    prob, keep = _problem(case)
    s = _lib.Setup()
    w = np.zeros(1 << 20)
    st = lib.shim_plan(C.byref(prob), C.byref(s), w.ctypes.data_as(C.POINTER(C.c_double)),
                       w.size)
    return st, s, w


def _opt(lib, case):
    omega, n_p, n_t = case
    om = np.ascontiguousarray(omega, dtype=np.float64)
    params = np.zeros((om.size, 3))
    lam, nl = C.c_double(), C.c_int()
    dp = C.POINTER(C.c_double)
    st = lib.shim_opt(om.size, om.ctypes.data_as(dp), n_p, n_t, params.ctypes.data_as(dp),
                      C.byref(lam), C.byref(nl))
    return st, params, lam.value, nl.value


def _opt_disagreement(lib, case, o):
    st, params, lam, nl = _opt(lib, case)
    if st != 0:
        return f"status {st}"
    if nl != o.n_lambda or abs(lam - o.lam_max) > 1e-13 * o.lam_max:
        return "Lambda"
    if np.max(np.abs(params - o.params)) > 1e-10 * np.max(np.abs(o.params)):
        return "parameters"
    return None


def _disagreement(lib, case, o):
    """None if the set-up agrees with the oracle's, else what differs."""
    st, s, w = _plan(lib, case)
    if st != 0:
        return f"status {st}"
    a = M.setup_arrays(s)
    nf = a["nf"]
    w = w[:(a["n_t"] + 1) * nf].reshape(a["n_t"] + 1, nf)
    if a["n_t"] != o.n_t:
        return "N_t"
    checks = [("dt", a["dt"], o.dt, 1e-15), ("omega~", a["omega_tilde"], o.omega_t, 1e-14),
              ("T~_f", a["t_fm"], o.t_fm, 1e-14)]
    for name, got, want, rtol in checks:
        if not np.allclose(got, want, rtol=rtol, atol=0.0):
            return name
    if list(a["n_pm"]) != list(o.n_pm):
        return "N_p,m"
    # every case here is well conditioned (cond(M) < 40): the parameters are determined to 1e-12
    for name, got, want in [("parameters", a["params"], o.params), ("w", w, o.w), ("B", a["B"], o.B)]:
        if np.max(np.abs(got - want)) > 1e-10 * np.max(np.abs(want)):
            return name
    return None


def _compile(name, src_text, out_dir):
    os.makedirs(out_dir, exist_ok=True)
    with open(os.path.join(out_dir, "setup.cpp"), "w") as fh:
        fh.write(src_text)
    with open(os.path.join(out_dir, "shim.cpp"), "w") as fh:
        fh.write(SHIM)
    so = os.path.join(out_dir, f"libsetup_{name}.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(out_dir, "setup.cpp"), os.path.join(out_dir, "shim.cpp"),
                    "-o", so], check=True, capture_output=True)
    lib = C.CDLL(so)
    lib.shim_plan.restype = C.c_int
    lib.shim_plan.argtypes = [C.POINTER(_lib.Problem), C.POINTER(_lib.Setup),
                              C.POINTER(C.c_double), C.c_longlong]
    lib.shim_opt.restype = C.c_int
    lib.shim_opt.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_int,
                             C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]
    return lib


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    with open(os.path.join(CSRC, "setup.cpp")) as fh:
        original = fh.read()
    for name, (old, new, _) in MUTANTS.items():
        assert original.count(old) == 1, name
    base = tmp_path_factory.mktemp("setup_mutants")
    jobs = {None: original}
    jobs.update({n: original.replace(old, new) for n, (old, new, _) in MUTANTS.items()})
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {n: ex.submit(_compile, n or "unmutated", text, str(base / (n or "unmutated")))
                for n, text in jobs.items()}
        return {n: f.result() for n, f in futs.items()}


@pytest.fixture(scope="module")
def oracle_setups():
    return ([_oracle(c) for c in CASES],
            [F.opt_parameters_discrete(om, n_p, n_t) for om, n_p, n_t in OPT_CASES])


def _all_disagreements(lib, oracle_setups):
    plans, opts = oracle_setups
    return ([_disagreement(lib, c, o) for c, o in zip(CASES, plans)]
            + [_opt_disagreement(lib, c, o) for c, o in zip(OPT_CASES, opts)])


def test_unmutated_setup_agrees_with_oracle_and_library(builds, oracle_setups):
    build.build()
    _lib.load()
    assert _all_disagreements(builds[None], oracle_setups) == [None] * (len(CASES) + len(OPT_CASES))
    for case in OPT_CASES:
        st, params, lam, nl = _opt(builds[None], case)
        ref = M.opt_parameters(*case)
        assert np.array_equal(params, ref[0]) and lam == ref[1] and nl == ref[2], case
    for case in CASES:
        # the shim returns exactly what the library's own planner returns
        st, s, w = _plan(builds[None], case)
        prob, keep = _problem(case)
        ref = M.setup_arrays(M.plan(prob))
        got = M.setup_arrays(s)
        for k in ("dt", "n_t", "omega_tilde", "n_pm", "t_fm", "params", "B", "B_inv"):
            assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k])), (case, k)
        nt, nf = ref["n_t"], ref["nf"]
        assert np.array_equal(w[:(nt + 1) * nf].reshape(nt + 1, nf),
                              M.plan_weights(prob, nt, nf)), case


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_oracle_comparison_catches_setup_mutant(builds, oracle_setups, name):
    assert any(f is not None for f in _all_disagreements(builds[name], oracle_setups)), name
