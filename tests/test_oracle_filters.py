"""Pins for the oracle's set-up arithmetic (filters, weights, B) against values the
paper prints, closed forms and the paper's theorems.  CPU only."""

import json
from fractions import Fraction
import math
import os

import numpy as np
import pytest

from oracle import filters as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_filter_parameters.json")


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


# ---------------------------------------------------------------------------
# Algorithm 2 against the printed parameter tables
# ---------------------------------------------------------------------------

def test_table_params_continuous(printed_close):
    """Table tab:params: omega = 5, 9 with exact time integrals, N_p = 1, 2, 3."""
    g = golden()["continuous_omega_5_9"]
    for row in g["rows"]:
        r = F.opt_parameters_continuous(g["omega"], row["n_p"])
        assert list(r.n_pm) == row["n_pm"]
        printed_close(r.lam_max, row["lam_max"], f"lam_max N_p={row['n_p']}")
        for m, p in enumerate(row["params"]):
            for k in range(3):
                printed_close(r.params[m, k], p[k], f"N_p={row['n_p']} p[{m}][{k}]")


def _discrete_case(case):
    om = np.asarray(case["omega"])
    dt, n_t = F.implicit_time_step(om[0], om[-1], case["n_p"])
    omt = F.adjusted_frequency(om, dt, F.TRAPEZOIDAL)
    return dt, n_t, F.opt_parameters_discrete(omt, case["n_p"], n_t)


@pytest.mark.parametrize("idx", range(4))
def test_discrete_printed_cases(idx, printed_close):
    """The optimised-parameter cases of Section 'Numerical results': Lambda, N_lambda,
    N_t, T_f, N_{p,m} and (where printed correctly) the parameters themselves."""
    case = golden()["discrete_cases"][idx]
    dt, n_t, r = _discrete_case(case)
    assert n_t == case["n_t"]
    assert r.n_lambda == case["n_lambda"]
    assert list(r.n_pm) == case["n_pm"]
    if "lam_max_abs_tol" in case:
        assert abs(r.lam_max - float(case["lam_max"])) <= case["lam_max_abs_tol"]
    else:
        printed_close(r.lam_max, case["lam_max"], "lam_max")
    printed_close(r.t_f, case["t_f"], "T_f")
    assert abs(r.t_f - n_t * dt) < 1e-12 * r.t_f
    if case.get("params"):
        for m, p in enumerate(case["params"]):
            for k in range(3):
                printed_close(r.params[m, k], p[k], f"p[{m}][{k}]")
    if case.get("params_columns"):
        for k, key in enumerate("acs"):
            for m, text in enumerate(case["params_columns"][key]):
                printed_close(r.params[m, k], text, f"{key}[{m}]")


def test_discrete_tends_to_continuous():
    """The discrete (trapezoid) optimiser converges to the continuous one as N_t grows."""
    cont = F.opt_parameters_continuous([5.0, 9.0], 1).params
    errs = [np.max(np.abs(F.opt_parameters_discrete([5.0, 9.0], 1, nt).params - cont))
            for nt in (200, 400)]
    assert errs[1] < errs[0] / 3.0       # second order in dt
    assert errs[1] < 1e-3


# ---------------------------------------------------------------------------
# Quadrature, component functions, adjusted frequencies
# ---------------------------------------------------------------------------

def _sinc(x):
    return np.sinc(x / math.pi)


def _cosc(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-6
    out[~small] = (1.0 - np.cos(x[~small])) / x[~small]
    out[small] = x[small] / 2.0
    return out


def test_component_functions_closed_form():
    """eq. compFuncs: f_a = 2 sinc(lambda T), f_c = sinc((w-l)T) + sinc((w+l)T),
    f_s = cosc((w-l)T) + cosc((w+l)T) against the Gauss-Legendre integrals the
    continuous optimiser uses."""
    omega = np.array([5.0, 9.0])
    n_pm, t_fm, _ = F.period_counts(omega, 2)
    x, wx = np.polynomial.legendre.leggauss(512)
    basis = F._QuadratureBasis(omega, t_fm, [0.5 * t * (x + 1) for t in t_fm],
                               [0.5 * t * wx for t in t_fm])
    lam = np.linspace(0.01, 30.0, 301)
    for m in range(2):
        T, w = t_fm[m], omega[m]
        np.testing.assert_allclose(basis.f("a", lam, m), 2 * _sinc(lam * T), atol=1e-12)
        np.testing.assert_allclose(basis.f("c", lam, m), _sinc((w - lam) * T) + _sinc((w + lam) * T), atol=1e-12)
        np.testing.assert_allclose(basis.f("s", lam, m), _cosc((w - lam) * T) + _cosc((w + lam) * T), atol=1e-12)
        # derivative: centred difference of the closed form
        d = 1e-5
        fd = (_sinc((w - lam - d) * T) + _sinc((w + lam + d) * T)
              - _sinc((w - lam + d) * T) - _sinc((w + lam - d) * T)) / (2 * d)
        np.testing.assert_allclose(basis.fp("c", lam, m), fd, atol=1e-7)


def test_trapezoid_weights_exact_for_linears():
    """eq. DefNI: the rule integrates linear functions exactly on [0, T_{f,m}], and on
    a grid-aligned interval it is the plain trapezoid rule."""
    dt, n_t = 0.0137, 97
    # the last case has T_{f,m} < dt: no full panel, only the partial one from t_0
    t_fm = np.array([n_t * dt, 0.731, 1.0003, 0.5 * dt * 3, 0.4 * dt])
    sigma = F.trapezoid_weights(n_t, dt, t_fm)
    t = np.arange(n_t + 1) * dt
    for m, T in enumerate(t_fm):
        assert abs(sigma[:, m].sum() - T) < 1e-13
        assert abs(sigma[:, m] @ t - 0.5 * T * T) < 1e-13
        assert abs(sigma[:, m] @ (3.0 - 2.0 * t) - (3.0 * T - T * T)) < 1e-13
        last = int(math.floor(T / dt)) + 1
        assert np.all(sigma[last + 1:, m] == 0.0)
        assert np.all(sigma[:, m] >= 0.0)
    trap = np.full(n_t + 1, dt)
    trap[0] = trap[-1] = 0.5 * dt
    np.testing.assert_allclose(sigma[:, 0], trap, atol=1e-15)


def test_trapezoid_second_order():
    """Composite trapezoid error is O(dt^2) on a smooth integrand over a non-aligned end."""
    T = 1.2345
    errs = []
    for n in (100, 200):
        dt = 1.5 / n
        s = F.trapezoid_weights(n, dt, [T])[:, 0]
        t = np.arange(n + 1) * dt
        errs.append(abs(s @ np.cos(3.0 * t) - math.sin(3.0 * T) / 3.0))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_adjusted_frequency_defining_property():
    """eq. omegaImplicit: leapfrog applied to cos(omega~ t) reproduces -omega^2 exactly,
    i.e. (2 - 2 cos(omega~ dt)) / dt^2 = omega^2; the trapezoidal form satisfies
    (2 - 2 cos(omega~ dt)) / dt^2 = omega^2 cos(omega~ dt), and omega~ -> omega as dt -> 0."""
    om = np.array([3.0, 5.5, 9.3, 41.0])
    dt = 0.011
    wt = F.adjusted_frequency(om, dt, F.EXPLICIT)
    np.testing.assert_allclose((2 - 2 * np.cos(wt * dt)) / dt ** 2, om ** 2, rtol=1e-10)
    assert np.all(wt > om)
    wi = F.adjusted_frequency(om, dt, F.TRAPEZOIDAL)
    np.testing.assert_allclose((2 - 2 * np.cos(wi * dt)) / dt ** 2, om ** 2 * np.cos(wi * dt), rtol=1e-10)
    assert np.all(wi < om)
    np.testing.assert_allclose(F.adjusted_frequency(om, 1e-4), om, rtol=1e-5)


def test_explicit_time_step():
    """Explicit step: omega~_1 N_t dt = 2 pi N_p, dt below CFL * von Neumann limit, N_t minimal."""
    h = (1 / 64, 1 / 64)
    dt, n_t = F.explicit_time_step(h, 1.0, 0.5, 5.5, 1)
    assert n_t == 207                             # ceil((2 pi / 5.5) / (0.5 h / sqrt 2))
    wt = F.adjusted_frequency(5.5, dt)
    assert abs(wt * n_t * dt - 2 * math.pi) < 1e-12
    dt_stab = (1 / 64) / math.sqrt(2)
    assert dt <= 0.5 * dt_stab
    assert (2 * math.pi / 5.5) / (n_t - 1) > 0.5 * dt_stab
    # leapfrog stability margin: lambda_max^2 dt^2 / 4 < 1
    lam2 = 8 / (1 / 64) ** 2
    assert lam2 * dt * dt / 4 < 0.3


# ---------------------------------------------------------------------------
# Theorems 2 and 3 and the constraint structure
# ---------------------------------------------------------------------------

def _setup(omega, filter_mode, h=(1 / 64, 1 / 64), n_p=1):
    return F.make_setup(omega, h, 1.0, 0.5, n_p, filter_mode)


def test_theorem2_mu_is_nonzero_eigenvalue():
    """Theorem 2: the non-zero eigenvalue of B^{-1} C_lambda equals sum_m gamma_m beta_m(lambda)."""
    s = _setup([5.5, 9.3, 14.2], F.FILTER_TRADITIONAL)
    for lam in (2.0, 7.7, 12.0, 30.0):
        beta = F.discrete_beta(s.w, lam, s.dt)[0]
        C = np.outer(beta, np.ones(3))
        ev = np.linalg.eigvals(np.linalg.solve(s.B, C))
        nonzero = ev[np.argmax(np.abs(ev))]
        assert abs(nonzero - F.mu_discrete(s.B, s.w, lam, s.dt)[0]) < 1e-12
        assert np.sum(np.abs(ev) < 1e-12) == 2


@pytest.mark.parametrize("mode", [F.FILTER_TRADITIONAL, F.FILTER_OPTIMIZED])
def test_theorem3_mu_equals_one_at_frequencies(mode):
    """Theorem 3: mu(omega~_m) = 1 for any parameters."""
    s = _setup([5.5, 9.3, 14.2, 20.5], mode)
    np.testing.assert_allclose(F.mu_discrete(s.B, s.w, s.omega_t, s.dt), 1.0, atol=1e-11)


def test_optimised_constraints():
    """eq. constraintsT: with the optimised parameters the column sums of B are 1
    (gamma_m = 1) and mu_d has zero slope at every omega~_m."""
    s = _setup([5.5, 9.3, 14.2], F.FILTER_OPTIMIZED)
    np.testing.assert_allclose(s.B.sum(axis=0), 1.0, atol=1e-12)
    d = 1e-6
    slope = (F.mu_discrete(s.B, s.w, s.omega_t + d, s.dt) - F.mu_discrete(s.B, s.w, s.omega_t - d, s.dt)) / (2 * d)
    assert np.max(np.abs(slope)) < 1e-6


def test_traditional_parameters_flat_at_frequency():
    """eq. origParamAdjust: with p = (a_m, 1, 0) beta_{d,m} has zero slope at omega~_m for a
    single frequency (the trapezoid grid is aligned there), and a_m -> -1/4 as dt -> 0."""
    s = _setup([6.0], F.FILTER_TRADITIONAL)
    d = 1e-6
    b = lambda lam: F.discrete_beta(s.w, lam, s.dt)[:, 0]
    slope = (b(s.omega_t[0] + d) - b(s.omega_t[0] - d)) / (2 * d)
    assert abs(slope[0]) < 1e-7
    a = F.traditional_parameters([6.0], 1e-5)[0, 0]
    assert abs(a + 0.25) < 1e-8


def test_two_frequency_gamma_formula():
    """The N_f = 2 weights printed after Figure BetaTerms equal the column sums of B^{-1}."""
    s = _setup([5.5, 9.3], F.FILTER_TRADITIONAL)
    b11, b12, b21, b22 = s.B[0, 0], s.B[0, 1], s.B[1, 0], s.B[1, 1]
    det = b11 * b22 - b21 * b12
    g1 = (b22 - b21) / det
    g2 = (b11 - b12) / det
    np.testing.assert_allclose(np.linalg.inv(s.B).sum(axis=0), [g1, g2], rtol=1e-12)


def test_filter_matrix_definition():
    """B_{mj} equals the discrete filter function beta_{d,m} evaluated at omega~_j."""
    s = _setup([5.5, 9.3, 14.2], F.FILTER_OPTIMIZED)
    np.testing.assert_allclose(s.B, F.discrete_beta(s.w, s.omega_t, s.dt).T, atol=1e-14)


def test_period_count_of_the_first_frequency_is_n_p():
    """eq. TbarDef: T_f = N_p T_1, so N_{p,1} = floor(T_f / T_1) = N_p exactly.  Forming
    N_p omega_1 / omega_1 in floating point can round below N_p (about 7 % of random omega_1
    for N_p = 3); these values are such cases."""
    for n_p, w1 in [(3, 6.324608295390162), (5, 6.692997385840716), (6, 25.67958426865055),
                    (7, 18.463274230059614)]:
        assert math.floor(n_p * w1 / w1) == n_p - 1          # the rounding trap
        n_pm, t_fm, t_f = F.period_counts(np.array([w1, 2.3 * w1]), n_p)
        assert n_pm[0] == n_p
        assert abs(t_fm[0] - t_f) <= 1e-15 * t_f
    rng = np.random.default_rng(12)
    for _ in range(200):
        w = np.sort(rng.uniform(1.0, 80.0, size=4))
        n_p = int(rng.integers(1, 8))
        n_pm, _, _ = F.period_counts(w, n_p)
        assert n_pm[0] == n_p
        # brute force of the definition: the largest k with k T_m <= T_f, in exact arithmetic
        t_f = Fraction(n_p) / Fraction(float(w[0]))
        for m in range(4):
            k = int(n_pm[m])
            assert Fraction(k) / Fraction(float(w[m])) <= t_f < Fraction(k + 1) / Fraction(float(w[m]))
