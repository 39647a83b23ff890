"""Pins for the oracle's implicit trapezoidal wave solve ((alpha, beta) = (1/2, 0) in
eq. WaveScheme, first step eq. implicitFirstStep, forcing eq. WaveSchemeForcing, step
count of Section "Time-step determination"): the discrete Helmholtz solution is the
fixed point, the closed-form eigenmode solution (roots of the scheme's characteristic
polynomial), unconditional stability far beyond the explicit step limit, linearity,
GMRES against the direct solve, and planted mistakes that the pins catch.  CPU only."""

import math

import numpy as np
import pytest

from oracle import filters as F
from oracle import wave as W
from paper_2507_23613_gb300 import inputs


def _problem(n, omega, seed=11, b=200.0, c2=1.0, n_p=1, mode=F.FILTER_OPTIMIZED,
             length=None, steps_per_period=10, explicit_filter=False):
    dims = tuple(n)
    wl = inputs.gaussian_workload("t", dims, len(omega), omega, b, seed, length=length)
    g = W.Grid(dims, wl.length)
    return W.make_problem(g, omega, wl.forcing, c2=c2, n_p=n_p, filter_mode=mode,
                          time_stepping="implicit", steps_per_period=steps_per_period,
                          explicit_filter=explicit_filter)


def _mode_angle(lam2, dt, alpha=0.5, beta=0.0):
    """theta with W^n = cos(n theta) phi for the homogeneous scheme on a mode L_h phi = -lam2 phi:
    the roots of (1 + alpha x) r^2 - (2 - beta x) r + (1 + alpha x) = 0, x = lam2 dt^2, are
    exp(+-i theta) (a unit-modulus pair: the scheme neither grows nor decays)."""
    x = lam2 * dt * dt
    r = np.roots([1.0 + alpha * x, -(2.0 - beta * x), 1.0 + alpha * x])
    assert np.allclose(np.abs(r), 1.0, atol=1e-12)
    return float(np.max(np.abs(np.angle(r))))


def _closed_form_Pi(s, lam2, a, v):
    """Coefficients of Pi(V) on one Dirichlet mode: W^n = [sum_j (v_j - u_j) cos(n theta)
    + sum_j u_j cos(omega~_j t^n)] phi with u_j = a_j / (omega_j^2 - lam2)."""
    u = a / (s.omega ** 2 - lam2)
    theta = _mode_angle(lam2, s.dt)
    n = np.arange(s.n_t + 1)
    W_hat = np.cos(n * theta) * np.sum(v - u) + np.cos(np.outer(n * s.dt, s.omega_t)) @ u
    return np.linalg.solve(s.B, s.w.T @ W_hat)


def test_implicit_step_count_and_final_time():
    """N_t = ceil(10 N_p omega_Nf / omega_1); the adjusted frequency omega~_1 makes N_p of its
    periods exactly N_t dt; dt far exceeds the explicit limit at moderate grids."""
    p = _problem((32, 32), [3.0, 6.0, 12.0])
    s = p.setup
    assert s.n_t == 40
    assert s.scheme == F.TRAPEZOIDAL
    assert abs(s.n_t * s.dt - 2 * math.pi / s.omega_t[0]) < 1e-12
    # omega~ from its defining property: the continuous-time solution cos(omega~ t) U solves
    # the scheme for (L_h + omega^2) U = f, i.e. 2 cos(omega~ dt) - 2 = -(omega dt)^2 cos(omega~ dt)
    x = (s.omega * s.dt) ** 2
    c = np.cos(s.omega_t * s.dt)
    np.testing.assert_allclose(2 * c - 2, -x * c, atol=1e-13)
    dt_explicit = 1.0 / math.sqrt(2 * 32.0 ** 2)
    assert s.dt > 2 * dt_explicit
    p2 = _problem((16, 16), [5.0, 7.0], n_p=2, steps_per_period=6)
    assert p2.setup.n_t == math.ceil(6 * 2 * 7.0 / 5.0)


@pytest.mark.parametrize("n", [8, 16, 24])
def test_implicit_fixed_point_is_discrete_helmholtz(n):
    """eq. discreteHelmholtz: with the adjusted frequencies of eq. omegaImplicit the direct
    Helmholtz solution is a fixed point of the implicit map, Pi(U) = U and Pi(Pi(U)) = U."""
    p = _problem((n, n), [5.5, 9.3, 14.0])
    U = W.helmholtz_direct(p)
    PU = W.apply_Pi(p, U)
    scale = np.max(np.abs(U))
    assert np.max(np.abs(PU - U)) / scale < 1e-12
    assert np.max(np.abs(W.apply_Pi(p, PU) - U)) / scale < 1e-12


def test_implicit_fixed_point_3d_two_layer_and_explicit_filter():
    dims = (8, 8, 8)
    c2 = inputs.two_layer_c2(dims, (1.0, 1.0, 1.0), 1.0, 1.5, 0.5)
    for ef in (False, True):
        p = _problem(dims, [4.1, 7.9, 12.5], c2=c2, b=60.0, explicit_filter=ef)
        U = W.helmholtz_direct(p)
        assert np.max(np.abs(W.apply_Pi(p, U) - U)) / np.max(np.abs(U)) < 1e-12


def test_implicit_fixed_point_fourth_order():
    p = W.make_problem(W.Grid((16, 16), (1.0, 1.0)), [5.5, 9.3],
                       inputs.gaussian_workload("t", (16, 16), 2, [5.5, 9.3], 200.0, 3).forcing,
                       order=4, time_stepping="implicit")
    U = W.helmholtz_direct(p)
    assert np.max(np.abs(W.apply_Pi(p, U) - U)) / np.max(np.abs(U)) < 1e-12


def test_implicit_fourth_order_3d_fixed_point_and_eigenmodes():
    """Fourth-order L_4h in 3D with implicit steps: the direct Helmholtz solution of the
    two-layer cube is the fixed point, and superposed Dirichlet modes follow the closed form
    with the fourth-order eigenvalues (theta from the roots of the characteristic
    polynomial)."""
    dims = (8, 8, 8)
    c2 = inputs.two_layer_c2(dims, (1.0, 1.0, 1.0), 1.0, 1.5, 0.5)
    wl = inputs.gaussian_workload("t", dims, 3, [4.1, 7.9, 12.5], 60.0, 4)
    p = W.make_problem(W.Grid(dims, wl.length), wl.omega, wl.forcing, c2=c2, order=4,
                       time_stepping="implicit")
    U = W.helmholtz_direct(p)
    assert np.max(np.abs(W.apply_Pi(p, U) - U)) / np.max(np.abs(U)) < 1e-12
    g = W.Grid((6, 7, 8), (1.0, 1.2, 0.9))
    rng = np.random.default_rng(21)
    f = np.zeros((2,) + g.shape)
    V = np.zeros_like(f)
    coeffs = []
    for k in [(1, 1, 1), (3, 2, 6), (5, 6, 7)]:
        phi, lam2 = W.dirichlet_mode(g, k, order=4)
        a, v = rng.normal(size=2), rng.normal(size=2)
        f += a[:, None, None, None] * phi
        V += v[:, None, None, None] * phi
        coeffs.append((phi, lam2, a, v))
    p = W.make_problem(g, [4.0, 9.5], f, order=4, time_stepping="implicit")
    want = np.zeros_like(f)
    for phi, lam2, a, v in coeffs:
        want += _closed_form_Pi(p.setup, lam2, a, v)[:, None, None, None] * phi
    np.testing.assert_allclose(W.apply_Pi(p, V), want, atol=1e-12)


def test_implicit_eigenmode_closed_form_2d():
    """Dirichlet modes from the lowest to the highest (the highest with lam dt beyond the
    explicit stability limit 2) follow the closed form to rounding."""
    g = W.Grid((20, 24), (1.0, 1.2))
    omega = np.array([5.5, 9.3, 13.1])
    rng = np.random.default_rng(5)
    for k in [(1, 1), (2, 3), (7, 2), (19, 23)]:
        phi, lam2 = W.dirichlet_mode(g, k)
        a = rng.normal(size=3)
        v = rng.normal(size=3)
        p = W.make_problem(g, omega, a[:, None, None] * phi, time_stepping="implicit")
        got = W.apply_Pi(p, v[:, None, None] * phi)
        want = _closed_form_Pi(p.setup, lam2, a, v)
        np.testing.assert_allclose(got, want[:, None, None] * phi,
                                   atol=1e-12 * max(1.0, np.max(np.abs(want))))
    assert math.sqrt(lam2) * p.setup.dt > 2.5   # explicit leapfrog needs lam dt <= 2


def test_implicit_eigenmode_superposition_3d():
    g = W.Grid((6, 7, 8), (1.0, 1.0, 1.0))
    omega = np.array([4.0, 9.5])
    rng = np.random.default_rng(9)
    f = np.zeros((2,) + g.shape)
    V = np.zeros_like(f)
    coeffs = []
    for k in [(1, 1, 1), (2, 5, 3), (5, 6, 7)]:
        phi, lam2 = W.dirichlet_mode(g, k)
        a, v = rng.normal(size=2), rng.normal(size=2)
        f += a[:, None, None, None] * phi
        V += v[:, None, None, None] * phi
        coeffs.append((phi, lam2, a, v))
    p = W.make_problem(g, omega, f, time_stepping="implicit")
    want = np.zeros_like(f)
    for phi, lam2, a, v in coeffs:
        want += _closed_form_Pi(p.setup, lam2, a, v)[:, None, None, None] * phi
    np.testing.assert_allclose(W.apply_Pi(p, V), want, atol=1e-12)


def test_implicit_linearity():
    p = _problem((14, 10), [5.5, 9.3, 12.0])
    rng = np.random.default_rng(2)
    x = rng.normal(size=p.forcing.shape)
    y = rng.normal(size=p.forcing.shape)
    for arr in (x, y):
        for m in range(arr.shape[0]):
            W.zero_boundary(arr[m], p.grid)
    Sx = W.apply_Pi(p, x, forced=False)
    Sy = W.apply_Pi(p, y, forced=False)
    np.testing.assert_allclose(W.apply_Pi(p, 2.5 * x - y, forced=False), 2.5 * Sx - Sy, atol=1e-12)
    b = W.apply_Pi(p, np.zeros_like(x))
    np.testing.assert_allclose(W.apply_Pi(p, x), Sx + b, atol=1e-12)


def test_implicit_gmres_converges_to_direct_solution():
    p = _problem((12, 12), [5.5, 9.3])
    U = W.helmholtz_direct(p)
    x, info = W.gmres(p, restart=200, tol=1e-12, max_iters=400)
    assert info.converged
    assert np.max(np.abs(x - U)) / np.max(np.abs(U)) < 1e-9
    assert np.max(W.helmholtz_residual(p, x)) < 1e-9


def test_planted_mistake_forcing_factor(monkeypatch):
    """Planted mistake: dropping the factor (beta + 2 alpha cos(omega~ dt)) of eq.
    WaveSchemeForcing breaks the fixed point."""
    p = _problem((12, 12), [5.5, 9.3])
    U = W.helmholtz_direct(p)
    s = p.setup

    def no_factor(prob, n):
        F_ = np.zeros(prob.grid.shape)
        inner = prob.grid.interior()
        for m in range(prob.nf):
            F_[inner] += prob.forcing[m][inner] * math.cos(s.omega_t[m] * n * s.dt)
        return F_

    monkeypatch.setattr(W, "composite_forcing", no_factor)
    assert np.max(np.abs(W.apply_Pi(p, U) - U)) / np.max(np.abs(U)) > 1e-3


def test_planted_mistake_explicit_frequencies():
    """Planted mistake: the explicit scheme's omega~ with implicit steps is caught by the
    eigenmode pin."""
    g = W.Grid((12, 12), (1.0, 1.0))
    phi, lam2 = W.dirichlet_mode(g, (2, 1))
    a, v = np.array([1.0, -0.5]), np.array([0.3, 0.8])
    p = W.make_problem(g, [5.5, 9.3], a[:, None, None] * phi, time_stepping="implicit")
    want = _closed_form_Pi(p.setup, lam2, a, v)[:, None, None] * phi
    assert np.max(np.abs(W.apply_Pi(p, v[:, None, None] * phi) - want)) < 1e-12
    s = p.setup
    s.omega_t = F.adjusted_frequency(s.omega, s.dt, F.EXPLICIT)
    s.B = F.filter_matrix(s.w, s.omega_t, s.dt)
    assert np.max(np.abs(W.apply_Pi(p, v[:, None, None] * phi) - want)) > 1e-4
