"""Pins for the oracle's MFWH map, iterations and residual against the discrete
Helmholtz solution (sparse direct solve), the closed-form Dirichlet eigenmode
recurrence, linearity, the spectrum of S, a dense solve and brute force.  CPU only."""

import math

import numpy as np
import pytest

from oracle import filters as F
from oracle import wave as W
from paper_2507_23613_gb300 import inputs


def _problem(n, omega, seed=11, b=200.0, mode=F.FILTER_OPTIMIZED, c2=1.0, length=None):
    dims = tuple(n)
    wl = inputs.gaussian_workload("t", dims, len(omega), omega, b, seed, length=length)
    g = W.Grid(dims, wl.length)
    return W.make_problem(g, omega, wl.forcing, c2=c2, filter_mode=mode)


def _closed_form_Pi(s, lam2, a, v):
    """Coefficients of Pi(V) on one Dirichlet mode phi with L_h phi = -lam2 phi.

    For W^0 = sum_j v_j phi and forcing a_j phi the leapfrog solution is exactly
    W^n = [sum_j (v_j - u_j) T_n(1 - lam2 dt^2 / 2) + sum_j u_j cos(omega~_j t^n)] phi
    with u_j = a_j / (omega_j^2 - lam2) (the discrete Helmholtz coefficient) and
    T_n the Chebyshev polynomial (the error recurrence of Section 'Analysis' carried
    to the discrete level).  Filtering with w and solving with B gives the new V.
    """
    u = a / (s.omega ** 2 - lam2)
    x = 1.0 - 0.5 * lam2 * s.dt ** 2
    n = np.arange(s.n_t + 1)
    cheb = np.cos(n * np.arccos(x))
    cosw = np.cos(np.outer(n * s.dt, s.omega_t))
    W_hat = cheb * np.sum(v - u) + cosw @ u
    q = s.w.T @ W_hat
    return np.linalg.solve(s.B, q)


# ---------------------------------------------------------------------------
# Discrete Helmholtz solution is the fixed point
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 16, 32])
def test_fixed_point_is_discrete_helmholtz(n):
    """eq. discreteHelmholtz: the direct solution U satisfies Pi(U) = U and Pi(Pi(U)) = U."""
    p = _problem((n, n), [5.5, 9.3])
    U = W.helmholtz_direct(p)
    PU = W.apply_Pi(p, U)
    scale = np.max(np.abs(U))
    assert np.max(np.abs(PU - U)) / scale < 1e-12
    assert np.max(np.abs(W.apply_Pi(p, PU) - U)) / scale < 1e-12


def test_fixed_point_3d_two_layer():
    """Same invariant in 3D with the non-divergence two-layer operator c^2 Delta_h."""
    dims = (8, 8, 8)
    c2 = inputs.two_layer_c2(dims, (1.0, 1.0, 1.0), 1.0, 1.5, 0.5)
    p = _problem(dims, [4.1, 7.9, 12.5], c2=c2, b=60.0)
    U = W.helmholtz_direct(p)
    PU = W.apply_Pi(p, U)
    assert np.max(np.abs(PU - U)) / np.max(np.abs(U)) < 1e-12


@pytest.mark.parametrize("dims", [(12, 10), (8, 7, 6)])
def test_fixed_point_with_random_c2_field(dims):
    """The same invariant with c^2 drawn independently at every grid point (c in [1, 1.5]):
    the sparse direct solution of (c_j^2 Delta_h + omega^2) U = f is the fixed point of the
    map, whose time step takes c_max from the field."""
    c2 = inputs.random_c2(dims, 21, 1.0, 1.5)
    p = _problem(dims, [4.1, 7.9, 12.5], c2=c2, b=60.0)
    U = W.helmholtz_direct(p)
    PU = W.apply_Pi(p, U)
    assert np.max(np.abs(PU - U)) / np.max(np.abs(U)) < 1e-12
    # a constant field (c^2 = 1.7) solves like the constant-speed problem: L_h scales by c^2
    pc = _problem(dims, [4.1, 7.9, 12.5], c2=np.full(c2.shape, 1.7), b=60.0)
    ps = _problem(dims, [4.1, 7.9, 12.5], c2=1.7, b=60.0)
    np.testing.assert_allclose(W.helmholtz_direct(pc), W.helmholtz_direct(ps), rtol=0, atol=1e-13)


def test_fixed_point_fails_with_unadjusted_B():
    """Planted mistake: building B with the unadjusted omega_j instead of omega~_j breaks
    the fixed point, so the invariant does test that reading."""
    p = _problem((16, 16), [5.5, 9.3])
    U = W.helmholtz_direct(p)
    s = p.setup
    s.B = F.filter_matrix(s.w, s.omega, s.dt)
    assert np.max(np.abs(W.apply_Pi(p, U) - U)) / np.max(np.abs(U)) > 1e-5


# ---------------------------------------------------------------------------
# Closed-form eigenmode recurrence
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [F.FILTER_OPTIMIZED, F.FILTER_TRADITIONAL])
def test_eigenmode_closed_form_2d(mode):
    p0 = _problem((20, 24), [5.5, 9.3, 13.1], mode=mode, length=(1.0, 1.2))
    g = p0.grid
    rng = np.random.default_rng(5)
    for k in [(1, 1), (2, 3), (7, 2), (19, 23)]:
        phi, lam2 = W.dirichlet_mode(g, k)
        a = rng.normal(size=3)
        v = rng.normal(size=3)
        p = W.make_problem(g, p0.setup.omega, a[:, None, None] * phi, filter_mode=mode)
        got = W.apply_Pi(p, v[:, None, None] * phi)
        want = _closed_form_Pi(p.setup, lam2, a, v)
        np.testing.assert_allclose(got, want[:, None, None] * phi, atol=1e-12 * max(1.0, np.max(np.abs(want))))


def test_eigenmode_superposition_3d():
    """A sum of modes in 3D with different coefficients per mode and frequency."""
    g = W.Grid((6, 7, 8), (1.0, 1.0, 1.0))
    omega = np.array([4.0, 9.5])
    rng = np.random.default_rng(9)
    modes = [(1, 1, 1), (2, 5, 3), (5, 6, 7)]
    f = np.zeros((2,) + g.shape)
    V = np.zeros_like(f)
    want = np.zeros_like(f)
    coeffs = []
    for k in modes:
        phi, lam2 = W.dirichlet_mode(g, k)
        a, v = rng.normal(size=2), rng.normal(size=2)
        f += a[:, None, None, None] * phi
        V += v[:, None, None, None] * phi
        coeffs.append((phi, lam2, a, v))
    p = W.make_problem(g, omega, f)
    for phi, lam2, a, v in coeffs:
        want += _closed_form_Pi(p.setup, lam2, a, v)[:, None, None, None] * phi
    np.testing.assert_allclose(W.apply_Pi(p, V), want, atol=1e-12)


def test_closed_form_catches_dropped_half_in_first_step(monkeypatch):
    """Planted mistake: a first step without the factor 1/2 (eq. implicitFirstStep)
    is caught by the eigenmode pin."""
    g = W.Grid((12, 12), (1.0, 1.0))
    phi, lam2 = W.dirichlet_mode(g, (2, 1))
    a, v = np.array([1.0, -0.5]), np.array([0.3, 0.8])
    p = W.make_problem(g, [5.5, 9.3], a[:, None, None] * phi)
    want = _closed_form_Pi(p.setup, lam2, a, v)[:, None, None] * phi
    good = W.apply_Pi(p, v[:, None, None] * phi)
    assert np.max(np.abs(good - want)) < 1e-12
    orig = W.laplacian
    calls = {"n": 0}

    def doubled_first(Wg, grid, c2, order=2):   # doubles L_h only on its first call (W^1)
        calls["n"] += 1
        return orig(Wg, grid, c2, order) * (2.0 if calls["n"] == 1 else 1.0)

    monkeypatch.setattr(W, "laplacian", doubled_first)
    bad = W.apply_Pi(p, v[:, None, None] * phi)
    assert np.max(np.abs(bad - want)) > 1e-4


# ---------------------------------------------------------------------------
# Linearity and the spectrum of S
# ---------------------------------------------------------------------------

def test_affine_structure():
    """eq. discreteMFWHmapping: Pi(V) = S V + b with S linear and b = Pi(0)."""
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


def _dense_S(p):
    inner = p.grid.interior()
    idx = [(m,) + tuple(j) for m in range(p.nf)
           for j in np.ndindex(*[s - 2 for s in p.grid.shape])]
    N = len(idx)
    S = np.zeros((N, N))
    for c, (m, *j) in enumerate(idx):
        e = np.zeros_like(p.forcing)
        e[(m,) + tuple(k + 1 for k in j)] = 1.0
        col = W.apply_Pi(p, e, forced=False)
        S[:, c] = col[(slice(None),) + inner].reshape(-1)
    return S


def test_spectrum_of_S_is_mu_d():
    """Theorems 1-2 at the discrete level: S acts on each Dirichlet mode as the rank-one
    B^{-1} C, so its eigenvalues are mu_d(lambda~_nu) over the modes plus zeros, where
    cos(lambda~ dt) = 1 - lambda_h^2 dt^2 / 2 (the adjusted eigenvalues of Section
    'Numerical results')."""
    p = _problem((6, 7), [5.5, 9.3], mode=F.FILTER_TRADITIONAL)
    s = p.setup
    S = _dense_S(p)
    ev = np.linalg.eigvals(S)
    lam_t = []
    for kx in range(1, 6):
        for ky in range(1, 7):
            _, lam2 = W.dirichlet_mode(p.grid, (kx, ky))
            lam_t.append(math.acos(1.0 - 0.5 * lam2 * s.dt ** 2) / s.dt)
    mu = F.mu_discrete(s.B, s.w, np.array(lam_t), s.dt)
    want = np.sort(np.concatenate([mu, np.zeros(len(mu))]).real)
    got = np.sort(ev.real)
    np.testing.assert_allclose(got, want, atol=1e-10)
    assert np.max(np.abs(ev.imag)) < 1e-10


def test_resonant_frequency_leaves_a_unit_eigenvalue():
    """A frequency at a discrete eigenvalue, omega_1 = lambda_h of the (1, 1) Dirichlet mode,
    makes the discrete Helmholtz operator singular.  At the MFWH level the mode's adjusted
    eigenvalue equals omega~_1 (the same map sends lambda_h to lambda~ and omega_1 to
    omega~_1), and mu_d(omega~_1) = 1 (Theorem 3, constraints eq. constraintsT), so S has the
    eigenvalue 1 and A = I - S is singular: the fixed-point system has no unique solution.
    Moving omega_1 off the eigenvalue by 1 % keeps every eigenvalue of S away from 1."""
    g = W.Grid((6, 6), (1.0, 1.0))
    _, lam2 = W.dirichlet_mode(g, (1, 1))
    for shift, resonant in ((1.0, True), (1.01, False)):
        omega = [math.sqrt(lam2) * shift, 9.3]
        wl = inputs.gaussian_workload("t", (6, 6), 2, omega, 200.0, 11)
        p = W.make_problem(g, omega, wl.forcing, filter_mode=F.FILTER_TRADITIONAL)
        gap = np.min(np.abs(np.linalg.eigvals(_dense_S(p)) - 1.0))
        if resonant:
            assert gap < 1e-9, gap
        else:
            assert gap > 1e-3, gap


# ---------------------------------------------------------------------------
# GMRES, FPI rate and the residual
# ---------------------------------------------------------------------------

def test_gmres_matches_dense_and_direct():
    p = _problem((9, 9), [5.5, 9.3])
    S = _dense_S(p)
    inner = (slice(None),) + p.grid.interior()
    b = W.apply_Pi(p, np.zeros_like(p.forcing))
    x_dense = np.linalg.solve(np.eye(S.shape[0]) - S, b[inner].reshape(-1))
    x, info = W.gmres(p, restart=10, tol=1e-13, max_iters=400)
    assert info.converged
    np.testing.assert_allclose(x[inner].reshape(-1), x_dense, atol=1e-10 * np.max(np.abs(x_dense)))
    U = W.helmholtz_direct(p)
    assert np.max(np.abs(x - U)) < 1e-9 * np.max(np.abs(U))
    assert np.max(W.helmholtz_residual(p, x)) < 1e-9


def test_fpi_residual_definition():
    """eq. residual: (r^{(k)})^2 is the sum of squared changes over the N_f frequencies and the
    N_a points of Omega_h (the interior points), divided by N_f N_a.  Worked cases on a 6 x 5
    grid (20 interior points) with N_f = 2: one interior change of 3 gives 3 / sqrt(40); the
    same change c everywhere in the interior gives |c|; changes on boundary points do not
    count."""
    g = W.Grid((6, 5), (1.0, 1.0))
    old = np.zeros((2,) + g.shape)
    new = old.copy()
    new[1, 2, 3] = 3.0
    assert abs(W.fpi_residual(new, old, g) - 3.0 / math.sqrt(40.0)) < 1e-15
    new = old.copy()
    new[(slice(None),) + g.interior()] = -0.25
    assert abs(W.fpi_residual(new, old, g) - 0.25) < 1e-15
    new[:, 0, :] = 7.0
    new[:, :, -1] = -5.0
    assert abs(W.fpi_residual(new, old, g) - 0.25) < 1e-15


def test_gmres_starts_from_the_initial_guess():
    """GMRES from V0 iterates on the residual b - A V0: started at the fixed point U (the
    direct Helmholtz solution, for which A U = b) it stops before any Arnoldi step and returns
    U; started at U / 2 (residual b / 2) its first step stays below the initial relative
    residual 1/2, and it reaches U."""
    p = _problem((9, 9), [5.5, 9.3])
    U = W.helmholtz_direct(p)
    x, info = W.gmres(p, V0=U, restart=10, tol=1e-8, max_iters=50)
    assert info.converged and info.iterations == 0
    assert np.max(np.abs(x - U)) == 0.0
    x, info = W.gmres(p, V0=0.5 * U, restart=10, tol=1e-8, max_iters=1)
    assert info.iterations == 1 and info.history[0] < 0.5 + 1e-12   # GMRES never increases it
    x, info = W.gmres(p, V0=0.5 * U, restart=10, tol=1e-13, max_iters=400)
    assert info.converged
    assert np.max(np.abs(x - U)) < 1e-9 * np.max(np.abs(U))


def test_gmres_full_krylov_is_exact():
    """Without restarts GMRES terminates with the exact solution after at most dim steps."""
    p = _problem((5, 5), [5.5, 9.3])
    x, info = W.gmres(p, restart=40, tol=1e-14, max_iters=40)
    U = W.helmholtz_direct(p)
    assert info.iterations <= 32
    assert np.max(np.abs(x - U)) < 1e-10 * np.max(np.abs(U))


def test_fpi_rate_matches_acr():
    """Theorem 1: the asymptotic FPI rate equals max over modes of |mu_d(lambda~)|."""
    p = _problem((12, 12), [5.5, 9.3])
    s = p.setup
    lam_t = []
    for kx in range(1, 12):
        for ky in range(1, 12):
            _, lam2 = W.dirichlet_mode(p.grid, (kx, ky))
            lam_t.append(math.acos(1.0 - 0.5 * lam2 * s.dt ** 2) / s.dt)
    acr = np.max(np.abs(F.mu_discrete(s.B, s.w, np.array(lam_t), s.dt)))
    its = W.fixed_point_iteration(p, np.zeros_like(p.forcing), 160)
    r = [W.fpi_residual(its[k], its[k - 1], p.grid) for k in range(1, len(its))]
    rate = (r[-1] / r[-41]) ** (1.0 / 40)
    assert abs(rate - acr) < 0.01 * acr


def test_residual_of_exact_solution_and_zero():
    p = _problem((16, 16), [5.5, 9.3])
    U = W.helmholtz_direct(p)
    assert np.max(W.helmholtz_residual(p, U)) < 1e-12
    np.testing.assert_allclose(W.helmholtz_residual(p, np.zeros_like(U)), 1.0)


def test_laplacian_brute_force():
    """L_h against an explicit loop over interior points (2D and 3D, variable c^2)."""
    rng = np.random.default_rng(4)
    g = W.Grid((5, 6), (1.0, 1.3))
    A = rng.normal(size=g.shape)
    c2 = rng.uniform(0.5, 2.0, size=g.shape)
    hx, hy = g.h
    want = np.zeros_like(A)
    for j in range(1, g.shape[0] - 1):
        for i in range(1, g.shape[1] - 1):
            want[j, i] = c2[j, i] * ((A[j, i + 1] - 2 * A[j, i] + A[j, i - 1]) / hx ** 2
                                     + (A[j + 1, i] - 2 * A[j, i] + A[j - 1, i]) / hy ** 2)
    np.testing.assert_allclose(W.laplacian(A, g, c2), want, atol=1e-10)
    g3 = W.Grid((4, 3, 5), (1.0, 1.0, 2.0))
    A3 = rng.normal(size=g3.shape)
    hx, hy, hz = g3.h
    want3 = np.zeros_like(A3)
    for k in range(1, g3.shape[0] - 1):
        for j in range(1, g3.shape[1] - 1):
            for i in range(1, g3.shape[2] - 1):
                want3[k, j, i] = ((A3[k, j, i + 1] - 2 * A3[k, j, i] + A3[k, j, i - 1]) / hx ** 2
                                  + (A3[k, j + 1, i] - 2 * A3[k, j, i] + A3[k, j - 1, i]) / hy ** 2
                                  + (A3[k + 1, j, i] - 2 * A3[k, j, i] + A3[k - 1, j, i]) / hz ** 2)
    np.testing.assert_allclose(W.laplacian(A3, g3, 1.0), want3, atol=1e-10)
    # the sparse matrix used by the direct solve is the same operator
    L = W.laplacian_matrix(g, c2)
    np.testing.assert_allclose(L @ A[1:-1, 1:-1].ravel() - (W.laplacian(A, g, c2)[1:-1, 1:-1].ravel()
                               - _boundary_contrib(A, g, c2)), 0.0, atol=1e-9)


def _boundary_contrib(A, g, c2):
    """Part of L_h A at interior points that comes from boundary values of A."""
    B = np.zeros_like(A)
    B[0, :], B[-1, :], B[:, 0], B[:, -1] = A[0, :], A[-1, :], A[:, 0], A[:, -1]
    return W.laplacian(B, g, c2)[1:-1, 1:-1].ravel()


def test_small_config_fpi_trajectory_is_finite():
    """The 65^2, N_f = 2 workload: 40 fixed-point iterations run, the iterates stay finite and
    the fixed-point residual decays at no more than the predicted rate bound."""
    wl = inputs.square_small()
    g = W.Grid(wl.n, wl.length)
    p = W.make_problem(g, wl.omega, wl.forcing)
    assert p.setup.n_t == 207
    its = W.fixed_point_iteration(p, np.zeros_like(wl.forcing), 40)
    assert all(np.all(np.isfinite(v)) for v in its)
    r = [W.fpi_residual(its[k], its[k - 1], g) for k in range(1, 40)]
    assert r[-1] < r[0]
