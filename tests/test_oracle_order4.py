"""Pins for the oracle's fourth-order spatial operator L_{4h} (the p = 4 case of
L_{ph}, Section "Discretizing the wave equation and filter") with odd-reflection
ghost values for homogeneous Dirichlet data: brute force, the convergence order,
the closed-form Dirichlet spectrum, the leapfrog stability bound behind the time
step, the fixed point of the MFWH map and the closed-form eigenmode recurrence,
and the set-up of the paper's explicit three-frequency fourth-order example.  CPU only."""

import math

import numpy as np
import pytest

from oracle import filters as F
from oracle import wave as W
from paper_2507_23613_gb300 import inputs


def _ghost(A, j, n):
    """Value at index j along an axis with n cells: odd reflection outside 0..n."""
    return A(j) if 0 <= j <= n else (-A(-j) if j < 0 else -A(2 * n - j))


def test_order4_laplacian_brute_force_2d_and_3d():
    rng = np.random.default_rng(41)
    g = W.Grid((6, 7), (1.0, 1.4))
    A = rng.normal(size=g.shape)
    W.zero_boundary(A, g)
    c2 = rng.uniform(0.5, 2.0, size=g.shape)
    hx, hy = g.h
    nx, ny = g.n
    want = np.zeros_like(A)
    for j in range(1, ny):
        for i in range(1, nx):
            ax = lambda t: _ghost(lambda q: A[j, q], t, nx)
            ay = lambda t: _ghost(lambda q: A[q, i], t, ny)
            dxx = (-ax(i - 2) + 16 * ax(i - 1) - 30 * ax(i) + 16 * ax(i + 1) - ax(i + 2)) / (12 * hx * hx)
            dyy = (-ay(j - 2) + 16 * ay(j - 1) - 30 * ay(j) + 16 * ay(j + 1) - ay(j + 2)) / (12 * hy * hy)
            want[j, i] = c2[j, i] * (dxx + dyy)
    np.testing.assert_allclose(W.laplacian(A, g, c2, order=4), want, atol=1e-9)
    g3 = W.Grid((4, 3, 5), (1.0, 1.0, 2.0))
    B = rng.normal(size=g3.shape)
    W.zero_boundary(B, g3)
    h = g3.h
    n = g3.n
    want3 = np.zeros_like(B)
    for k in range(1, n[2]):
        for j in range(1, n[1]):
            for i in range(1, n[0]):
                lines = [lambda t: _ghost(lambda q: B[k, j, q], t, n[0]),
                         lambda t: _ghost(lambda q: B[k, q, i], t, n[1]),
                         lambda t: _ghost(lambda q: B[q, j, i], t, n[2])]
                idx = (i, j, k)
                acc = 0.0
                for a in range(3):
                    f, c = lines[a], idx[a]
                    acc += (-f(c - 2) + 16 * f(c - 1) - 30 * f(c) + 16 * f(c + 1) - f(c + 2)) / (12 * h[a] ** 2)
                want3[k, j, i] = acc
    np.testing.assert_allclose(W.laplacian(B, g3, 1.0, order=4), want3, atol=1e-9)
    # the sparse matrix of the direct solve is the same operator (interior values only)
    for grid, arr, cc in ((g, A, c2), (g3, B, 1.0)):
        L = W.laplacian_matrix(grid, cc, order=4)
        inner = grid.interior()
        np.testing.assert_allclose(L @ arr[inner].ravel(),
                                   W.laplacian(arr, grid, cc, order=4)[inner].ravel(), atol=1e-9)


def test_order4_laplacian_is_fourth_order_accurate():
    """On u = sin(pi x) sin(2 pi y) (odd about every boundary, so the ghost values are
    exact) the error of L_4h u against -5 pi^2 u falls 16-fold when h halves; L_2h's
    falls 4-fold."""
    errs = {2: [], 4: []}
    for n in (16, 32, 64):
        g = W.Grid((n, n), (1.0, 1.0))
        x, y = g.coords()
        u = np.sin(math.pi * x) * np.sin(2 * math.pi * y)
        exact = -5.0 * math.pi ** 2 * u
        inner = g.interior()
        for order in (2, 4):
            errs[order].append(np.max(np.abs(W.laplacian(u, g, 1.0, order)[inner] - exact[inner])))
    r4 = [errs[4][i] / errs[4][i + 1] for i in range(2)]
    r2 = [errs[2][i] / errs[2][i + 1] for i in range(2)]
    assert all(15.0 < r < 16.5 for r in r4), r4
    assert all(3.9 < r < 4.1 for r in r2), r2


@pytest.mark.parametrize("k", [(1, 1), (3, 2), (9, 11), (15, 13)])
def test_order4_dirichlet_spectrum(k):
    g = W.Grid((16, 14), (1.0, 0.8))
    phi, lam2 = W.dirichlet_mode(g, k, order=4)
    inner = g.interior()
    np.testing.assert_allclose(W.laplacian(phi, g, 1.0, order=4)[inner], -lam2 * phi[inner],
                               atol=1e-10 * lam2)
    # and it differs from the second-order eigenvalue (except in the limit of small k h)
    _, lam2_2 = W.dirichlet_mode(g, k, order=2)
    assert lam2 > lam2_2


def test_order4_time_step_is_the_leapfrog_stability_limit():
    """dt_stab(order 4) = sqrt(3)/2 dt_stab(order 2).  Leapfrog on the highest Dirichlet
    mode stays bounded just below dt_stab and grows just above it."""
    n = 24
    g = W.Grid((n, n), (1.0, 1.0))
    dt2, _ = F.explicit_time_step(g.h, 1.0, 1.0, 1.0, 1, order=2)
    dt4, _ = F.explicit_time_step(g.h, 1.0, 1.0, 1.0, 1, order=4)
    h = 1.0 / n
    stab2 = 1.0 / math.sqrt(2.0 / h ** 2)
    stab4 = stab2 * math.sqrt(3.0) / 2.0
    phi, lam2 = W.dirichlet_mode(g, (n - 1, n - 1), order=4)
    for dt, grows in ((stab4 * 0.999, False), (stab4 * 1.02, True)):
        w_prev, w = phi.copy(), phi.copy()
        for _ in range(400):
            w_prev, w = w, 2 * w - w_prev + dt * dt * W.laplacian(w, g, 1.0, order=4)
        amp = np.max(np.abs(w))
        assert (amp > 1e3) == grows, (dt / stab4, amp)
    # the explicit step chosen for a problem respects the bound (cfl = 1 gives dt <= stab)
    assert dt4 <= stab4 * (1 + 1e-12) and dt2 <= stab2 * (1 + 1e-12)


@pytest.mark.parametrize("dims", [(8, 8), (12, 10), (6, 5, 7)])
def test_order4_fixed_point_is_discrete_helmholtz(dims):
    om = [5.5, 9.3] if len(dims) == 2 else [6.0, 9.0]
    wl = inputs.gaussian_workload("o4", dims, len(om), om, 120.0, 7)
    g = W.Grid(dims, wl.length)
    p = W.make_problem(g, om, wl.forcing, order=4)
    U = W.helmholtz_direct(p)
    np.testing.assert_allclose(W.apply_Pi(p, U), U, atol=1e-12 * np.max(np.abs(U)))
    assert np.max(W.helmholtz_residual(p, U)) < 1e-12
    # with the second-order map the fourth-order solution is not a fixed point
    p2 = W.make_problem(g, om, wl.forcing, order=2)
    assert np.max(np.abs(W.apply_Pi(p2, U) - U)) > 1e-6 * np.max(np.abs(U))


def test_order4_eigenmode_closed_form():
    """The Chebyshev closed form of one Pi application on a Dirichlet mode (as for order 2)
    with the fourth-order eigenvalue."""
    g = W.Grid((18, 16), (1.0, 1.0))
    om = np.array([5.5, 9.3, 13.1])
    rng = np.random.default_rng(8)
    for k in [(1, 2), (5, 3), (17, 15)]:
        phi, lam2 = W.dirichlet_mode(g, k, order=4)
        a = rng.normal(size=3)
        v = rng.normal(size=3)
        p = W.make_problem(g, om, a[:, None, None] * phi, order=4,
                           filter_mode=F.FILTER_TRADITIONAL)
        s = p.setup
        u = a / (s.omega ** 2 - lam2)
        x = 1.0 - 0.5 * lam2 * s.dt ** 2
        nn = np.arange(s.n_t + 1)
        W_hat = np.cos(nn * np.arccos(x)) * np.sum(v - u) + np.cos(np.outer(nn * s.dt, s.omega_t)) @ u
        want = np.linalg.solve(s.B, s.w.T @ W_hat)
        got = W.apply_Pi(p, v[:, None, None] * phi)
        np.testing.assert_allclose(got, want[:, None, None] * phi,
                                   atol=1e-12 * max(1.0, np.max(np.abs(want))))


def test_paper_three_frequency_fourth_order_setup():
    """The explicit example with omega = {5.1, 10.1, 15.1}, N_p = 2 on a 128^2 square
    (Figure multiFreq3SquareNp2Exp) has N_{p,m} = {2, 3, 5} (its caption)."""
    g = W.Grid((128, 128), (1.0, 1.0))
    s = F.make_setup([5.1, 10.1, 15.1], g.h, 1.0, 0.5, 2, F.FILTER_TRADITIONAL, order=4)
    assert list(s.n_pm) == [2, 3, 5]
    dt_stab = math.sqrt(3.0) / 2.0 / math.sqrt(2.0 * 128.0 ** 2)
    assert s.dt < 0.5 * dt_stab * (1 + 1e-12)
