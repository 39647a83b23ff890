"""Pins for the oracle's explicit-filter variant of the MFWH update (footnote to
eq. filterII: v^{(j,k)} in place of v^{(j,k+1)} in the sum, i.e.
B_mm V_m^{k+1} = q_m - sum_{j != m} B_mj V_j^k): the discrete Helmholtz solution is
still the fixed point, one application on a Dirichlet mode follows the closed form,
and GMRES on the explicit map reaches the same solution.  CPU only."""

import numpy as np
import pytest

from oracle import filters as F
from oracle import wave as W
from paper_2507_23613_gb300 import inputs


def _problem(explicit, mode=F.FILTER_OPTIMIZED, dims=(16, 14)):
    wl = inputs.gaussian_workload("ef", dims, 3, [5.5, 9.3, 13.1], 200.0, 11)
    g = W.Grid(dims, wl.length)
    return W.make_problem(g, wl.omega, wl.forcing, filter_mode=mode, explicit_filter=explicit)


@pytest.mark.parametrize("mode", [F.FILTER_OPTIMIZED, F.FILTER_TRADITIONAL])
def test_explicit_filter_fixed_point(mode):
    p = _problem(True, mode)
    U = W.helmholtz_direct(p)
    np.testing.assert_allclose(W.apply_Pi(p, U), U, atol=1e-12 * np.max(np.abs(U)))
    # away from the fixed point the explicit and implicit maps differ
    V = 0.5 * U
    pi = _problem(False, mode)
    assert np.max(np.abs(W.apply_Pi(p, V) - W.apply_Pi(pi, V))) > 1e-3 * np.max(np.abs(U))


def test_explicit_filter_eigenmode_closed_form():
    g = W.Grid((18, 16), (1.0, 1.0))
    om = np.array([5.5, 9.3, 13.1])
    rng = np.random.default_rng(9)
    for k in [(1, 1), (4, 2), (17, 15)]:
        phi, lam2 = W.dirichlet_mode(g, k)
        a = rng.normal(size=3)
        v = rng.normal(size=3)
        p = W.make_problem(g, om, a[:, None, None] * phi, explicit_filter=True)
        s = p.setup
        u = a / (s.omega ** 2 - lam2)
        x = 1.0 - 0.5 * lam2 * s.dt ** 2
        n = np.arange(s.n_t + 1)
        W_hat = np.cos(n * np.arccos(x)) * np.sum(v - u) + np.cos(np.outer(n * s.dt, s.omega_t)) @ u
        q = s.w.T @ W_hat
        off = s.B - np.diag(np.diag(s.B))
        want = (q - off @ v) / np.diag(s.B)
        got = W.apply_Pi(p, v[:, None, None] * phi)
        np.testing.assert_allclose(got, want[:, None, None] * phi,
                                   atol=1e-12 * max(1.0, np.max(np.abs(want))))


def test_explicit_filter_gmres_reaches_direct_solution():
    p = _problem(True, dims=(12, 10))
    U = W.helmholtz_direct(p)
    V, info = W.gmres(p, restart=200, tol=1e-12, max_iters=200)
    assert info.converged and info.rel_residual < 1e-12
    np.testing.assert_allclose(V, U, atol=1e-9 * np.max(np.abs(U)))
