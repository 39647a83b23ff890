"""GPU parity: libmfwh (through its C ABI) against the FP64 oracle, element by
element on seeded inputs, plus full-size property checks in the benchmark's
launch configuration.  Tolerance: 1e-10 relative (max norm, per frequency)
for FP64 results."""

import math

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs
from oracle import filters as F
from oracle import wave as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10
EPS = np.finfo(np.float64).eps


def opt_tol(prob):
    """Parity bound for maps built on least-squares filter parameters.

    Algorithm 2's least-squares problem has a non-zero residual, so its solution
    is determined only to about eps * cond(M)^2; two correct solvers (the oracle's
    and the library's) differ by that much, and Pi inherits the difference.
    Parameters given as inputs (traditional or user) are held to TOL.
    """
    cm = prob.setup.cond_M
    return TOL if not np.isfinite(cm) else max(TOL, 10.0 * EPS * cm * cm)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, want):
    """max_j |got - want| / max_j |want| for each frequency m."""
    got = np.asarray(got).reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    scale = np.maximum(np.max(np.abs(want), axis=1), 1e-300)
    return np.max(np.abs(got - want), axis=1) / scale


def make_pair(wl, c_hi=None, mode=0, user=None):
    kw = {"n_p": wl.n_p, "cfl": wl.cfl, "filter_mode": mode, "user_params": user}
    c2 = 1.0
    if c_hi is not None:
        kw.update(c_lo=1.0, c_hi=c_hi, interface=0.5, layer_axis=len(wl.n) - 1)
        c2 = inputs.two_layer_c2(wl.n, wl.length, 1.0, c_hi, 0.5)
    solver = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), **kw)
    fm = {0: F.FILTER_OPTIMIZED, 1: F.FILTER_TRADITIONAL, 2: F.FILTER_USER}[mode]
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=fm, user_params=user)
    return solver, prob


def random_v(wl, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=wl.forcing.shape) * 0.01
    g = W.Grid(wl.n, wl.length)
    for m in range(v.shape[0]):
        W.zero_boundary(v[m], g)
    return v


def check_pi(solver, prob, v, forced, tol=None):
    tol = opt_tol(prob) if tol is None else tol
    out = torch.empty(v.shape, dtype=torch.float64, device="cuda")
    solver.apply_Pi(dev(v), out, forced=forced)
    torch.cuda.synchronize()
    want = W.apply_Pi(prob, v, forced=forced)
    err = rel_err(out.cpu().numpy(), want)
    assert np.all(err <= tol), (err, tol)
    return err


# ---------------------------------------------------------------------------
# One application of Pi
# ---------------------------------------------------------------------------

def test_pi_small_square_forced_and_homogeneous():
    wl = inputs.square_small()
    solver, prob = make_pair(wl)
    assert solver.setup["n_t"] == prob.setup.n_t == 207
    check_pi(solver, prob, random_v(wl, 1), forced=True)
    check_pi(solver, prob, random_v(wl, 2), forced=False)
    check_pi(solver, prob, np.zeros_like(wl.forcing), forced=True)


def _ragged_nf8():
    wl = inputs.gaussian_workload("ragged", (70, 45), 8,
                                  lambda r: inputs.draw_frequencies(r, 8, 10.0, 60.0), 400.0, 77,
                                  length=(1.3, 0.9))
    wl.n_p = 2
    return wl


@pytest.mark.parametrize("mode", [1, 2])
def test_pi_ragged_rectangle_nf8(mode):
    """70 x 45 cells (tiles of 32 x 8 with ragged edges), lengths 1.3 x 0.9, N_f = 8,
    traditional or seeded user filter parameters (the same inputs on both sides)."""
    wl = _ragged_nf8()
    user = inputs.random_filter_params(501, 8) if mode == 2 else None
    solver, prob = make_pair(wl, mode=mode, user=user)
    check_pi(solver, prob, random_v(wl, 3), forced=True)
    check_pi(solver, prob, random_v(wl, 4), forced=False)


def test_pi_ragged_rectangle_nf8_optimised():
    """Same grid with each side's own least-squares parameters (cond(M) ~ 6e4 here)."""
    wl = _ragged_nf8()
    solver, prob = make_pair(wl)
    check_pi(solver, prob, random_v(wl, 3), forced=True, tol=opt_tol(prob))


@pytest.mark.parametrize("mode", [1, 2])
def test_pi_traditional_and_user_filters(mode):
    wl = inputs.gaussian_workload("t", (40, 33), 3, [6.1, 9.7, 15.2], 200.0, 12)
    user = np.array([[-0.25, 1.0, 0.05], [0.2, 0.8, -0.1], [-0.1, 1.1, 0.0]]) if mode == 2 else None
    solver, prob = make_pair(wl, mode=mode, user=user)
    check_pi(solver, prob, random_v(wl, 5), forced=True)


def test_pi_3d_two_layer():
    wl = inputs.gaussian_workload("cube", (20, 18, 16), 4, [8.3, 12.1, 19.0, 27.5], 300.0, 21)
    solver, prob = make_pair(wl, c_hi=1.5)
    check_pi(solver, prob, random_v(wl, 6), forced=True)
    check_pi(solver, prob, random_v(wl, 7), forced=False)


@pytest.mark.parametrize("nf", [1, 16])
def test_pi_extreme_frequency_counts(nf):
    om = np.linspace(5.0, 5.0 + 3.0 * (nf - 1), nf)
    wl = inputs.gaussian_workload("nf", (33, 31), nf, om, 150.0, 30 + nf)
    wl.n_p = 2 if nf > 1 else 1
    solver, prob = make_pair(wl)
    check_pi(solver, prob, random_v(wl, 8), forced=True)


def test_pi_single_interior_point():
    """n = 2 cells per axis: one interior point, the smallest grid."""
    wl = inputs.gaussian_workload("tiny", (2, 2), 2, [3.0, 5.0], 5.0, 1)
    solver, prob = make_pair(wl)
    check_pi(solver, prob, random_v(wl, 9), forced=True)


def test_pi_in_place():
    wl = inputs.square_small()
    solver, prob = make_pair(wl)
    v = random_v(wl, 10)
    buf = dev(v)
    solver.apply_Pi(buf, buf, forced=True)
    torch.cuda.synchronize()
    assert np.all(rel_err(buf.cpu().numpy(), W.apply_Pi(prob, v)) <= opt_tol(prob))


@pytest.mark.parametrize("shape,nf,seed,layer", [((70, 45), 8, 77, None), ((40, 33), 16, 31, None),
                                                  ((64, 64), 2, 5, None), ((2, 2), 2, 1, None),
                                                  ((200, 170), 4, 9, None),
                                                  ((150, 140), 3, 10, 0), ((130, 160), 3, 11, 1)])
def test_time_blocking_is_bit_identical(shape, nf, seed, layer):
    """Temporal blocking (2, 3, 4 or 8 leapfrog steps per pass over HBM, halo tiles in shared
    memory, tiles of 32 x 64, 32 x 48, 32 x 32 and 32 x 16 points, one to four rows per thread,
    CTAs of 512 or 256 threads, and persistent CTAs that copy the next tile while stepping one)
    performs
    the same floating-point operations per point as one step per launch, so Pi, S and the
    GMRES iterate are bit-identical for every depth and tile; also checked against the
    oracle.  N_t is not a
    multiple of the depth on these grids (ragged last launch); the larger grids have CTAs whose
    whole halo is interior (the kernels' test-free path) and two-layer media split along x or
    y (c = 1 and 1.4 on either side of 0.37 of the length)."""
    om = np.linspace(6.0, 6.0 + 2.5 * (nf - 1), nf)
    wl = inputs.gaussian_workload("tb", shape, nf, om, 150.0, seed)
    wl.n_p = 2 if nf > 2 else 1
    v = random_v(wl, seed + 1)
    kw = {} if layer is None else dict(c_lo=1.0, c_hi=1.4, interface=0.37, layer_axis=layer)
    outs = {}
    for tb, tshape in ((1, 0), (2, 4), (2, 1), (2, 5), (3, 4), (3, 1), (3, 5), (4, 0), (4, 1),
                       (4, 2), (4, 3), (4, 4), (4, 5), (8, 0), (8, 1), (8, 2), (8, 3)):
        solver = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                          filter_mode=_lib.FILTER_TRADITIONAL, time_block=tb, tile_shape=tshape,
                          **kw)
        res = []
        for forced in (True, False):
            out = torch.empty(v.shape, dtype=torch.float64, device="cuda")
            solver.apply_Pi(dev(v), out, forced=forced)
            res.append(out.cpu().numpy())
        x = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
        solver.solve_gmres(x, restart=5, tol=0.0, max_iters=7, raise_on_error=False)
        res.append(x.cpu().numpy())
        outs[(tb, tshape)] = res
        solver.close()
    for key, got in outs.items():
        for a, b in zip(got, outs[(1, 0)]):
            assert np.array_equal(a, b), (key, np.max(np.abs(a - b)))
    c2 = 1.0
    if layer is not None:
        x = np.meshgrid(*[np.arange(n + 1) / n * L for n, L in zip(reversed(wl.n),
                                                                   reversed(wl.length))],
                        indexing="ij")
        coord = x[1] if layer == 0 else x[0]
        c2 = np.where(coord < 0.37, 1.0, 1.4 ** 2)
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=F.FILTER_TRADITIONAL)
    assert np.all(rel_err(outs[(8, 0)][0], W.apply_Pi(prob, v, forced=True)) <= TOL)
    assert np.all(rel_err(outs[(8, 0)][1], W.apply_Pi(prob, v, forced=False)) <= TOL)


# ---------------------------------------------------------------------------
# Iterations and the residual
# ---------------------------------------------------------------------------

def test_fpi_trajectory_small_square():
    """The 65^2 workload: 40 fixed-point iterations from zero, every iterate of the oracle
    trajectory checked at k = 1, 10, 20, 40."""
    wl = inputs.square_small()
    solver, prob = make_pair(wl)
    its = W.fixed_point_iteration(prob, np.zeros_like(wl.forcing), 40)
    v = np.zeros_like(wl.forcing)
    done = 0
    for k in (1, 10, 20, 40):
        solver.solve_fpi(v, k - done)
        done = k
        err = rel_err(v, its[k - 1])
        assert np.all(err <= opt_tol(prob)), (k, err)


def test_residual_parity():
    wl = inputs.gaussian_workload("t", (48, 40), 3, [6.1, 9.7, 15.2], 200.0, 13)
    solver, prob = make_pair(wl)
    for v in (random_v(wl, 11), W.helmholtz_direct(prob)):
        got = solver.residual(dev(v))
        want = W.helmholtz_residual(prob, v)
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-15)


def test_gmres_fixed_iterations_parity():
    """Same Krylov iterate after a fixed number of Arnoldi steps (tol = 0)."""
    wl = inputs.gaussian_workload("t", (33, 33), 3, [6.1, 9.7, 15.2], 200.0, 14)
    solver, prob = make_pair(wl)
    v = np.zeros_like(wl.forcing)
    info = solver.solve_gmres(v, restart=8, tol=0.0, max_iters=20, raise_on_error=False)
    assert info["status"] == _lib.ERR_NOT_CONVERGED and info["iterations"] == 20
    x, oinfo = W.gmres(prob, restart=8, tol=0.0, max_iters=20)
    assert oinfo.iterations == 20
    assert np.all(rel_err(v, x) <= max(1e-9, opt_tol(prob))), rel_err(v, x)
    np.testing.assert_allclose(info["history"], oinfo.history, rtol=1e-7)


def test_gmres_converges_to_discrete_helmholtz():
    wl = inputs.gaussian_workload("t", (33, 33), 3, [6.1, 9.7, 15.2], 200.0, 15)
    solver, prob = make_pair(wl)
    v = np.zeros_like(wl.forcing)
    info = solver.solve_gmres(v, restart=60, tol=1e-12, max_iters=400, spurious_tol=1e-8)
    U = W.helmholtz_direct(prob)
    assert np.all(rel_err(v, U) <= 1e-9), rel_err(v, U)
    np.testing.assert_allclose(info["helmholtz_residual"], W.helmholtz_residual(prob, v), rtol=1e-6, atol=1e-14)


def test_gmres_warm_start_from_solution():
    wl = inputs.gaussian_workload("t", (24, 24), 2, [5.5, 9.3], 200.0, 16)
    solver, prob = make_pair(wl)
    U = W.helmholtz_direct(prob)
    v = U.copy()
    info = solver.solve_gmres(v, restart=10, tol=1e-10, max_iters=50)
    assert info["iterations"] == 0
    assert np.all(rel_err(v, U) <= 1e-12)


def test_host_and_device_buffers_agree():
    wl = inputs.gaussian_workload("t", (40, 40), 2, [5.5, 9.3], 200.0, 17)
    solver, prob = make_pair(wl)
    vh = np.zeros_like(wl.forcing)
    solver.solve_gmres(vh, restart=10, tol=1e-9, max_iters=200)
    vd = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    solver.solve_gmres(vd, restart=10, tol=1e-9, max_iters=200)
    assert np.array_equal(vh, vd.cpu().numpy())


# ---------------------------------------------------------------------------
# Degenerate and invalid inputs
# ---------------------------------------------------------------------------

def test_zero_forcing_gives_zero_solution():
    wl = inputs.gaussian_workload("t", (20, 20), 2, [5.5, 9.3], 200.0, 18)
    wl.forcing[:] = 0.0
    solver, _ = make_pair(wl)
    v = np.ones_like(wl.forcing)
    info = solver.solve_gmres(v, restart=5, tol=1e-8, max_iters=10)
    assert np.all(v == 0.0) and info["iterations"] == 0


def test_nonfinite_forcing_is_reported():
    wl = inputs.gaussian_workload("t", (20, 20), 2, [5.5, 9.3], 200.0, 19)
    wl.forcing[0, 5, 5] = np.nan
    solver, _ = make_pair(wl)
    v = np.zeros_like(wl.forcing)
    info = solver.solve_gmres(v, restart=5, tol=1e-8, max_iters=10, raise_on_error=False)
    assert info["status"] == _lib.ERR_NONFINITE


def test_invalid_calls_are_rejected():
    wl = inputs.gaussian_workload("t", (20, 20), 2, [5.5, 9.3], 200.0, 20)
    solver, _ = make_pair(wl)
    host = np.zeros_like(wl.forcing)
    with pytest.raises(_lib.MfwhError) as e:
        solver.apply_Pi(host, host)
    assert e.value.status == _lib.ERR_INVALID_ARG
    with pytest.raises(_lib.MfwhError) as e:
        solver.solve_gmres(host, restart=0)
    assert e.value.status == _lib.ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# Full size (1025^2, N_f = 8, N_p = 2): properties that hold at any size
# ---------------------------------------------------------------------------

def _closed_form_Pi(s, lam2, a, v):
    u = a / (s.omega ** 2 - lam2)
    x = 1.0 - 0.5 * lam2 * s.dt ** 2
    n = np.arange(s.n_t + 1)
    cheb = np.cos(n * np.arccos(x))
    cosw = np.cos(np.outer(n * s.dt, s.omega_t))
    q = s.w.T @ (cheb * np.sum(v - u) + cosw @ u)
    return np.linalg.solve(s.B, q)


@pytest.mark.parametrize("mode", [0, 2])
def test_full_size_eigenmode_closed_form(mode):
    """At the benchmark size Pi maps a Dirichlet mode to the same mode with the
    coefficients of the closed-form recurrence (N_f x N_f algebra only), with the
    least-squares filter (mode 0) and with seeded user parameters (mode 2)."""
    wl = inputs.square_large()
    g = W.Grid(wl.n, wl.length)
    user = inputs.random_filter_params(502, wl.nf) if mode == 2 else None
    fm = F.FILTER_USER if mode == 2 else F.FILTER_OPTIMIZED
    setup = F.make_setup(wl.omega, g.h, 1.0, wl.cfl, wl.n_p, fm, user)
    tol = TOL if mode == 2 else max(TOL, 10.0 * EPS * setup.cond_M ** 2)
    rng = np.random.default_rng(44)
    for k in [(3, 5), (200, 17)]:
        phi, lam2 = W.dirichlet_mode(g, k)
        a = rng.normal(size=wl.nf)
        v = rng.normal(size=wl.nf)
        f = a[:, None, None] * phi
        solver = M.Solver(wl.n, wl.length, wl.omega, dev(f), n_p=wl.n_p, cfl=wl.cfl,
                          filter_mode=mode, user_params=user)
        assert solver.setup["n_t"] == setup.n_t
        out = torch.empty(f.shape, dtype=torch.float64, device="cuda")
        solver.apply_Pi(dev(v[:, None, None] * phi), out, forced=True)
        want = _closed_form_Pi(setup, lam2, a, v)[:, None, None] * phi
        err = rel_err(out.cpu().numpy(), want)
        assert np.all(err <= tol), (k, err, tol)
        solver.close()


@pytest.mark.parametrize("prec,tb,tol", [(_lib.PREC_FP64, 1, TOL),
                                         (_lib.PREC_FP32_KAHAN, 4, 3e-4)])
def test_full_size_3d_eigenmode_closed_form(prec, tb, tol):
    """The 257^3, N_f = 4 configuration (c = 1 so that Dirichlet modes are eigenfunctions):
    Pi maps a mode to the same mode with the closed-form coefficients, on the FP64 one-step
    kernel (to 1e-10) and on the FP32 blocked kernel at depth 4 (to the FP32 bound)."""
    wl = inputs.cube_layered()
    g = W.Grid(wl.n, wl.length)
    setup = F.make_setup(wl.omega, g.h, 1.0, wl.cfl, wl.n_p, F.FILTER_TRADITIONAL)
    rng = np.random.default_rng(45)
    phi, lam2 = W.dirichlet_mode(g, (5, 3, 7))
    a = rng.normal(size=wl.nf)
    v = rng.normal(size=wl.nf)
    f = a[:, None, None, None] * phi
    solver = M.Solver(wl.n, wl.length, wl.omega, dev(f), n_p=wl.n_p, cfl=wl.cfl,
                      filter_mode=1, precision=prec, time_block=tb)
    assert solver.setup["n_t"] == setup.n_t
    out = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    solver.apply_Pi(dev(v[:, None, None, None] * phi), out, forced=True)
    want = _closed_form_Pi(setup, lam2, a, v)[:, None, None, None] * phi
    err = rel_err(out.cpu().numpy(), want)
    assert np.all(err <= tol), (err, tol)
    solver.close()


def test_gmres_long_basis_parity():
    """No restart with a basis longer than one multi-dot launch handles (40 > 32 vectors)."""
    wl = inputs.gaussian_workload("t", (33, 33), 3, [6.1, 9.7, 15.2], 200.0, 15)
    solver, prob = make_pair(wl)
    v = np.zeros_like(wl.forcing)
    info = solver.solve_gmres(v, restart=100, tol=0.0, max_iters=40, raise_on_error=False)
    assert info["iterations"] == 40 and info["restarts"] == 1
    x, oinfo = W.gmres(prob, restart=100, tol=0.0, max_iters=40)
    assert np.all(rel_err(v, x) <= max(1e-9, opt_tol(prob))), rel_err(v, x)
    # The library's maps keep the filter sums as float pairs: a few 2^-48 relative per update,
    # at most about N_t 2^-46 of the sums per map.  The relative residuals of the history are
    # compared to that absolute level (about 1.4e-12 here; measured differences near 1e-14).
    np.testing.assert_allclose(info["history"], oinfo.history, rtol=1e-6,
                               atol=prob.setup.n_t * 2.0 ** -46)


def test_full_size_gmres_cycle_residual_is_true_residual():
    """Two GMRES(20) cycles on the benchmark workload: the Arnoldi residual estimate the
    solver reports equals the true residual ||Pi(V) - V||_2 / ||Pi(0)||_2 of the returned V
    (to the accuracy of the maps), and the estimate does not increase within a cycle."""
    wl = inputs.square_large()
    solver = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl)
    v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    info = solver.solve_gmres(v, restart=20, tol=1e-8, max_iters=40, raise_on_error=False)
    assert info["status"] in (_lib.OK, _lib.ERR_NOT_CONVERGED)
    assert info["iterations"] == 40 and info["pi_applications"] == 42
    h = info["history"]
    assert np.all(np.diff(h[:20]) <= 1e-15) and np.all(np.diff(h[20:]) <= 1e-15)
    pv = torch.empty_like(v)
    solver.apply_Pi(v, pv, forced=True)
    b = torch.empty_like(v)
    solver.apply_Pi(None, b, forced=True)
    torch.cuda.synchronize()
    nb = float(torch.linalg.norm(b))
    true_res = float(torch.linalg.norm(pv - v)) / nb
    # Each map carries the float-pair filter sums' error, at most about N_t 2^-46 of its
    # output.  The estimate combines 20 products S v_j per cycle (coefficients y with
    # sum |y_j| <= sqrt(40) ||V||); the true residual takes one more map of V.
    eps_map = solver.setup["n_t"] * 2.0 ** -46
    bound = eps_map * (float(torch.linalg.norm(pv)) + 40 ** 0.5 * float(torch.linalg.norm(v))) / nb
    assert abs(true_res - info["rel_residual"]) <= 1e-6 * info["rel_residual"] + 1e-13 + bound, \
        (true_res, info["rel_residual"], bound)
    assert np.all(np.isfinite(info["helmholtz_residual"]))


# ---------------------------------------------------------------------------
# c^2 given per grid point (MFWH_C_FIELD): L = c^2 Delta, non-divergence form
# ---------------------------------------------------------------------------

def _field_pair(wl, c2, mode=1, order=2):
    solver = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                      filter_mode=mode, order=order, c2_field=dev(c2))
    fm = {0: F.FILTER_OPTIMIZED, 1: F.FILTER_TRADITIONAL}[mode]
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=fm, order=order)
    assert solver.setup["n_t"] == prob.setup.n_t
    return solver, prob


@pytest.mark.parametrize("dims,order", [((20, 18, 16), 2), ((40, 33), 2), ((40, 33), 4),
                                        ((22, 19, 17), 4)])
def test_pi_random_c2_field(dims, order):
    """c drawn uniformly in [1, 1.5] at every point (2D and 3D, second and fourth order),
    forced and homogeneous maps element by element against the oracle."""
    om = [8.3, 12.1, 19.0] if len(dims) == 3 else [6.1, 9.7, 15.2]
    wl = inputs.gaussian_workload("field", dims, 3, om, 300.0, 23)
    c2 = inputs.random_c2(dims, 24, 1.0, 1.5)
    for mode in (1, 0):
        solver, prob = _field_pair(wl, c2, mode=mode, order=order)
        check_pi(solver, prob, random_v(wl, 25), forced=True)
        check_pi(solver, prob, random_v(wl, 26), forced=False)
        solver.close()


def test_field_of_two_layers_matches_two_layer_mode():
    """A field holding the two-layer medium gives the two-layer handle's map (different
    rounding order of the same operator), and its residual matches the oracle's."""
    wl = inputs.gaussian_workload("cube", (20, 18, 16), 4, [8.3, 12.1, 19.0, 27.5], 300.0, 21)
    c2 = inputs.two_layer_c2(wl.n, wl.length, 1.0, 1.5, 0.5)
    sf, prob = _field_pair(wl, c2, mode=0)
    sl, _ = make_pair(wl, c_hi=1.5)
    v = dev(random_v(wl, 27))
    a = torch.empty_like(v)
    b = torch.empty_like(v)
    sf.apply_Pi(v, a, forced=True)
    sl.apply_Pi(v, b, forced=True)
    torch.cuda.synchronize()
    assert np.all(rel_err(a.cpu().numpy(), b.cpu().numpy().reshape(a.shape)) <= 1e-12)
    r = random_v(wl, 28)
    np.testing.assert_allclose(sf.residual(dev(r)), W.helmholtz_residual(prob, r), rtol=1e-9)
    np.testing.assert_allclose(sf.residual(dev(r)), sl.residual(dev(r)), rtol=1e-12)


def test_gmres_with_c2_field_reaches_discrete_helmholtz():
    """GMRES on a random medium converges to the sparse direct solution of
    (c_j^2 Delta_h + omega^2) U = f."""
    wl = inputs.gaussian_workload("fieldg", (30, 26), 3, [6.1, 9.7, 15.2], 200.0, 29)
    c2 = inputs.random_c2(wl.n, 30, 1.0, 1.5)
    solver, prob = _field_pair(wl, c2, mode=0)
    v = np.zeros_like(wl.forcing)
    info = solver.solve_gmres(v, restart=100, tol=1e-12, max_iters=600, spurious_tol=1e-8)
    U = W.helmholtz_direct(prob)
    assert np.all(rel_err(v, U) <= 1e-9), (rel_err(v, U), info["iterations"])
