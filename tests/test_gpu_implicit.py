"""GPU parity of the implicit trapezoidal wave solve (eq. WaveScheme with (alpha, beta) =
(1/2, 0), multigrid solves on the device) against the FP64 oracle, whose steps are sparse LU
solves: one map Pi (forced and homogeneous, implicit and explicit filter) on one-CTA, grid-wide,
anisotropic, ragged-coarsest and 3D two-layer hierarchies; the discrete Helmholtz solution as
the fixed point; GMRES to the direct solution; the multigrid statistics; batches mixing
implicit and explicit handles."""

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs
from oracle import filters as F
from oracle import wave as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10          # FP64 parity (relative max norm per frequency)
MG_TOL = 1e-13       # step solves converged to near rounding for the parity cases


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, want):
    got = np.asarray(got).reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return np.max(np.abs(got - want), axis=1) / np.maximum(np.max(np.abs(want), axis=1), 1e-300)


def random_v(wl, seed, scale=0.01):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=wl.forcing.shape) * scale
    g = W.Grid(wl.n, wl.length)
    for m in range(v.shape[0]):
        W.zero_boundary(v[m], g)
    return v


CASES = {
    # name: (cells, length, omega, b, c_hi, levels expected to be grid-wide)
    "one_cta_2d": ((32, 32), (1.0, 1.0), [5.5, 9.3, 14.0], 200.0, None),
    "grid_2d": ((128, 128), (1.0, 1.0), [5.5, 9.3, 14.0], 300.0, None),
    "aniso_2d": ((256, 128), (1.0, 0.5), [6.0, 11.0], 300.0, None),
    "ragged_coarsest_2d": ((96, 80), (1.2, 1.0), [4.5, 8.0, 12.5], 200.0, None),
    "cube3d_two_layer": ((32, 32, 32), (1.0, 1.0, 1.0), [4.1, 7.9, 12.5], 60.0, 1.5),
    "cube3d_o4": ((20, 20, 20), (1.0, 1.0, 1.0), [4.1, 7.9, 12.5], 60.0, 1.5),
}


def pair(name, filter_update=0, mg_tol=MG_TOL, n_p=1, mode=F.FILTER_OPTIMIZED, order=2):
    n, length, omega, b, c_hi = CASES[name]
    wl = inputs.gaussian_workload(name, n, len(omega), omega, b, 17, length=length)
    kw = dict(n_p=n_p, filter_mode={F.FILTER_OPTIMIZED: 0, F.FILTER_TRADITIONAL: 1}[mode],
              time_stepping="implicit", mg_tol=mg_tol, filter_update=filter_update, order=order)
    c2 = 1.0
    if c_hi is not None:
        kw.update(c_lo=1.0, c_hi=c_hi, interface=0.5, layer_axis=len(n) - 1)
        c2 = inputs.two_layer_c2(n, length, 1.0, c_hi, 0.5)
    s = M.Solver(n, length, omega, dev(wl.forcing), **kw)
    p = W.make_problem(W.Grid(n, length), omega, wl.forcing, c2=c2, n_p=n_p, filter_mode=mode,
                       time_stepping="implicit", explicit_filter=filter_update == 1, order=order)
    assert s.setup["n_t"] == p.setup.n_t
    assert abs(s.setup["dt"] - p.setup.dt) < 1e-15 * p.setup.dt
    return s, p, wl


def apply(s, v, forced):
    out = torch.empty(v.shape, dtype=torch.float64, device="cuda")
    s.apply_Pi(dev(v), out, forced=forced)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_implicit_pi_matches_oracle(name):
    s, p, wl = pair(name)
    v = random_v(wl, 5)
    for forced in (True, False):
        got = apply(s, v, forced)
        want = W.apply_Pi(p, v, forced=forced)
        assert np.all(rel_err(got, want) < TOL), (forced, rel_err(got, want))
    st = s.mg_stats()
    n_t = s.setup["n_t"]
    assert st["solves"] == 2 * n_t
    assert st["unconverged"] == 0
    assert st["levels"] >= 2 or name == "one_cta_2d"
    # boundary values of the output are 0
    got = apply(s, v, True).reshape(wl.forcing.shape)
    g = W.Grid(wl.n, wl.length)
    edge = got.copy()
    for m in range(edge.shape[0]):
        W.zero_boundary(edge[m], g)
    assert np.array_equal(edge, got)


@pytest.mark.parametrize("nf", [1, 16])
def test_implicit_pi_extreme_frequency_counts(nf):
    """One and the maximum number of frequencies (traditional filters: both sides use the
    closed-form parameters of eq. origParamAdjust)."""
    om = np.linspace(5.0, 5.0 + 3.0 * (nf - 1), nf)
    n, length = (128, 128), (1.0, 1.0)
    wl = inputs.gaussian_workload("nfimp", n, nf, om, 150.0, 40 + nf)
    n_p = 2 if nf > 1 else 1
    s = M.Solver(n, length, om, dev(wl.forcing), n_p=n_p, filter_mode=1,
                 time_stepping="implicit", mg_tol=MG_TOL)
    p = W.make_problem(W.Grid(n, length), om, wl.forcing, n_p=n_p,
                       filter_mode=F.FILTER_TRADITIONAL, time_stepping="implicit")
    assert s.setup["n_t"] == p.setup.n_t
    v = random_v(wl, 9)
    got = apply(s, v, True)
    assert np.all(rel_err(got, W.apply_Pi(p, v, forced=True)) < TOL)


def test_implicit_pi_explicit_filter_and_traditional():
    s, p, wl = pair("grid_2d", filter_update=1, mode=F.FILTER_TRADITIONAL)
    v = random_v(wl, 8)
    got = apply(s, v, True)
    assert np.all(rel_err(got, W.apply_Pi(p, v, forced=True)) < TOL)
    got0 = apply(s, np.zeros_like(v), True)
    assert np.all(rel_err(got0, W.apply_Pi(p, np.zeros_like(v), forced=True)) < TOL)


def test_implicit_fixed_point_is_discrete_helmholtz():
    """The GPU's implicit map keeps the direct Helmholtz solution fixed (eq. discreteHelmholtz)."""
    s, p, wl = pair("grid_2d", n_p=2)
    U = W.helmholtz_direct(p)
    got = apply(s, U, True)
    assert np.all(rel_err(got, U) < 1e-10)


def test_implicit_gmres_converges_to_direct_solution():
    s, p, wl = pair("grid_2d", mg_tol=0.0)       # library default tolerance 1e-10
    U = W.helmholtz_direct(p)
    v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    s.mg_stats(reset=True)
    info = s.solve_gmres(v, restart=100, tol=1e-10, max_iters=400)
    x = v.cpu().numpy()
    assert info["rel_residual"] < 1e-10
    assert np.all(rel_err(x, U) < 1e-7)
    assert np.max(info["helmholtz_residual"]) < 1e-7
    st = s.mg_stats()
    assert st["unconverged"] == 0
    assert st["solves"] == info["pi_applications"] * s.setup["n_t"]
    assert 1.0 <= st["cycles"] / st["solves"] <= 15.0


def test_implicit_graph_mode_and_batch():
    s1, p1, wl1 = pair("grid_2d", mg_tol=1e-12)
    s2, p2, wl2 = pair("one_cta_2d", mg_tol=1e-12)
    e = M.Solver(wl2.n, wl2.length, wl2.omega, dev(wl2.forcing))     # explicit handle
    v = random_v(wl1, 3)
    a = apply(s1, v, True)
    s1.set_graphs(True)                      # implicit handles run without graphs
    b = apply(s1, v, True)
    assert np.array_equal(a, b)
    vs = [torch.zeros(w.forcing.shape, dtype=torch.float64, device="cuda") for w in (wl1, wl2, wl2)]
    st, infos, secs = M.solve_batch([s1, s2, e], vs, restart=100, tol=1e-11, max_iters=400)
    assert st == _lib.OK
    for sol, prob in ((vs[0], p1), (vs[1], p2)):
        U = W.helmholtz_direct(prob)
        assert np.all(rel_err(sol.cpu().numpy(), U) < 1e-7)
    assert all(i["rel_residual"] < 1e-11 for i in infos)
    e.close()


@pytest.mark.parametrize("name", ["grid_2d", "aniso_2d", "cube3d_o4"])
def test_implicit_fourth_order_pi_matches_oracle(name):
    """Fourth-order L_4h (odd-reflection ghosts) in the FP64 residual, the second-order
    multigrid as the correction solver (damped by 6/7); in 3D the residual runs in the
    grid-wide phases.  The step tolerance is 1e-12: the rounding floor of the fourth-order
    residual (diagonal ~500 on the anisotropic grid) lies near 5e-14."""
    s, p, wl = pair(name, order=4, mg_tol=1e-12)
    v = random_v(wl, 6)
    for forced in (True, False):
        got = apply(s, v, forced)
        want = W.apply_Pi(p, v, forced=forced)
        assert np.all(rel_err(got, want) < TOL), (forced, rel_err(got, want))
    st = s.mg_stats()
    assert st["unconverged"] == 0


def test_implicit_fourth_order_fixed_point_and_gmres():
    s, p, wl = pair("grid_2d", order=4, n_p=2, mg_tol=1e-12)
    U = W.helmholtz_direct(p)
    assert np.all(rel_err(apply(s, U, True), U) < 1e-10)
    s2, p2, wl2 = pair("grid_2d", order=4, mg_tol=1e-12)
    U2 = W.helmholtz_direct(p2)
    v = torch.zeros(wl2.forcing.shape, dtype=torch.float64, device="cuda")
    info = s2.solve_gmres(v, restart=100, tol=1e-10, max_iters=400)
    assert np.all(rel_err(v.cpu().numpy(), U2) < 1e-7)
    assert np.max(info["helmholtz_residual"]) < 1e-7


def test_implicit_fourth_order_3d_fixed_point():
    s, p, wl = pair("cube3d_o4", order=4, mg_tol=1e-12)
    assert s.mg_stats()["levels"] == 3
    U = W.helmholtz_direct(p)
    assert np.all(rel_err(apply(s, U, True), U) < 1e-10)
    assert s.mg_stats()["unconverged"] == 0


def test_implicit_full_size_eigenmode_closed_form():
    """The 1025^2, N_f = 8, N_p = 2 workload with implicit steps: Pi maps a Dirichlet mode to
    the same mode with the closed-form coefficients (theta from the roots of the scheme's
    characteristic polynomial), through the full multigrid hierarchy (10 levels)."""
    wl = inputs.square_large()
    g = W.Grid(wl.n, wl.length)
    setup = F.make_setup(wl.omega, g.h, 1.0, wl.cfl, wl.n_p, F.FILTER_TRADITIONAL,
                         time_stepping="implicit")
    rng = np.random.default_rng(46)
    for k in [(3, 5), (200, 17)]:
        phi, lam2 = W.dirichlet_mode(g, k)
        a = rng.normal(size=wl.nf)
        v = rng.normal(size=wl.nf)
        f = a[:, None, None] * phi
        s = M.Solver(wl.n, wl.length, wl.omega, dev(f), n_p=wl.n_p, cfl=wl.cfl,
                     filter_mode=1, time_stepping="implicit", mg_tol=1e-13)
        assert s.setup["n_t"] == setup.n_t
        got = apply(s, v[:, None, None] * phi, True)
        x = lam2 * setup.dt ** 2
        r = np.roots([1.0 + 0.5 * x, -2.0, 1.0 + 0.5 * x])
        theta = float(np.max(np.abs(np.angle(r))))
        u = a / (setup.omega ** 2 - lam2)
        n = np.arange(setup.n_t + 1)
        W_hat = (np.cos(n * theta) * np.sum(v - u)
                 + np.cos(np.outer(n * setup.dt, setup.omega_t)) @ u)
        want = np.linalg.solve(setup.B, setup.w.T @ W_hat)[:, None, None] * phi
        assert np.all(rel_err(got, want) < 1e-9), (k, rel_err(got, want))
        assert s.mg_stats()["levels"] == 10
        s.close()


def test_implicit_rejects_grids_without_a_small_level():
    with pytest.raises(_lib.MfwhError) as err:
        M.Solver((32, 32), (1.0, 1.0), [5.0, 9.0], time_stepping="implicit", order=4)
    assert err.value.status == _lib.ERR_INVALID_ARG
    with pytest.raises(_lib.MfwhError) as err:
        M.Solver((101, 100), (1.0, 1.0), [5.0, 9.0], time_stepping="implicit")
    assert err.value.status == _lib.ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["grid_2d", "cube3d_two_layer"])
def test_barrier_timeout_is_reported_and_handle_recovers(name):
    """Failure detection without a fault.  With a barrier wait limit of 1 ns a wait of the
    step kernel's grid barrier runs out: the kernel records it, lets its blocks through the
    remaining barriers (every loop bounded, every index geometric), the later step launches
    return at once, and the solve reports MFWH_ERR_TIMEOUT.  With the default limit restored
    the same handle's map matches the oracle again."""
    s, p, wl = pair(name)
    v = random_v(wl, 9)
    s.set_wait_limit(1e-9)
    x = dev(v)
    with pytest.raises(_lib.MfwhError) as e:
        s.solve_fpi(x, 1)
    assert e.value.status == _lib.ERR_TIMEOUT
    assert "timed out" in str(e.value)
    s.set_wait_limit(0.0)                 # back to the default (2 s)
    got = apply(s, v, True)
    s.last_timing()                       # no flag left set: the call succeeds
    want = W.apply_Pi(p, v, forced=True)
    assert np.all(rel_err(got, want) < TOL), rel_err(got, want)
    with pytest.raises(_lib.MfwhError) as e:
        s.set_wait_limit(float("nan"))
    assert e.value.status == _lib.ERR_INVALID_ARG
    s.close()
