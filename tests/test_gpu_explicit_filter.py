"""GPU parity of the explicit-filter update (B_mm V_m^{k+1} = q_m - sum_{j != m} B_mj V_j^k,
the footnote to eq. filterII) against the oracle: one map in every kernel family (FP64 one
step and blocked, FP32 blocked and one step in 3D), in-place fixed-point iterations, graph
mode, and GMRES on the explicit map reaching the discrete Helmholtz solution."""

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs
from oracle import filters as F
from oracle import wave as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10
TOL_PI32 = 2e-5


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


def random_v(wl, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=wl.forcing.shape) * 0.01
    g = W.Grid(wl.n, wl.length)
    for m in range(v.shape[0]):
        W.zero_boundary(v[m], g)
    return v


def apply(s, v, forced):
    out = torch.empty(v.shape, dtype=torch.float64, device="cuda")
    s.apply_Pi(dev(v), out, forced=forced)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def make(wl, c_hi=None, **kw):
    kw.setdefault("filter_mode", _lib.FILTER_TRADITIONAL)
    kw2 = dict(kw)
    c2 = 1.0
    if c_hi is not None:
        kw2.update(c_lo=1.0, c_hi=c_hi, interface=0.5, layer_axis=len(wl.n) - 1)
        c2 = inputs.two_layer_c2(wl.n, wl.length, 1.0, c_hi, 0.5)
    s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                 filter_update=_lib.UPDATE_EXPLICIT, **kw2)
    fm = {0: F.FILTER_OPTIMIZED, 1: F.FILTER_TRADITIONAL}[kw["filter_mode"]]
    p = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                       n_p=wl.n_p, filter_mode=fm, explicit_filter=True)
    return s, p


@pytest.mark.parametrize("variant", ["fp64_one_step", "fp64_blocked", "fp32_blocked", "fp32_3d"])
def test_explicit_filter_pi(variant):
    if variant == "fp32_3d":
        wl = inputs.gaussian_workload("ef3", (18, 16, 14), 3, [7.0, 11.0, 16.0], 150.0, 81)
        s, p = make(wl, c_hi=1.5, precision=_lib.PREC_FP32_BLOCKSUM)
        tol = TOL_PI32
    else:
        wl = inputs.gaussian_workload("ef2", (70, 45), 4, [6.0, 9.5, 13.0, 18.5], 250.0, 82,
                                      length=(1.3, 0.9))
        wl.n_p = 2
        kw = {"fp64_one_step": dict(time_block=1), "fp64_blocked": dict(time_block=8),
              "fp32_blocked": dict(precision=_lib.PREC_FP32_BLOCKSUM)}[variant]
        s, p = make(wl, **kw)
        tol = TOL_PI32 if "fp32" in variant else TOL
    for forced, seed in ((True, 1), (False, 2)):
        v = random_v(wl, seed)
        err = rel_err(apply(s, v, forced), W.apply_Pi(p, v, forced=forced))
        assert np.all(err <= tol), (forced, err)
    # zero input: the E term vanishes (b = Pi(0))
    z = np.zeros_like(wl.forcing)
    assert np.all(rel_err(apply(s, z, True), W.apply_Pi(p, z)) <= tol)


def test_explicit_filter_in_place_iterations_and_graphs():
    """Fixed-point iterations update V in place (the E term reads V^k where V^{k+1} is
    written); graph replay gives the same bits."""
    wl = inputs.square_small()
    s, p = make(wl)
    g = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    s.solve_fpi(g, 6)
    V = np.zeros_like(wl.forcing)
    for _ in range(6):
        V = W.apply_Pi(p, V)
    assert np.all(rel_err(g.cpu().numpy(), V) <= TOL)
    s2, _ = make(wl)
    s2.set_graphs(True)
    g2 = torch.zeros_like(g)
    s2.solve_fpi(g2, 6)
    assert torch.equal(g, g2)


def test_explicit_filter_gmres_reaches_helmholtz_solution():
    wl = inputs.square_small()
    s, p = make(wl, filter_mode=_lib.FILTER_OPTIMIZED)
    U = W.helmholtz_direct(p)
    x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    info = s.solve_gmres(x, restart=200, tol=1e-12, max_iters=200)
    assert info["status"] == _lib.OK
    assert np.all(rel_err(x.cpu().numpy(), U) <= 1e-9)
