"""GPU parity of the FP32 wave path (precision MFWH_PREC_FP32_KAHAN): FP32 wave
levels advanced in increment form, Kahan-compensated filter sums, FP64 filter
solve, GMRES and residual.  Results are compared with the FP64 oracle per
frequency m as e_m = max_j |V_gpu - V_oracle| / max_j |V_oracle|.

Stated FP32 error bounds (measured values on GB300 in brackets):
  * one map Pi on grids up to 70 x 45, N_t <= 207:          e_m <= 2e-5   [<= 3.2e-6]
  * one map Pi, 3D two-layer 20 x 18 x 16:                   e_m <= 2e-5   [<= 1.3e-6]
  * GMRES to 1e-12 on the 65^2 workload vs the discrete
    Helmholtz solution:                                      e_m <= 2e-6   [2.1e-7],
    Helmholtz residual r_h <= 5e-5 [4.3e-6]
The error comes from rounding the wave levels to FP32 at every step (a random
walk over N_t steps) and from the FP32 weights and coefficients; the Kahan
sums keep the filter accumulation itself at FP32 rounding level.
"""

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs
from oracle import filters as F
from oracle import wave as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_PI32 = 2e-5
TOL_SOL32 = 2e-6
TOL_RH32 = 5e-5


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


def apply(solver, v, forced):
    out = torch.empty(v.shape, dtype=torch.float64, device="cuda")
    solver.apply_Pi(dev(v), out, forced=forced)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def fp32_solver(wl, **kw):
    kw.setdefault("filter_mode", _lib.FILTER_TRADITIONAL)
    return M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                    precision=_lib.PREC_FP32_KAHAN, **kw)


def _ragged_nf8():
    wl = inputs.gaussian_workload("ragged", (70, 45), 8,
                                  lambda r: inputs.draw_frequencies(r, 8, 10.0, 60.0), 400.0, 77,
                                  length=(1.3, 0.9))
    wl.n_p = 2
    return wl


@pytest.mark.parametrize("which", ["square65", "ragged70x45_nf8", "tiny", "nf16"])
def test_fp32_blocking_depths_and_tiles_are_bit_identical(which):
    """Every temporal-blocking depth (1, 4, 8, 16) and tile shape performs the same FP32
    operations per point: Pi, S and a few GMRES iterations agree bit for bit."""
    if which == "square65":
        wl = inputs.square_small()
    elif which == "ragged70x45_nf8":
        wl = _ragged_nf8()
    elif which == "tiny":
        wl = inputs.gaussian_workload("tiny", (2, 2), 2, [3.0, 5.0], 5.0, 1)
    else:
        om = np.linspace(5.0, 50.0, 16)
        wl = inputs.gaussian_workload("nf16", (33, 31), 16, om, 150.0, 46)
        wl.n_p = 2
    v = random_v(wl, 11)
    outs = {}
    for tb, shape in [(1, 0), (4, 0), (8, 1), (16, 0), (16, 1), (16, 2)]:
        s = fp32_solver(wl, time_block=tb, tile_shape=shape)
        res = [apply(s, v, True), apply(s, v, False)]
        x = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
        s.solve_gmres(x, restart=4, tol=0.0, max_iters=6, raise_on_error=False)
        res.append(x.cpu().numpy())
        outs[(tb, shape)] = res
        s.close()
    for key, res in outs.items():
        for a, b in zip(res, outs[(1, 0)]):
            assert np.array_equal(a, b), (key, np.max(np.abs(a - b)))


@pytest.mark.parametrize("which", ["square65", "ragged70x45_nf8"])
def test_fp32_pi_error_per_frequency(which):
    wl = inputs.square_small() if which == "square65" else _ragged_nf8()
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=F.FILTER_TRADITIONAL)
    s = fp32_solver(wl)
    v = random_v(wl, 3)
    for forced in (True, False):
        err = rel_err(apply(s, v, forced), W.apply_Pi(prob, v, forced=forced))
        assert np.all(err <= TOL_PI32), (forced, err)
    err0 = rel_err(apply(s, np.zeros_like(v), True), W.apply_Pi(prob, np.zeros_like(v)))
    assert np.all(err0 <= TOL_PI32), err0


def test_fp32_pi_3d_two_layer():
    wl = inputs.gaussian_workload("cube", (20, 18, 16), 3, [7.0, 11.0, 16.0], 150.0, 5)
    c2 = inputs.two_layer_c2(wl.n, wl.length, 1.0, 1.5, 0.5)
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=F.FILTER_TRADITIONAL)
    s = fp32_solver(wl, c_lo=1.0, c_hi=1.5, interface=0.5, layer_axis=2)
    v = random_v(wl, 4)
    err = rel_err(apply(s, v, True), W.apply_Pi(prob, v, True))
    assert np.all(err <= TOL_PI32), err


@pytest.mark.parametrize("case", ["cube_two_layer", "thin", "nf16"])
def test_fp32_3d_blocked_is_bit_identical_and_matches_oracle(case):
    """3D temporal blocking (depths 2 and 4, 32 x 8 x 8 tiles with halo) performs the
    one-step kernel's FP32 operations per point: Pi, S and GMRES iterates agree bit for bit
    under Kahan sums; the blocked BLOCKSUM map stays within the FP32 bound of the oracle."""
    kw = {}
    if case == "cube_two_layer":
        wl = inputs.gaussian_workload("cube", (20, 18, 16), 3, [7.0, 11.0, 16.0], 150.0, 5)
        kw = dict(c_lo=1.0, c_hi=1.5, interface=0.5, layer_axis=2)
        c2 = inputs.two_layer_c2(wl.n, wl.length, 1.0, 1.5, 0.5)
    elif case == "thin":
        wl = inputs.gaussian_workload("thin", (40, 6, 9), 2, [6.0, 11.0], 100.0, 6,
                                      length=(2.0, 0.3, 0.45))
        c2 = 1.0
    else:
        om = np.linspace(5.0, 50.0, 16)
        wl = inputs.gaussian_workload("nf16c", (12, 10, 14), 16, om, 60.0, 47)
        wl.n_p = 2
        c2 = 1.0
    v = random_v(wl, 12)
    outs = {}
    for tb in (1, 2, 4):
        s = fp32_solver(wl, time_block=tb, **kw)
        res = [apply(s, v, True), apply(s, v, False)]
        x = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
        s.solve_gmres(x, restart=4, tol=0.0, max_iters=5, raise_on_error=False)
        res.append(x.cpu().numpy())
        outs[tb] = res
        s.close()
    for tb in (2, 4):
        for a, b in zip(outs[tb], outs[1]):
            assert np.array_equal(a, b), (tb, np.max(np.abs(a - b)))
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=F.FILTER_TRADITIONAL)
    sb = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                  precision=_lib.PREC_FP32_BLOCKSUM, time_block=4,
                  filter_mode=_lib.FILTER_TRADITIONAL, **kw)
    err = rel_err(apply(sb, v, True), W.apply_Pi(prob, v, True))
    assert np.all(err <= TOL_PI32), err


def test_fp32_two_layer_2d_blocked_matches_unblocked():
    """Layer coefficients selected per point inside the blocked kernel (interface at y = 0.5)."""
    wl = inputs.gaussian_workload("layer2d", (64, 48), 4, [6.0, 9.0, 13.0, 18.0], 200.0, 8)
    wl.n_p = 2
    kw = dict(c_lo=1.0, c_hi=1.5, interface=0.5, layer_axis=1)
    v = random_v(wl, 5)
    a = fp32_solver(wl, time_block=1, **kw)
    b = fp32_solver(wl, time_block=16, **kw)
    assert np.array_equal(apply(a, v, True), apply(b, v, True))
    c2 = inputs.two_layer_c2(wl.n, wl.length, 1.0, 1.5, 0.5)
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=F.FILTER_TRADITIONAL)
    err = rel_err(apply(b, v, True), W.apply_Pi(prob, v, True))
    assert np.all(err <= TOL_PI32), err


def test_fp32_gmres_reaches_discrete_helmholtz_solution():
    wl = inputs.square_small()
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, cfl=wl.cfl, n_p=wl.n_p)
    U = W.helmholtz_direct(prob)
    s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                 precision=_lib.PREC_FP32_KAHAN)
    x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    info = s.solve_gmres(x, restart=200, tol=1e-12, max_iters=200)
    assert info["status"] == _lib.OK
    err = rel_err(x.cpu().numpy(), U)
    assert np.all(err <= TOL_SOL32), err
    assert np.all(info["helmholtz_residual"] <= TOL_RH32), info["helmholtz_residual"]
    r = s.residual(x)
    np.testing.assert_allclose(r, W.helmholtz_residual(prob, x.cpu().numpy()), rtol=1e-9)


# ---------------------------------------------------------------------------
# Mixed-precision defect correction (mfwh_solve_refined)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [_lib.PREC_FP32_KAHAN, _lib.PREC_FP32_BLOCKSUM])
def test_refined_fp32_reaches_fp64_accuracy(prec):
    """FP32 wave solves inside an FP64 defect-correction loop reach the discrete Helmholtz
    solution to FP64-level accuracy (the FP32-only solve stops near 2e-7)."""
    wl = inputs.square_small()
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, cfl=wl.cfl, n_p=wl.n_p)
    U = W.helmholtz_direct(prob)
    s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                 precision=prec)
    before = apply(s, np.zeros_like(wl.forcing), True)
    x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    info = s.solve_refined(x, target=1e-10, inner_tol=1e-7, restart=100, max_iters=100,
                           max_refinements=8)
    assert info["status"] == _lib.OK and 1 <= info["refinements"] <= 8
    err = rel_err(x.cpu().numpy(), U)
    assert np.all(err <= 1e-9), err
    rh = W.helmholtz_residual(prob, x.cpu().numpy())
    assert np.all(rh <= 1e-10), rh
    np.testing.assert_allclose(info["helmholtz_residual"], rh, rtol=1e-6, atol=1e-14)
    # the handle's own forcing is back in place for the wave solve
    assert np.array_equal(apply(s, np.zeros_like(wl.forcing), True), before)


def test_relaxed_products_reach_fp64_accuracy():
    """Relaxed inner solves (FP64 products until the inner residual is below 1e-3, FP32 after)
    inside FP64 refinement reach the discrete Helmholtz solution to FP64-level accuracy; with
    the switch set below the inner tolerance every product is FP64 and the result is the FP64
    refinement's (same Arnoldi steps); an FP64 handle and a switch outside (0, 1) are refused."""
    wl = inputs.square_small()
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, cfl=wl.cfl, n_p=wl.n_p)
    U = W.helmholtz_direct(prob)
    s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                 precision=_lib.PREC_FP32_BLOCKSUM)
    x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    info = s.solve_relaxed(x, target=1e-10, inner_tol=1e-7, relax_below=1e-3, restart=100,
                           max_iters=200, max_refinements=8)
    assert info["status"] == _lib.OK
    assert np.all(rel_err(x.cpu().numpy(), U) <= 1e-9)
    assert np.all(W.helmholtz_residual(prob, x.cpu().numpy()) <= 1e-10)
    # the switch never reached: FP64 products only, as an FP64 handle's refinement
    f64 = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl)
    y = torch.zeros_like(x)
    z = torch.zeros_like(x)
    a = s.solve_relaxed(y, target=1e-9, inner_tol=1e-10, relax_below=1e-12, restart=100,
                        max_iters=100)
    b = f64.solve_refined(z, target=1e-9, inner_tol=1e-10, restart=100, max_iters=100)
    assert a["iterations"] == b["iterations"] and a["refinements"] == b["refinements"]
    assert torch.equal(y, z)
    for solver, relax in ((f64, 1e-3), (s, 0.0), (s, 1.0)):
        with pytest.raises(_lib.MfwhError) as e:
            solver.solve_relaxed(torch.zeros_like(x), relax_below=relax)
        assert e.value.status == _lib.ERR_INVALID_ARG


def test_refined_fp64_handle_and_warm_start():
    wl = inputs.square_small()
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, cfl=wl.cfl, n_p=wl.n_p)
    U = W.helmholtz_direct(prob)
    s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl)
    x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    info = s.solve_refined(x, target=1e-9, inner_tol=1e-10, restart=100, max_iters=100)
    assert info["status"] == _lib.OK
    assert np.all(rel_err(x.cpu().numpy(), U) <= 1e-9)
    # starting from the solution: no correction is needed
    info2 = s.solve_refined(x, target=1e-8, inner_tol=1e-10, restart=100, max_iters=100)
    assert info2["refinements"] == 0 and info2["iterations"] == 0
    # a target that cannot be met within the allowed corrections is reported
    y = torch.zeros_like(x)
    info3 = s.solve_refined(y, target=1e-14, inner_tol=1e-2, restart=5, max_iters=5,
                            max_refinements=1, raise_on_error=False)
    assert info3["status"] == _lib.ERR_NOT_CONVERGED and info3["refinements"] == 1
