"""GPU tests of the many-problem machinery: CUDA-graph mode (one graph launch per
application of Pi), concurrent batched GMRES solves, and the autotuner.  Graph replay
and concurrency change neither the kernels nor their order per problem, so results
are compared bit for bit with direct launches."""

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs
from oracle import wave as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def random_v(wl, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=wl.forcing.shape) * 0.01
    g = W.Grid(wl.n, wl.length)
    for m in range(v.shape[0]):
        W.zero_boundary(v[m], g)
    return v


def problems():
    out = [inputs.square_small()]
    wl = inputs.gaussian_workload("b1", (96, 80), 5, [6.0, 9.5, 13.0, 17.5, 22.0], 250.0, 51)
    wl.n_p = 2
    out.append(wl)
    out.append(inputs.gaussian_workload("b2", (40, 33), 3, [5.0, 8.0, 12.0], 150.0, 52))
    wl = inputs.gaussian_workload("b3", (20, 18, 16), 2, [7.0, 11.0], 150.0, 53)
    out.append(wl)
    return out


def run_all(s, v):
    res = []
    for forced in (True, False):
        out = torch.empty(v.shape, dtype=torch.float64, device="cuda")
        s.apply_Pi(dev(v), out, forced=forced)
        res.append(out.cpu().numpy())
    x = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
    s.solve_gmres(x, restart=6, tol=0.0, max_iters=9, raise_on_error=False)
    res.append(x.cpu().numpy())
    return res


@pytest.mark.parametrize("prec", [_lib.PREC_FP64, _lib.PREC_FP32_BLOCKSUM])
def test_graph_mode_is_bit_identical(prec):
    for k, wl in enumerate(problems()[:3]):
        v = random_v(wl, 60 + k)
        kw = dict(n_p=wl.n_p, cfl=wl.cfl, precision=prec)
        a = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), **kw)
        b = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), **kw)
        b.set_graphs(True)
        ra, rb = run_all(a, v), run_all(b, v)
        rb2 = run_all(b, v)          # replaying the captured graphs again
        for x, y, z in zip(ra, rb, rb2):
            assert np.array_equal(x, y) and np.array_equal(x, z)
        _, steps, launches = b.last_timing()
        assert steps > 0
        b.set_graphs(False)
        for x, y in zip(ra, run_all(b, v)):
            assert np.array_equal(x, y)


def test_graph_mode_refined_solve():
    wl = inputs.square_small()
    kw = dict(n_p=wl.n_p, cfl=wl.cfl, precision=_lib.PREC_FP32_KAHAN)
    a = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), **kw)
    b = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), **kw)
    b.set_graphs(True)
    xa = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    xb = torch.zeros_like(xa)
    ia = a.solve_refined(xa, target=1e-9, inner_tol=1e-7, restart=60, max_iters=200)
    ib = b.solve_refined(xb, target=1e-9, inner_tol=1e-7, restart=60, max_iters=200)
    assert ia["iterations"] == ib["iterations"]
    assert torch.equal(xa, xb)


def test_batch_solve_matches_single_solves():
    wls = problems()
    precs = [_lib.PREC_FP64, _lib.PREC_FP32_BLOCKSUM, _lib.PREC_FP64, _lib.PREC_FP32_KAHAN]
    single, singles_info = [], []
    for wl, prec in zip(wls, precs):
        s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                     precision=prec)
        x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
        singles_info.append(s.solve_gmres(x, restart=10, tol=1e-9, max_iters=60,
                                          raise_on_error=False))
        single.append(x.cpu().numpy())
        s.close()
    streams = [torch.cuda.Stream() for _ in wls]
    solvers = []
    for wl, prec, st in zip(wls, precs, streams):
        s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), stream=st.cuda_stream,
                     n_p=wl.n_p, cfl=wl.cfl, precision=prec)
        s.set_graphs(True)
        solvers.append(s)
    torch.cuda.synchronize()
    xs = [torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda") for wl in wls]
    torch.cuda.synchronize()
    st, infos, secs = M.solve_batch(solvers, xs, restart=10, tol=1e-9, max_iters=60,
                                    raise_on_error=False)
    torch.cuda.synchronize()
    for x, ref, info, ref_info in zip(xs, single, infos, singles_info):
        assert np.array_equal(x.cpu().numpy(), ref)
        assert info["iterations"] == ref_info["iterations"]
    assert np.all(secs > 0)
    # the same handle twice is rejected
    with pytest.raises(_lib.MfwhError) as e:
        M.solve_batch([solvers[0], solvers[0]], xs[:2])
    assert e.value.status == _lib.ERR_INVALID_ARG


def test_autotune_picks_a_valid_configuration():
    wl = inputs.gaussian_workload("tune", (256, 256), 4, [10.0, 14.0, 19.0, 25.0], 300.0, 9)
    for prec in (_lib.PREC_FP32_BLOCKSUM, _lib.PREC_FP64):
        tb, shape, ms = M.autotune(wl.n, wl.length, wl.omega, n_p=2, cfl=0.5, precision=prec)
        if prec == _lib.PREC_FP64:
            assert (tb, shape) in ((1, 0), (2, 5), (3, 5), (4, 5), (4, 4), (4, 3), (8, 3))
        else:
            assert tb in (4, 8, 16) and shape in (0, 1, 2)
        assert ms > 0
        assert M.autotune(wl.n, wl.length, wl.omega, n_p=2, cfl=0.5, precision=prec) == (tb, shape, ms)
        s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=2, cfl=0.5, precision=prec,
                     time_block=tb, tile_shape=shape)
        s.close()
    tb, shape, ms = M.autotune((12, 10, 8), (1.0, 1.0, 1.0), [6.0, 9.0],
                               precision=_lib.PREC_FP32_BLOCKSUM)
    assert (tb, shape) == (1, 0)


@pytest.mark.parametrize("restart,max_iters,host", [(10, 60, False), (4, 11, True)])
def test_lockstep_batch_matches_single_solves(restart, max_iters, host):
    """The lockstep batch (one graph launch per application of the map across all problems)
    runs each problem's GMRES with the same kernels in the same order as a single solve, so the
    iterates are bit-identical; with restart 4 and 11 iterations problems restart from non-zero
    iterates (a product of the iterate in a round) and stop unconverged; host buffers are
    staged in and out."""
    wls = problems()
    precs = [_lib.PREC_FP64, _lib.PREC_FP32_BLOCKSUM, _lib.PREC_FP64, _lib.PREC_FP32_KAHAN]
    single, singles_info = [], []
    for k, (wl, prec) in enumerate(zip(wls, precs)):
        s = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                     precision=prec)
        x = dev(random_v(wl, 70 + k))
        singles_info.append(s.solve_gmres(x, restart=restart, tol=1e-9, max_iters=max_iters,
                                          raise_on_error=False))
        single.append(x.cpu().numpy())
        s.close()
    solvers = [M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing), n_p=wl.n_p, cfl=wl.cfl,
                        precision=prec) for wl, prec in zip(wls, precs)]
    xs = [random_v(wl, 70 + k) for k, wl in enumerate(wls)]
    if not host:
        xs = [dev(x) for x in xs]
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    st, infos, secs = M.solve_batch_graph(solvers, xs, restart=restart, tol=1e-9,
                                          max_iters=max_iters, stream=side.cuda_stream,
                                          raise_on_error=False)
    torch.cuda.synchronize()
    for x, ref, info, ref_info in zip(xs, single, infos, singles_info):
        got = x if host else x.cpu().numpy()
        assert np.array_equal(got, ref)
        assert info["iterations"] == ref_info["iterations"]
        assert info["pi_applications"] == ref_info["pi_applications"]
        assert info["restarts"] == ref_info["restarts"]
        np.testing.assert_array_equal(info["helmholtz_residual"], ref_info["helmholtz_residual"])
    assert np.all(secs > 0)
    want = _lib.OK if all(r["status"] == _lib.OK for r in singles_info) else _lib.ERR_NOT_CONVERGED
    assert st == want
    for s in solvers:
        s.close()


def test_lockstep_batch_rejects_implicit_and_repeated_handles():
    wl = problems()[2]
    a = M.Solver(wl.n, wl.length, wl.omega, dev(wl.forcing))
    imp = M.Solver((32, 32), (1.0, 1.0), [5.5, 9.3], time_stepping="implicit")
    x = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    y = torch.zeros((2, 33, 33), dtype=torch.float64, device="cuda")
    for hs, vs in (([a, a], [x, x]), ([a, imp], [x, y])):
        with pytest.raises(_lib.MfwhError) as e:
            M.solve_batch_graph(hs, vs)
        assert e.value.status == _lib.ERR_INVALID_ARG
