"""GPU parity on the benchmark workload itself: the 1025^2, N_f = 8, N_p = 2 problem with
Gaussian sources (inputs.square_large(), the default seed that bench.py solves), in the
launch configuration bench.py times.  One forced map Pi(V) and one homogeneous map S V of
a seeded V are compared element by element, per frequency, with the FP64 oracle.

Two filter settings:
  - seeded user parameters, the same numbers on both sides: <= 1e-10 relative (max norm);
  - each side's own least-squares parameters (Algorithm 2): the bound max(1e-10,
    10 eps cond(M)^2) within which two correct least-squares solvers agree.
The oracle maps (about a minute each on one host core) run in spawned worker processes
while the GPU computes its own.
"""

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs

import oracle_jobs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10
EPS = np.finfo(np.float64).eps
SEED = 2000          # inputs.square_large's default: the workload bench.py times
USER_SEED = 503
V_SEEDS = {True: 61, False: 62}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load()


def rel_err(got, want):
    got = np.asarray(got).reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    scale = np.maximum(np.max(np.abs(want), axis=1), 1e-300)
    return np.max(np.abs(got - want), axis=1) / scale


@pytest.mark.parametrize("mode", [2, 0], ids=["user_params", "least_squares_params"])
def test_bench_workload_maps_match_oracle(mode):
    wl = inputs.square_large(SEED)
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=2, mp_context=ctx) as pool:
        jobs = {forced: pool.submit(oracle_jobs.bench_workload_map, SEED, mode, USER_SEED,
                                    V_SEEDS[forced], forced)
                for forced in (True, False)}
        user = inputs.random_filter_params(USER_SEED, wl.nf) if mode == 2 else None
        solver = M.Solver(wl.n, wl.length, wl.omega,
                          torch.from_numpy(wl.forcing).cuda(), n_p=wl.n_p, cfl=wl.cfl,
                          filter_mode=mode, user_params=user)
        got = {}
        for forced in (True, False):
            v = torch.from_numpy(oracle_jobs.random_v(wl, V_SEEDS[forced])).cuda()
            out = torch.empty_like(v)
            solver.apply_Pi(v, out, forced=forced)
            torch.cuda.synchronize()
            got[forced] = out.cpu().numpy()
        n_t = solver.setup["n_t"]
        solver.close()
        results = {forced: job.result() for forced, job in jobs.items()}
    for forced in (True, False):
        want, cond_m, n_t_oracle = results[forced]
        assert n_t == n_t_oracle == 2761
        tol = TOL if mode == 2 else max(TOL, 10.0 * EPS * cond_m * cond_m)
        err = rel_err(got[forced], want)
        print(f"mode {mode} forced {forced}: per-frequency error {np.array2string(err, precision=2)}"
              f" (tol {tol:.2e})")
        assert np.all(err <= tol), (forced, err, tol)
