"""Oracle jobs that GPU tests run in worker processes (test infrastructure).

The FP64 oracle needs tens of seconds for one map of the 1025^2, N_f = 8 workload, so
tests that compare that workload element by element run several oracle maps at once in a
process pool started with the "spawn" method (a child never inherits a CUDA context).
Workers rebuild their inputs from seeds, so only seeds cross the process boundary going in.
"""

import numpy as np

from paper_2507_23613_gb300 import inputs
from oracle import filters as F
from oracle import wave as W


def random_v(wl, seed, scale=0.01):
    """Seeded white-noise iterate V (zero on the boundary) for the workload wl."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=wl.forcing.shape) * scale
    g = W.Grid(wl.n, wl.length)
    for m in range(v.shape[0]):
        W.zero_boundary(v[m], g)
    return v


def bench_workload_map(seed, filter_mode, user_seed, v_seed, forced):
    """The oracle's map Pi(V) (forced) or S V (homogeneous) on the 1025^2, N_f = 8, N_p = 2
    workload inputs.square_large(seed), with filter_mode 0 (least-squares parameters of
    Algorithm 2) or 2 (user parameters inputs.random_filter_params(user_seed, 8)).
    Returns (output, cond(M) of the optimiser's matrix, N_t)."""
    wl = inputs.square_large(seed)
    user = inputs.random_filter_params(user_seed, wl.nf) if filter_mode == 2 else None
    fm = F.FILTER_USER if filter_mode == 2 else F.FILTER_OPTIMIZED
    prob = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=wl.c2, cfl=wl.cfl,
                          n_p=wl.n_p, filter_mode=fm, user_params=user)
    v = random_v(wl, v_seed)
    out = W.apply_Pi(prob, v, forced=forced)
    return out, float(prob.setup.cond_M), int(prob.setup.n_t)
