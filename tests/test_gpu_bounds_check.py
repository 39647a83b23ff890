"""The index-checked debugging build of the library (libmfwh_bc.so, built with
-DMFWH_BOUNDS_CHECK).  Its FP64 step kernels (one step per launch, the blocked kernel and the
persistent pipelined kernel, 2D and 3D) test the index of each checked global and
shared-memory access against its array's extent and record an out-of-range index in the
handle's fault record instead of making the access.

On valid problems the checked build must record nothing and give results bit-identical to the
normal build.  One process loads one build of the library, so the checked build runs in a
child process and the parent compares its results with the normal build's."""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Run by both processes: maps and a few GMRES iterations on small grids that reach every
# checked kernel; returns the results and each handle's fault count.
CASES = r'''
import numpy as np
import torch
import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, inputs


def run_cases():
    torch.cuda.set_device(0)
    out, faults = {}, {}
    cases = [
        ("default_2d", (70, 45), 3, {}),                       # pipelined kernel, depth 3
        ("one_step_2d", (70, 45), 3, dict(time_block=1)),      # k_init, k_step, k_last
        ("blocked_8_2d", (70, 45), 3, dict(time_block=8, tile_shape=3)),
        ("two_layer_2d", (130, 160), 2, dict(c_lo=1.0, c_hi=1.4, interface=0.37, layer_axis=1)),
        ("one_step_3d", (12, 10, 8), 2, {}),
    ]
    for name, n, nf, kw in cases:
        om = np.linspace(6.0, 6.0 + 2.5 * (nf - 1), nf)
        wl = inputs.gaussian_workload(name, n, nf, om, 150.0, 17)
        rng = np.random.default_rng(5)
        v = rng.normal(size=wl.forcing.shape) * 0.01
        s = M.Solver(wl.n, wl.length, wl.omega, torch.from_numpy(wl.forcing).cuda(),
                     filter_mode=_lib.FILTER_TRADITIONAL, **kw)
        res = []
        for forced in (True, False):
            o = torch.empty(v.shape, dtype=torch.float64, device="cuda")
            s.apply_Pi(torch.from_numpy(v).cuda(), o, forced=forced)
            res.append(o.cpu().numpy())
        x = torch.zeros(v.shape, dtype=torch.float64, device="cuda")
        s.solve_gmres(x, restart=4, tol=0.0, max_iters=6, raise_on_error=False)
        res.append(x.cpu().numpy())
        out[name] = np.stack(res)
        faults[name] = s.debug_bounds()[0]
        s.close()
    return out, faults
'''

CHILD = CASES + r'''
import sys
out, faults = run_cases()
np.savez(sys.argv[1], **out, **{"faults_" + k: np.int64(v) for k, v in faults.items()})
'''


@pytest.mark.gpu
def test_checked_build_records_no_fault_and_matches_the_normal_build(tmp_path):
    from paper_2507_23613_gb300 import build
    lib_bc = build.build(bounds_check=True)
    env = dict(os.environ, MFWH_LIBRARY=lib_bc, PYTHONPATH=ROOT)
    dump = str(tmp_path / "checked.npz")
    r = subprocess.run([sys.executable, "-c", CHILD, dump], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.load(dump)

    scope = {}
    exec(CASES, scope)
    want, faults_normal = scope["run_cases"]()
    for name, ref in want.items():
        assert faults_normal[name] == -1          # the normal build compiles no checks
        assert int(got["faults_" + name]) == 0, name
        assert np.array_equal(got[name], ref), (name, np.max(np.abs(got[name] - ref)))
