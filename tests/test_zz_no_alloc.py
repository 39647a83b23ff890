"""The allocation-free residual entry point (mfwh_residual_noalloc) against the
handle-based mfwh_residual.

mfwh_residual_noalloc is for callers that cannot allocate device memory where
they need the check (device memory owned by another allocator, or loops that
cannot accept the implicit synchronisation of cudaMalloc / cudaFree); it keeps
its reduction scratch in a fixed device array of the library instead.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest

import paper_2507_23613_gb300 as M
from paper_2507_23613_gb300 import _lib, build, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return _lib.load()


def _noalloc(lib, prob, f, v, stream):
    r = np.zeros(prob.nf)
    st = lib.mfwh_residual_noalloc(C.byref(prob), C.c_void_p(f.data_ptr()), C.c_void_p(v.data_ptr()),
                                   r.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream))
    return st, r


@pytest.mark.parametrize("dims,c_hi,order", [((48, 40), None, 2), ((20, 18, 16), 1.5, 2),
                                             ((48, 40), None, 4), ((20, 18, 16), "field", 2)])
def test_noalloc_matches_handle_residual_twice(lib, dims, c_hi, order):
    nf = 3
    wl = inputs.gaussian_workload("noalloc", dims, nf, [6.1, 9.7, 15.2], 200.0, 41)
    if c_hi == "field":         # c^2 per grid point, on the device for both entry points
        kw = dict(c2_field=torch.from_numpy(inputs.random_c2(dims, 43)).cuda())
    else:
        kw = {} if c_hi is None else dict(c_lo=1.0, c_hi=c_hi, interface=0.5,
                                          layer_axis=len(dims) - 1)
    kw["order"] = order
    f = torch.from_numpy(wl.forcing).cuda()
    solver = M.Solver(wl.n, wl.length, wl.omega, f, **kw)
    prob, keep = M.make_problem(wl.n, wl.length, wl.omega, **kw)
    rng = np.random.default_rng(7)
    # Two calls in a row with different inputs: on torch's current stream, and on the legacy
    # default stream (stream NULL).  Both paths run the same residual kernels with the same
    # geometry, so the results are bit-identical to the handle's.
    for call, stream in enumerate([torch.cuda.current_stream().cuda_stream, None]):
        v = torch.from_numpy(rng.normal(size=wl.forcing.shape) * 0.01).cuda()
        want = solver.residual(v)
        st, got = _noalloc(lib, prob, f, v, stream)
        assert st == _lib.OK, lib.mfwh_last_error()
        assert np.array_equal(got, want), (call, got, want)
    # a third call on a stream that is not torch's current one
    side = torch.cuda.Stream()
    v = torch.from_numpy(rng.normal(size=wl.forcing.shape) * 0.01).cuda()
    want = solver.residual(v)
    side.wait_stream(torch.cuda.current_stream())
    st, got = _noalloc(lib, prob, f, v, side.cuda_stream)
    assert st == _lib.OK, lib.mfwh_last_error()
    assert np.array_equal(got, want), (got, want)
    solver.close()


def test_noalloc_rejects_host_pointers_and_bad_sizes(lib):
    wl = inputs.gaussian_workload("noalloc", (16, 16), 2, [5.5, 9.3], 200.0, 42)
    prob, keep = M.make_problem(wl.n, wl.length, wl.omega)
    host = np.zeros_like(wl.forcing)
    r = np.zeros(2)
    st = lib.mfwh_residual_noalloc(C.byref(prob), C.c_void_p(host.ctypes.data), C.c_void_p(host.ctypes.data),
                                   r.ctypes.data_as(C.POINTER(C.c_double)), None)
    assert st == _lib.ERR_INVALID_ARG
    assert "device" in lib.mfwh_last_error().decode()
    f = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    for field, value in [("order", 3), ("nf", 17)]:
        saved = getattr(prob, field)
        setattr(prob, field, value)
        st = lib.mfwh_residual_noalloc(C.byref(prob), C.c_void_p(f.data_ptr()),
                                       C.c_void_p(f.data_ptr()),
                                       r.ctypes.data_as(C.POINTER(C.c_double)), None)
        assert st == _lib.ERR_INVALID_ARG, field
        setattr(prob, field, saved)
