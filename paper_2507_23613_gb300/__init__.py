"""GB300-native Multi-Frequency WaveHoltz (arXiv 2507.23613): Python binding of libmfwh.

The compute path is the CUDA library libmfwh.so (include/mfwh.h); this package
only marshals arguments.  Device buffers are torch CUDA tensors (float64,
contiguous), host buffers numpy float64 arrays; both hold N_f grid functions
over all grid points, x fastest ([N_f, (nz+1,) ny+1, nx+1]).
"""

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MfwhError  # noqa: F401


def _as_ptr(x):
    """Raw pointer of a torch tensor or numpy array (float64, contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _numel(x):
    return int(x.numel()) if hasattr(x, "numel") else int(x.size)


def _sized(x, count, what):
    """_as_ptr of a buffer that must hold at least count float64 values.  The library reads or
    writes count values through the pointer and cannot check the buffer's size itself, so a
    short buffer is refused here, before any call."""
    ptr = _as_ptr(x)
    if x is not None and _numel(x) < count:
        raise ValueError(f"{what}: {_numel(x)} values, the problem needs {count} "
                         "(nf x grid points)")
    return ptr


def _problem_values(problem):
    """nf x grid points of an mfwh_problem: the length of its [nf][points] buffers."""
    points = 1
    for a in range(problem.dim):
        points *= int(problem.n[a]) + 1
    return int(problem.nf) * points


def _dptr(arr):
    return arr.ctypes.data_as(C.POINTER(C.c_double))


def make_problem(n, length, omega, forcing=None, c_lo=1.0, c_hi=None, interface=0.5,
                 layer_axis=2, n_p=1, cfl=0.5, filter_mode=_lib.FILTER_OPTIMIZED,
                 user_params=None, n_delta=20, c_delta=2.0, time_block=0, precision=None,
                 tile_shape=0, order=2, filter_update=0, time_stepping="explicit",
                 steps_per_period=0, mg_tol=0.0, mg_max_cycles=0, c2_field=None):
    """Fill an mfwh_problem.  Returned keep-alive list holds the arrays it points to.
    time_stepping: "explicit" (leapfrog) or "implicit" (trapezoidal, multigrid solves).
    c2_field: c^2 at every grid point (numpy array or CUDA tensor, float64, grid shape);
    selects MFWH_C_FIELD."""
    p = _lib.Problem()
    p.dim = len(n)
    for a in range(3):
        p.n[a] = int(n[a]) if a < len(n) else 0
        p.length[a] = float(length[a]) if a < len(n) else 0.0
    om = np.ascontiguousarray(omega, dtype=np.float64)
    p.nf = om.size
    p.omega = _dptr(om)
    keep = [om]
    points = 1
    for a in range(len(n)):
        points *= int(n[a]) + 1
    if forcing is not None:
        ptr = _sized(forcing, om.size * points, "forcing")
        p.forcing = C.cast(ptr, C.POINTER(C.c_double))
        keep.append(forcing)
    p.c_mode = _lib.C_CONST if c_hi is None else _lib.C_TWO_LAYER
    if c2_field is not None:
        if c_hi is not None:
            raise ValueError("give either c_hi (two layers) or c2_field, not both")
        p.c_mode = _lib.C_FIELD
        p.c2_field = C.cast(_sized(c2_field, points, "c2_field"), C.POINTER(C.c_double))
        keep.append(c2_field)
    p.c_lo = float(c_lo)
    p.c_hi = float(c_hi if c_hi is not None else c_lo)
    p.interface = float(interface)
    p.layer_axis = int(layer_axis)
    p.n_p = int(n_p)
    p.cfl = float(cfl)
    p.filter_mode = int(filter_mode)
    if user_params is not None:
        up = np.ascontiguousarray(user_params, dtype=np.float64).reshape(-1)
        if int(filter_mode) == _lib.FILTER_USER and up.size < 3 * om.size:
            raise ValueError(f"user_params: {up.size} values, the problem needs {3 * om.size} "
                             "((a, c, s) per frequency)")
        p.user_params = _dptr(up)
        keep.append(up)
    p.n_delta = int(n_delta)
    p.c_delta = float(c_delta)
    p.precision = _lib.PREC_FP64 if precision is None else int(precision)
    p.time_block = int(time_block)
    p.tile_shape = int(tile_shape)
    p.order = int(order)
    p.filter_update = int(filter_update)
    if time_stepping not in ("explicit", "implicit"):
        raise ValueError("time_stepping must be 'explicit' or 'implicit'")
    p.time_stepping = _lib.TIME_IMPLICIT if time_stepping == "implicit" else _lib.TIME_EXPLICIT
    p.steps_per_period = int(steps_per_period)
    p.mg_tol = float(mg_tol)
    p.mg_max_cycles = int(mg_max_cycles)
    return p, keep


def plan(problem):
    s = _lib.Setup()
    _lib.check(_lib.load().mfwh_plan(C.byref(problem), C.byref(s)))
    return s


def plan_multigrid(problem):
    """Multigrid hierarchy of an implicit problem (host only): (levels, coarse, cells), cells a
    list of (nx, ny, nz) per level and coarse the first level solved by one CTA."""
    levels, coarse = C.c_int(), C.c_int()
    cells = (C.c_int64 * 3 * 16)()
    _lib.check(_lib.load().mfwh_plan_multigrid(C.byref(problem), C.byref(levels),
                                               C.byref(coarse), cells))
    return levels.value, coarse.value, [tuple(cells[l]) for l in range(levels.value)]


def plan_weights(problem, n_t, nf):
    w = np.zeros((n_t + 1) * nf)
    _lib.check(_lib.load().mfwh_plan_weights(C.byref(problem), _dptr(w), w.size))
    return w.reshape(n_t + 1, nf)


def adjusted_frequency(omega, dt, alpha=0.0, beta=1.0):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    out = np.zeros_like(om)
    _lib.check(_lib.load().mfwh_adjusted_frequency(om.size, _dptr(om), dt, alpha, beta, _dptr(out)))
    return out


def opt_parameters(omega, n_p, n_t, n_delta=20, c_delta=2.0):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    out = np.zeros((om.size, 3))
    lam = C.c_double()
    nl = C.c_int()
    _lib.check(_lib.load().mfwh_opt_parameters(om.size, _dptr(om), n_p, n_t, n_delta, c_delta,
                                               _dptr(out), C.byref(lam), C.byref(nl)))
    return out, lam.value, nl.value


def mfwh_residual_noalloc(problem, forcing, v, stream=None):
    """Helmholtz residual through the allocation-free entry point (no handle; the
    library's fixed device scratch array).  forcing, v: device tensors."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    r = np.zeros(problem.nf)
    count = _problem_values(problem)
    _lib.check(_lib.load().mfwh_residual_noalloc(C.byref(problem), _sized(forcing, count, "forcing"),
                                                 _sized(v, count, "v"), _dptr(r),
                                                 C.c_void_p(stream)))
    return r


def autotune(n, length, omega, stream=None, **kw):
    """Best (time_block, tile_shape, ms per step) for a problem on the current device."""
    problem, keep = make_problem(n, length, omega, None, **kw)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    tb, shape, ms = C.c_int(), C.c_int(), C.c_double()
    _lib.check(_lib.load().mfwh_autotune(C.byref(problem), C.c_void_p(stream), C.byref(tb),
                                         C.byref(shape), C.byref(ms)))
    return tb.value, shape.value, ms.value


def solve_batch(solvers, vs, restart=20, tol=1e-8, max_iters=1000, raise_on_error=True):
    """Concurrent GMRES solves of independent problems (mfwh_solve_batch).
    Returns (status, per-problem info dicts, per-problem seconds)."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s._handle.value for s in solvers])
    if len(vs) != n:
        raise ValueError("one solution buffer per solver")
    ptrs = (C.c_void_p * n)(*[_sized(v, sv.values, "v").value for sv, v in zip(solvers, vs)])
    infos = (_lib.SolveInfo * n)()
    secs = np.zeros(n)
    st = _lib.load().mfwh_solve_batch(hs, n, int(restart), float(tol), int(max_iters), ptrs,
                                      infos, _dptr(secs))
    if raise_on_error:
        _lib.check(st)
    out = [{"iterations": infos[i].iterations, "pi_applications": infos[i].pi_applications,
            "rel_residual": infos[i].rel_residual,
            "helmholtz_residual": np.array(infos[i].helmholtz_residual[:solvers[i].nf])}
           for i in range(n)]
    return st, out, secs


def solve_batch_graph(solvers, vs, restart=20, tol=1e-8, max_iters=1000, stream=None,
                      raise_on_error=True):
    """Lockstep GMRES of independent problems, one CUDA-graph launch per application of the map
    across the batch (mfwh_solve_batch_graph).  Returns (status, info dicts, seconds)."""
    n = len(solvers)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    hs = (C.c_void_p * n)(*[s._handle.value for s in solvers])
    if len(vs) != n:
        raise ValueError("one solution buffer per solver")
    ptrs = (C.c_void_p * n)(*[_sized(v, sv.values, "v").value for sv, v in zip(solvers, vs)])
    infos = (_lib.SolveInfo * n)()
    secs = np.zeros(n)
    st = _lib.load().mfwh_solve_batch_graph(hs, n, int(restart), float(tol), int(max_iters), ptrs,
                                            infos, _dptr(secs), C.c_void_p(stream))
    if raise_on_error:
        _lib.check(st)
    out = [{"iterations": infos[i].iterations, "pi_applications": infos[i].pi_applications,
            "restarts": infos[i].restarts, "rel_residual": infos[i].rel_residual,
            "helmholtz_residual": np.array(infos[i].helmholtz_residual[:solvers[i].nf])}
           for i in range(n)]
    return st, out, secs


def setup_arrays(s):
    """numpy views of an mfwh_setup's tables, trimmed to nf."""
    nf = s.nf
    return {
        "dt": s.dt, "n_t": s.n_t, "nf": nf,
        "omega_tilde": np.array(s.omega_tilde[:nf]),
        "n_pm": np.array(s.n_pm[:nf]),
        "t_fm": np.array(s.t_fm[:nf]),
        "params": np.array([[s.params[m][k] for k in range(3)] for m in range(nf)]),
        "B": np.array([[s.B[m][j] for j in range(nf)] for m in range(nf)]),
        "B_inv": np.array([[s.B_inv[m][j] for j in range(nf)] for m in range(nf)]),
        "lam_max": s.lam_max, "n_lambda": s.n_lambda,
        "points": s.points, "interior_points": s.interior_points,
    }


class Solver:
    """One MFWH problem on the current CUDA device (an mfwh_handle_t)."""

    def __init__(self, n, length, omega, forcing=None, stream=None, **kw):
        lib = _lib.load()
        self._problem, self._keep = make_problem(n, length, omega, forcing, **kw)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._handle = C.c_void_p()
        _lib.check(lib.mfwh_create(C.byref(self._problem), C.c_void_p(stream), C.byref(self._handle)))
        self._keep = None
        self.nf = len(omega)
        s = _lib.Setup()
        _lib.check(lib.mfwh_get_setup(self._handle, C.byref(s)))
        self.setup = setup_arrays(s)
        self.values = self.nf * int(self.setup["points"])   # length of every [nf][points] buffer

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            _lib.load().mfwh_destroy(self._handle)
            self._handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_forcing(self, forcing):
        _lib.check(_lib.load().mfwh_set_forcing(self._handle,
                                                _sized(forcing, self.values, "forcing")))

    def mfwh_apply_Pi(self, v_in, v_out, forced=True):
        _lib.check(_lib.load().mfwh_apply_Pi(self._handle, _sized(v_in, self.values, "v_in"),
                                             _sized(v_out, self.values, "v_out"), int(forced)))

    apply_Pi = mfwh_apply_Pi

    def solve_fpi(self, v, iters):
        _lib.check(_lib.load().mfwh_solve_fpi(self._handle, int(iters),
                                              _sized(v, self.values, "v")))

    def solve_gmres(self, v, restart=20, tol=1e-8, max_iters=1000, spurious_tol=0.0,
                    history=512, raise_on_error=True):
        info = _lib.SolveInfo()
        hist = np.zeros(max(history, 1))
        info.history_capacity = history
        info.history = _dptr(hist)
        st = _lib.load().mfwh_solve_gmres(self._handle, int(restart), float(tol), int(max_iters),
                                          float(spurious_tol), _sized(v, self.values, "v"),
                                          C.byref(info))
        if raise_on_error:
            _lib.check(st)
        out = {
            "status": st,
            "iterations": info.iterations,
            "pi_applications": info.pi_applications,
            "restarts": info.restarts,
            "rel_residual": info.rel_residual,
            "helmholtz_residual": np.array(info.helmholtz_residual[:self.nf]),
            "history": hist[:info.history_len].copy(),
        }
        return out

    def solve_refined(self, v, target=1e-6, inner_tol=1e-5, restart=200, max_iters=1000,
                      max_refinements=8, history=512, raise_on_error=True):
        """Mixed-precision defect correction to max_m r_h <= target (mfwh_solve_refined)."""
        info = _lib.SolveInfo()
        hist = np.zeros(max(history, 1))
        info.history_capacity = history
        info.history = _dptr(hist)
        st = _lib.load().mfwh_solve_refined(self._handle, int(restart), float(inner_tol),
                                            int(max_iters), float(target), int(max_refinements),
                                            _sized(v, self.values, "v"), C.byref(info))
        if raise_on_error:
            _lib.check(st)
        return {
            "status": st,
            "iterations": info.iterations,
            "pi_applications": info.pi_applications,
            "restarts": info.restarts,
            "refinements": info.refinements,
            "rel_residual": info.rel_residual,
            "helmholtz_residual": np.array(info.helmholtz_residual[:self.nf]),
            "history": hist[:info.history_len].copy(),
        }

    def solve_relaxed(self, v, target=1e-6, inner_tol=1e-6, relax_below=1e-2, restart=200,
                      max_iters=1000, max_refinements=8, history=512, raise_on_error=True):
        """Refinement whose inner solves switch from FP64 to FP32 products once their residual
        is below relax_below (mfwh_solve_relaxed; FP32 handles)."""
        info = _lib.SolveInfo()
        hist = np.zeros(max(history, 1))
        info.history_capacity = history
        info.history = _dptr(hist)
        st = _lib.load().mfwh_solve_relaxed(self._handle, int(restart), float(inner_tol),
                                            float(relax_below), int(max_iters), float(target),
                                            int(max_refinements), _sized(v, self.values, "v"),
                                            C.byref(info))
        if raise_on_error:
            _lib.check(st)
        return {
            "status": st,
            "iterations": info.iterations,
            "pi_applications": info.pi_applications,
            "restarts": info.restarts,
            "refinements": info.refinements,
            "rel_residual": info.rel_residual,
            "helmholtz_residual": np.array(info.helmholtz_residual[:self.nf]),
            "history": hist[:info.history_len].copy(),
        }

    def warm_start_data(self, v, x_out, t_out, omega_scale=45.0):
        """Network inputs [nf][2][H][W] and targets [nf][1][H][W] (float32 device tensors)
        from a solution v of this problem (mfwh_warm_start_data)."""
        vp = _sized(v, self.values, "v")
        CNN._need(x_out, 2 * self.values, "x_out")
        CNN._need(t_out, self.values, "t_out")
        xp, tp = CNN._f32(x_out), CNN._f32(t_out)
        _lib.check(_lib.load().mfwh_warm_start_data(self._handle, float(omega_scale), vp, xp, tp))

    def warm_start(self, net, v, omega_scale=45.0):
        """Write the network's initial iterate into v (mfwh_warm_start); returns (kept, ratio)
        with ratio = ||b - (v - S v)|| / ||b|| of the returned start."""
        ratio = C.c_double()
        st = _lib.load().mfwh_warm_start(self._handle, net._h, float(omega_scale),
                                         _sized(v, self.values, "v"), C.byref(ratio))
        if st not in (_lib.OK, _lib.ERR_NOT_CONVERGED):
            _lib.check(st)
        return st == _lib.OK, ratio.value

    def set_wait_limit(self, seconds):
        """Limit (s) of one grid-barrier wait of the implicit step kernel; <= 0: default 2 s."""
        _lib.check(_lib.load().mfwh_set_wait_limit(self._handle, float(seconds)))

    def set_graphs(self, enable=True):
        _lib.check(_lib.load().mfwh_set_graphs(self._handle, int(bool(enable))))

    def debug_bounds(self):
        """(count, index, extent, line) of the index-checked build's fault record; count is
        -1 for the normal build (no checks compiled)."""
        count, index, extent, line = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int()
        _lib.check(_lib.load().mfwh_debug_bounds(self._handle, C.byref(count), C.byref(index),
                                                 C.byref(extent), C.byref(line)))
        return count.value, index.value, extent.value, line.value

    def residual(self, v):
        r = np.zeros(self.nf)
        _lib.check(_lib.load().mfwh_residual(self._handle, _sized(v, self.values, "v"), _dptr(r)))
        return r

    def last_timing(self):
        ms = C.c_double()
        sl = C.c_int64()
        tl = C.c_int64()
        _lib.check(_lib.load().mfwh_last_timing(self._handle, C.byref(ms), C.byref(sl), C.byref(tl)))
        return ms.value, sl.value, tl.value

    def mg_stats(self, reset=False):
        """Multigrid statistics of an implicit handle: dict with solves, cycles, unconverged,
        levels (accumulated since creation or the last reset)."""
        sv, cy, un = C.c_int64(), C.c_int64(), C.c_int64()
        lv = C.c_int()
        _lib.check(_lib.load().mfwh_mg_stats(self._handle, C.byref(sv), C.byref(cy), C.byref(un),
                                             C.byref(lv), int(bool(reset))))
        return {"solves": sv.value, "cycles": cy.value, "unconverged": un.value,
                "levels": lv.value}


class CNN:
    """The warm-start network (an mfwh_cnn_t): float32 device tensors [B][C][H][W] in and out."""

    def __init__(self, layers=5, channels=32, in_channels=2, seed=0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._h = C.c_void_p()
        _lib.check(_lib.load().mfwh_cnn_create(int(layers), int(channels), int(in_channels),
                                               int(seed), C.c_void_p(stream), C.byref(self._h)))
        self.layers, self.channels, self.in_channels = layers, channels, in_channels
        self.n_params = int(_lib.load().mfwh_cnn_param_count(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().mfwh_cnn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _lib.check(_lib.load().mfwh_cnn_set_params(self._h, a.ctypes.data_as(C.c_void_p), a.size))

    def get_params(self, grads=False):
        p = np.zeros(self.n_params, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32) if grads else None
        _lib.check(_lib.load().mfwh_cnn_get_params(
            self._h, p.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p) if grads else None,
            p.size))
        return (p, g) if grads else p

    @staticmethod
    def _need(t, count, what):
        """The library reads or writes count values through a tensor's pointer and cannot check
        its size: refuse a shorter tensor."""
        if _numel(t) < count:
            raise ValueError(f"{what}: {_numel(t)} values, {count} needed")

    @staticmethod
    def _f32(t):
        import torch
        if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise TypeError("expected a contiguous float32 CUDA tensor")
        return C.c_void_p(t.data_ptr())

    def _images(self, x):
        if len(x.shape) != 4 or x.shape[1] != self.in_channels:
            raise ValueError(f"x: expected [B][{self.in_channels}][H][W], got {tuple(x.shape)}")
        B, _, H, W = x.shape
        return int(B), int(H), int(W)

    def forward(self, x, y):
        B, H, W = self._images(x)
        self._need(y, B * H * W, "y")
        _lib.check(_lib.load().mfwh_cnn_forward(self._h, self._f32(x), B, H, W, self._f32(y)))

    def train_step(self, x, target, mask, lr):
        B, H, W = self._images(x)
        self._need(target, B * H * W, "target")
        self._need(mask, H * W, "mask")
        loss = C.c_float()
        _lib.check(_lib.load().mfwh_cnn_train_step(self._h, self._f32(x), self._f32(target),
                                                   self._f32(mask), B, H, W, float(lr),
                                                   C.byref(loss)))
        return loss.value
