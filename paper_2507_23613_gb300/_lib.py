"""ctypes binding of libmfwh (include/mfwh.h): argument marshalling only.

Every function of the C ABI is exposed under its own name.  Loading fails
loudly when the shared library has not been built: there is no fallback path.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# MFWH_LIBRARY selects another build of the library (the index-checked libmfwh_bc.so).
LIB_PATH = os.environ.get("MFWH_LIBRARY") or os.path.join(HERE, "libmfwh.so")

MAX_NF = 16

OK = 0
ERR_INVALID_ARG = 1
ERR_SINGULAR = 2
ERR_CUDA = 3
ERR_NOMEM = 4
ERR_NOT_CONVERGED = 5
ERR_SPURIOUS = 6
ERR_NONFINITE = 7
ERR_TIMEOUT = 8

FILTER_OPTIMIZED = 0
FILTER_TRADITIONAL = 1
FILTER_USER = 2
PREC_FP64 = 0
PREC_FP32_KAHAN = 1
PREC_FP32_BLOCKSUM = 2
UPDATE_IMPLICIT = 0
UPDATE_EXPLICIT = 1
C_CONST = 0
C_TWO_LAYER = 1
C_FIELD = 2
TIME_EXPLICIT = 0
TIME_IMPLICIT = 1

_dp = C.POINTER(C.c_double)


class Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_int64 * 3),
        ("length", C.c_double * 3),
        ("nf", C.c_int),
        ("omega", _dp),
        ("forcing", _dp),
        ("c_mode", C.c_int),
        ("c_lo", C.c_double),
        ("c_hi", C.c_double),
        ("interface", C.c_double),
        ("layer_axis", C.c_int),
        ("n_p", C.c_int),
        ("cfl", C.c_double),
        ("filter_mode", C.c_int),
        ("user_params", _dp),
        ("n_delta", C.c_int),
        ("c_delta", C.c_double),
        ("precision", C.c_int),
        ("time_block", C.c_int),
        ("order", C.c_int),
        ("filter_update", C.c_int),
        ("tile_shape", C.c_int),
        ("time_stepping", C.c_int),
        ("steps_per_period", C.c_int),
        ("mg_tol", C.c_double),
        ("mg_max_cycles", C.c_int),
        ("c2_field", _dp),
    ]


class Setup(C.Structure):
    _fields_ = [
        ("dt", C.c_double),
        ("n_t", C.c_int),
        ("nf", C.c_int),
        ("h", C.c_double * 3),
        ("omega_tilde", C.c_double * MAX_NF),
        ("n_pm", C.c_int * MAX_NF),
        ("t_fm", C.c_double * MAX_NF),
        ("params", (C.c_double * 3) * MAX_NF),
        ("B", (C.c_double * MAX_NF) * MAX_NF),
        ("B_inv", (C.c_double * MAX_NF) * MAX_NF),
        ("lam_max", C.c_double),
        ("n_lambda", C.c_int),
        ("points", C.c_int64),
        ("interior_points", C.c_int64),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iterations", C.c_int),
        ("pi_applications", C.c_int),
        ("restarts", C.c_int),
        ("rel_residual", C.c_double),
        ("helmholtz_residual", C.c_double * MAX_NF),
        ("history_len", C.c_int),
        ("history_capacity", C.c_int),
        ("history", _dp),
        ("refinements", C.c_int),
    ]


_SIGNATURES = {
    "mfwh_plan": (C.c_int, [C.POINTER(Problem), C.POINTER(Setup)]),
    "mfwh_plan_weights": (C.c_int, [C.POINTER(Problem), _dp, C.c_int64]),
    "mfwh_adjusted_frequency": (C.c_int, [C.c_int, _dp, C.c_double, C.c_double, C.c_double, _dp]),
    "mfwh_opt_parameters": (C.c_int, [C.c_int, _dp, C.c_int, C.c_int, C.c_int, C.c_double, _dp,
                                      _dp, C.POINTER(C.c_int)]),
    "mfwh_create": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.POINTER(C.c_void_p)]),
    "mfwh_set_forcing": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mfwh_apply_Pi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mfwh_solve_fpi": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mfwh_solve_gmres": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double,
                                   C.c_void_p, C.POINTER(SolveInfo)]),
    "mfwh_solve_refined": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double,
                                     C.c_int, C.c_void_p, C.POINTER(SolveInfo)]),
    "mfwh_solve_relaxed": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int,
                                     C.c_double, C.c_int, C.c_void_p, C.POINTER(SolveInfo)]),
    "mfwh_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "mfwh_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_double, C.c_int,
                                   C.POINTER(C.c_void_p), C.POINTER(SolveInfo), _dp]),
    "mfwh_solve_batch_graph": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_double,
                                         C.c_int, C.POINTER(C.c_void_p), C.POINTER(SolveInfo),
                                         _dp, C.c_void_p]),
    "mfwh_autotune": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "mfwh_cnn_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_void_p,
                                  C.POINTER(C.c_void_p)]),
    "mfwh_cnn_param_count": (C.c_int64, [C.c_void_p]),
    "mfwh_cnn_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "mfwh_cnn_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "mfwh_cnn_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "mfwh_cnn_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                      C.c_int, C.c_int, C.c_float, C.POINTER(C.c_float)]),
    "mfwh_cnn_destroy": (None, [C.c_void_p]),
    "mfwh_warm_start_data": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "mfwh_warm_start": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                  C.POINTER(C.c_double)]),
    "mfwh_residual": (C.c_int, [C.c_void_p, C.c_void_p, _dp]),
    "mfwh_residual_noalloc": (C.c_int, [C.POINTER(Problem), C.c_void_p, C.c_void_p, _dp, C.c_void_p]),
    "mfwh_get_setup": (C.c_int, [C.c_void_p, C.POINTER(Setup)]),
    "mfwh_last_timing": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mfwh_plan_multigrid": (C.c_int, [C.POINTER(Problem), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int64 * 3)]),
    "mfwh_mg_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64), C.POINTER(C.c_int), C.c_int]),
    "mfwh_set_wait_limit": (C.c_int, [C.c_void_p, C.c_double]),
    "mfwh_debug_bounds": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "mfwh_destroy": (None, [C.c_void_p]),
    "mfwh_last_error": (C.c_char_p, []),
    "mfwh_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libmfwh.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmfwh.so not built at {path}; run paper_2507_23613_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    return list(_SIGNATURES)


class MfwhError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} [status {status}]")
        self.status = status


def check(status):
    if status != OK:
        lib = load()
        raise MfwhError(status, lib.mfwh_last_error().decode(errors="replace"))
    return status


def __getattr__(name):
    # mfwh_* functions by their C names, e.g. _lib.mfwh_plan(...)
    if name.startswith("mfwh_"):
        return getattr(load(), name)
    raise AttributeError(name)
