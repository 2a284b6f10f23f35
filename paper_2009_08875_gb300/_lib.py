"""ctypes binding of libst (include/st.h).  Argument marshalling only: every computation
happens in the CUDA library; torch tensors supply device memory and the stream."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libst.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "st.h")

ST_OK, ST_ERR_ARG, ST_ERR_NOMEM, ST_ERR_CUDA, ST_ERR_BREAKDOWN, ST_ERR_MAXIT, ST_ERR_TIMEOUT, ST_ERR_CANCELLED = range(8)
STATUS_NAMES = {0: "ST_OK", 1: "ST_ERR_ARG", 2: "ST_ERR_NOMEM", 3: "ST_ERR_CUDA", 4: "ST_ERR_BREAKDOWN",
                5: "ST_ERR_MAXIT", 6: "ST_ERR_TIMEOUT", 7: "ST_ERR_CANCELLED"}


class StConfig(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("n_vcycles", ctypes.c_int), ("n_pre", ctypes.c_int),
                ("n_post", ctypes.c_int), ("tol", ctypes.c_double), ("tol_mode", ctypes.c_int),
                ("maxit", ctypes.c_int), ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("diffusion", ctypes.c_double * 3), ("reaction", ctypes.c_double),
                ("initial_guess", ctypes.c_int)]


class StSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int), ("relres", ctypes.c_double)]


ST_FP64, ST_MIXED_FP32, ST_MIXED_PRECOND, ST_MIXED_BF16, ST_FP64_DF = 0, 1, 2, 3, 4


class StProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("sweep_launches", ctypes.c_int64), ("sweep_ms", ctypes.c_double),
                ("sweep_fp64_ops", ctypes.c_double), ("sweep_bytes", ctypes.c_double),
                ("diag_launches", ctypes.c_int64), ("diag_ms", ctypes.c_double),
                ("diag_fp64_ops", ctypes.c_double), ("diag_bytes", ctypes.c_double),
                ("f32_launches", ctypes.c_int64), ("f32_ms", ctypes.c_double), ("f32_bytes", ctypes.c_double),
                ("f32_diag_launches", ctypes.c_int64), ("f32_diag_ms", ctypes.c_double),
                ("f32_diag_bytes", ctypes.c_double)]


# st_comm: the communicator callbacks of st_sharded_solve
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_void_p),
                               ctypes.POINTER(ctypes.c_int64))


class StComm(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("allreduce_sum", ALLREDUCE_FN), ("exchange", EXCHANGE_FN)]


class STError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "st_default_config": (None, [ctypes.POINTER(StConfig)]),
    "st_setup": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(StConfig), _P]),
    "st_setup_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(StConfig), _P]),
    "st_batch_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "st_problem_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(StSolveInfo), ctypes.POINTER(ctypes.c_int)]),
    "st_destroy": (ctypes.c_int, [_P]),
    "st_dims": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "st_apply_Kx": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "st_apply_Kx_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "st_apply_S_nodal": (ctypes.c_int, [_P, _P, _P]),
    "st_synthesize": (ctypes.c_int, [_P, _P, _P]),
    "st_analyze": (ctypes.c_int, [_P, _P, _P]),
    "st_apply_S": (ctypes.c_int, [_P, _P, _P]),
    "st_apply_KX": (ctypes.c_int, [_P, _P, _P]),
    "st_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "st_pcg_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "st_solve_info_get": (ctypes.c_int, [_P, ctypes.POINTER(StSolveInfo)]),
    "st_apply_S_f32": (ctypes.c_int, [_P, _P, _P]),
    "st_apply_KX_f32": (ctypes.c_int, [_P, _P, _P]),
    "st_apply_KX_bf16": (ctypes.c_int, [_P, _P, _P]),
    "st_solve_host": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double)]),
    "st_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "st_rows_nodal": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _P, _P, _P]),
    "st_rows_KX": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "st_wavelet_cols": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, _P, _P]),
    "st_vec_dot": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "st_vec_axpby": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, ctypes.c_double, _P]),
    "st_nested_solve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, _P, _P,
                                       ctypes.POINTER(ctypes.c_int)]),
    "st_set_smoother": (ctypes.c_int, [_P, ctypes.c_int]),
    "st_set_wave_rows": (ctypes.c_int, [_P, ctypes.c_int]),
    "st_profile_begin": (ctypes.c_int, [_P]),
    "st_profile_end": (ctypes.c_int, [_P, ctypes.POINTER(StProfile)]),
    "st_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(StConfig)]),
    "st_batch_add": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                    ctypes.POINTER(ctypes.c_int)]),
    "st_batch_run": (ctypes.c_int, [_P]),
    "st_batch_problem_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(StSolveInfo),
                                             ctypes.POINTER(ctypes.c_int)]),
    "st_batch_buckets": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "st_batch_destroy": (ctypes.c_int, [_P]),
    "st_server_start": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(StConfig), ctypes.c_int, ctypes.c_double]),
    "st_server_submit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "st_server_poll": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(StSolveInfo), ctypes.POINTER(ctypes.c_double)]),
    "st_server_submit_deadline": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                                 ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]),
    "st_server_cancel": (ctypes.c_int, [_P, ctypes.c_int64]),
    "st_server_stop": (ctypes.c_int, [_P]),
    "st_probe_fma_rates": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "st_sharded_solve": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]),
    "st_last_error": (ctypes.c_char_p, []),
}


def load():
    """Load libst.so; raises ImportError if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libst.so not found at {LIB_PATH}: run __graft_entry__.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status):
    if status != ST_OK:
        raise STError(status, load().st_last_error().decode())
    return status
