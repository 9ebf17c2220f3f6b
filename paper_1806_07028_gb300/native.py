"""ctypes view of the C ABI declared in include/pcamg.h (argument marshalling only).

The library is ``_build/libpcamg.so`` built by :func:`paper_1806_07028_gb300.build.build`
(nvcc, sm_103a). There is no fallback: if the library is missing, every call
raises :class:`NativeLibraryMissing`.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpcamg.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_NOT_LAPLACIAN, ERR_OOM, ERR_CUDA, ERR_ROUND_CAP, ERR_SINGULAR, \
    ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_COARSE_TOO_BIG, ERR_UNSUPPORTED = range(11)
FP64, FP32_IR = 0, 1
START_RANDOM, START_USER, START_LEARNED, START_MWM = 0, 1, 2, 3
P1_E_SCALED, P1_BOOLEAN = 0, 1

# every entry point of include/pcamg.h
EXPORTS = [
    "pcamg_default_params", "pcamg_setup", "pcamg_adapt", "pcamg_solve", "pcamg_solve_zero_rhs",
    "pcamg_solve_host", "pcamg_cycle", "pcamg_smooth_error", "pcamg_start_vector",
    "pcamg_num_hierarchies", "pcamg_num_levels", "pcamg_level_sizes", "pcamg_export_level",
    "pcamg_export_reweighted", "pcamg_last_error", "pcamg_status_string", "pcamg_destroy",
    "pcamg_residual", "pcamg_residual_f32", "pcamg_uniform", "pcamg_colour",
    "pcamg_kernel_launches", "pcamg_residual_noalloc", "pcamg_last_smooth_error",
    "pcamg_mpnn_num_params", "pcamg_mpnn_create", "pcamg_mpnn_destroy", "pcamg_mpnn_get_params",
    "pcamg_mpnn_set_params", "pcamg_mpnn_get_grad", "pcamg_mpnn_forward", "pcamg_mpnn_loss_grad",
    "pcamg_mpnn_adam_step", "pcamg_mpnn_save", "pcamg_mpnn_load", "pcamg_set_allocator",
    "pcamg_trim_memory", "pcamg_solve_multi",
]


class NativeLibraryMissing(RuntimeError):
    pass


class PCAMGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("threshold", C.c_double),
                ("numW", C.c_int32), ("iterW", C.c_int32), ("iterV", C.c_int32),
                ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("relax_sweeps", C.c_int32),
                ("seed", C.c_uint64), ("n_min", C.c_int32), ("max_levels", C.c_int32),
                ("round_cap", C.c_int32), ("p1_mode", C.c_int32), ("precision", C.c_int32),
                ("start", C.c_int32), ("dense_max", C.c_int32), ("use_graphs", C.c_int32),
                ("keep_setup", C.c_int32), ("profile", C.c_int32), ("tail_rows", C.c_int32),
                ("l1jac_rows", C.c_int32), ("tail_dense", C.c_int32), ("max_resetups", C.c_int32),
                ("mpnn", C.c_void_p), ("update_mode", C.c_int32), ("max_cover_rounds", C.c_int32),
                ("outer", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("resetups", C.c_int32), ("levels", C.c_int32),
                ("status", C.c_int32), ("rel_res", C.c_double), ("oc_mean", C.c_double),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("t_alg2_ms", C.c_double), ("t_alg4_ms", C.c_double), ("cycles", C.c_int64),
                ("res_hist", C.POINTER(C.c_double)), ("res_hist_cap", C.c_int32),
                ("res_hist_len", C.c_int32), ("prof_launches", C.c_int64),
                ("prof_ms", C.c_double), ("prof_bytes", C.c_double),
                ("rebuilt", C.POINTER(C.c_int32)), ("wcycles", C.c_int64),
                ("cyc_launches", C.c_int64), ("cyc_ms", C.c_double), ("cyc_bytes", C.c_double),
                ("gs_sweeps", C.c_int64), ("gs_ms", C.c_double), ("gs_bytes", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise NativeLibraryMissing(
                    f"{LIB_PATH} is not built; run paper_1806_07028_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            P = C.POINTER
            sig = {
                "pcamg_default_params": ([P(Params)], i32),
                "pcamg_setup": ([P(vp), P(Params), i32, i64, vp, vp, vp, vp, vp], i32),
                "pcamg_adapt": ([vp, vp], i32),
                "pcamg_solve": ([vp, vp, vp, P(Stats)], i32),
                "pcamg_solve_zero_rhs": ([vp, vp, P(Stats)], i32),
                "pcamg_solve_multi": ([vp, i32, vp, vp, vp, vp], i32),
                "pcamg_solve_host": ([P(Params), i32, i64, vp, vp, vp, vp, vp, P(Stats), vp], i32),
                "pcamg_cycle": ([vp, i32, i32, vp, vp], i32),
                "pcamg_smooth_error": ([vp, vp, vp], i32),
                "pcamg_start_vector": ([vp, vp], i32),
                "pcamg_num_hierarchies": ([vp], i32),
                "pcamg_num_levels": ([vp, i32], i32),
                "pcamg_level_sizes": ([vp, i32, i32, vp], i32),
                "pcamg_export_level": ([vp, i32, i32] + [vp] * 8, i32),
                "pcamg_export_reweighted": ([vp, i32, i32, vp, vp, vp], i32),
                "pcamg_last_error": ([vp], C.c_char_p),
                "pcamg_status_string": ([i32], C.c_char_p),
                "pcamg_destroy": ([vp], None),
                "pcamg_residual": ([i32, vp, vp, vp, vp, vp, vp, vp, vp], i32),
                "pcamg_residual_f32": ([i32, vp, vp, vp, vp, vp, vp, vp], i32),
                "pcamg_uniform": ([u64, i64, vp, vp], i32),
                "pcamg_colour": ([i32, vp, vp, u64, vp, P(i32), vp], i32),
                "pcamg_kernel_launches": ([], i64),
                "pcamg_residual_noalloc": ([i32, vp, vp, vp, vp, vp, vp, vp, vp], i32),
                "pcamg_last_smooth_error": ([vp, vp], i32),
                "pcamg_mpnn_num_params": ([], i64),
                "pcamg_mpnn_create": ([P(vp), vp], i32),
                "pcamg_mpnn_destroy": ([vp], None),
                "pcamg_mpnn_get_params": ([vp, vp], i32),
                "pcamg_mpnn_set_params": ([vp, vp], i32),
                "pcamg_mpnn_get_grad": ([vp, vp], i32),
                "pcamg_mpnn_forward": ([vp, vp, vp, vp], i32),
                "pcamg_mpnn_loss_grad": ([vp, vp, vp, vp, P(dbl)], i32),
                "pcamg_mpnn_adam_step": ([vp, C.c_float], i32),
                "pcamg_mpnn_save": ([vp, C.c_char_p], i32),
                "pcamg_mpnn_load": ([P(vp), C.c_char_p], i32),
                "pcamg_set_allocator": ([vp, vp, vp], i32),
                "pcamg_trim_memory": ([], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def status_name(s):
    try:
        return lib().pcamg_status_string(s).decode()
    except NativeLibraryMissing:
        return str(s)


def check(status, handle=None):
    if status != OK:
        msg = lib().pcamg_last_error(handle).decode(errors="replace")
        raise PCAMGError(status, msg)
