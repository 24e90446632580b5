"""ctypes declarations of the C ABI in include/pdlp.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdlp_b300.so")

OK, EINVAL, ENOMEM, ECUDA, EINTERNAL = 0, -1, -2, -3, -5
OPTIMAL, ITER_LIMIT, TIME_LIMIT, NUMERICAL = 0, 1, 2, 3
FP64, MIXED = 0, 1


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("time_limit_s", C.c_double),
                ("check_every", C.c_int32), ("scaling", C.c_int32), ("beta_suff", C.c_double),
                ("beta_nec", C.c_double), ("beta_art", C.c_double), ("step_scale", C.c_double),
                ("omega_theta", C.c_double), ("ruiz_iters", C.c_int32), ("power_iters", C.c_int32),
                ("eta", C.c_double), ("tile_slots", C.c_int32), ("inputs_on_device", C.c_int32),
                ("stream", C.c_void_p), ("log_capacity", C.c_int32), ("tile_chunks", C.c_int32),
                ("spmv_batch", C.c_int32), ("precision", C.c_int32),
                ("mixed_switch_tol", C.c_double), ("cluster_ctas", C.c_int32), ("resident", C.c_int32),
                ("step_rule", C.c_int32), ("engine", C.c_int32), ("batch_tail_iters", C.c_int64),
                ("host_layout", C.c_int32), ("spmv_stage", C.c_int32),
                ("batch_tune", C.c_int32), ("mixed_values", C.c_int32), ("adaptive_reject_cap", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("which", C.c_int32), ("iters", C.c_int64),
                ("restarts", C.c_int64), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("rel_primal", C.c_double), ("rel_dual", C.c_double), ("rel_gap", C.c_double),
                ("kkt_omega", C.c_double), ("omega", C.c_double), ("eta", C.c_double),
                ("solve_s", C.c_double), ("device_ms", C.c_double), ("launches", C.c_int64),
                ("fp32_iters", C.c_int64), ("accepted", C.c_int64)]


class CheckRecord(C.Structure):
    _fields_ = [("k", C.c_int64), ("t", C.c_int64), ("restart", C.c_int32), ("candidate", C.c_int32),
                ("omega", C.c_double), ("kkt_cur", C.c_double), ("kkt_avg", C.c_double),
                ("kkt_anchor", C.c_double), ("rel_primal", C.c_double), ("rel_dual", C.c_double),
                ("rel_gap", C.c_double)]


class Info(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("m1", C.c_int64), ("nnz", C.c_int64),
                ("slots_K", C.c_int64), ("slots_Kt", C.c_int64), ("tasks_K", C.c_int64),
                ("tasks_Kt", C.c_int64), ("split_chunks_K", C.c_int64), ("split_chunks_Kt", C.c_int64),
                ("tile_slots_K", C.c_int32), ("tile_slots_Kt", C.c_int32),
                ("tile_chunks_K", C.c_int32), ("tile_chunks_Kt", C.c_int32),
                ("spmv_batch_K", C.c_int32), ("spmv_batch_Kt", C.c_int32),
                ("algorithmic_bytes_per_iter", C.c_double), ("stored_bytes_per_iter", C.c_double),
                ("eta", C.c_double), ("omega0", C.c_double), ("norm_K", C.c_double),
                ("batch_team", C.c_int32), ("batch_resident", C.c_int32),
                ("wide_rows_K", C.c_int32), ("batch_resumed", C.c_int32),
                ("setup_validate_ms", C.c_double), ("setup_layout_ms", C.c_double),
                ("setup_device_ms", C.c_double), ("setup_tune_ms", C.c_double), ("setup_step_ms", C.c_double),
                ("spmv_stage_K", C.c_int32), ("spmv_stage_Kt", C.c_int32), ("batch_tuned", C.c_int32),
                ("tune_team", C.c_int32 * 8), ("tune_resident", C.c_int32 * 8), ("tune_gbs", C.c_double * 8),
                ("mixed_values", C.c_int32)]


# every function declared in include/pdlp.h: name -> (restype, argtypes)
_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
SIGNATURES = {
    "pdlp_default_params": (None, [C.POINTER(Params)]),
    "pdlp_setup": (C.c_int, [C.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                             C.POINTER(Params)]),
    "pdlp_solve": (C.c_int, [_vp, C.POINTER(Params), _vp, _vp, _d, C.POINTER(Result), _vp, _vp]),
    "pdlp_free": (None, [_vp]),
    "pdlp_last_error": (C.c_char_p, [_vp]),
    "pdlp_get_iterate": (C.c_int, [_vp, _i32, _vp, _vp]),
    "pdlp_get_restarts": (C.c_int64, [_vp, _vp, _i64]),
    "pdlp_get_log": (C.c_int64, [_vp, C.POINTER(CheckRecord), _i64]),
    "pdlp_spmv": (C.c_int, [_vp, _i32, _vp, _vp]),
    "pdlp_bound_duals": (C.c_int, [_vp, _vp, _vp]),
    "pdlp_get_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "pdlp_time_iterations": (C.c_int, [_vp, _i64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pdlp_spmv_csr_noalloc": (C.c_int, [_i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pdlp_batch_setup": (C.c_int, [C.POINTER(_vp), _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                   C.POINTER(Params)]),
    "pdlp_batch_solve": (C.c_int, [_vp, C.POINTER(Params), _vp, _vp, _vp, _vp, _vp, _vp]),
    "pdlp_batch_get_restarts": (C.c_int64, [_vp, _i64, _vp, _i64]),
    "pdlp_state_size": (C.c_int64, [_vp]),
    "pdlp_get_state": (C.c_int, [_vp, _vp, _i64]),
    "pdlp_solve_resume": (C.c_int, [_vp, C.POINTER(Params), _vp, _i64, C.POINTER(Result), _vp, _vp]),
    "pdlp_tc_gemm": (C.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _i32, _vp]),
    "pdlp_tc_gemm_split": (C.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "pdlp_tc_gemm_wait_selftest": (C.c_int, [_vp, _vp, _vp, _i64, _vp]),
    "pdlp_mlp_create": (C.c_int, [C.POINTER(_vp), _i32, _i32, _i32, _i32]),
    "pdlp_mlp_free": (None, [_vp]),
    "pdlp_mlp_last_error": (C.c_char_p, [_vp]),
    "pdlp_mlp_set_params": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pdlp_mlp_get_params": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pdlp_mlp_load_data": (C.c_int, [_vp, _i64, _vp, _vp]),
    "pdlp_mlp_forward": (C.c_int, [_vp, _i32, _vp, _vp]),
    "pdlp_mlp_gradients": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pdlp_mlp_train": (C.c_int, [_vp, _i32, _i32, C.c_float, C.c_float, C.c_uint64, _vp, _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the native library; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"native solver library not built: {path} (run paper_2312_14832_b300/build.py)")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
