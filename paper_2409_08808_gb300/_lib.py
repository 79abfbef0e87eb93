"""ctypes loader for libgoac.so (the C ABI declared in include/goac.h).

There is no fallback: if the compiled library is missing or cannot be loaded,
importing this module raises.  Build it with ``python -m
paper_2409_08808_gb300.build`` or ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgoac.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libgoac.so not built ({LIB_PATH}); run paper_2409_08808_gb300/build.py")

lib = C.CDLL(LIB_PATH)

_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_u32 = C.c_uint32
_u64 = C.c_uint64
_d = C.c_double
_st = C.c_int32

class GaParams(C.Structure):
    """goac_ga_params"""
    _fields_ = [("P", C.c_int32), ("n_gen", C.c_int32), ("n_elite", C.c_int32), ("p_mut_u32", C.c_uint32),
                ("precision", C.c_int32), ("patience", C.c_int32), ("gen0", C.c_uint32), ("time_budget_s", C.c_double)]


class GaStats(C.Structure):
    """goac_ga_stats"""
    _fields_ = [("generations", C.c_int32), ("best_generation", C.c_int32), ("stop_reason", C.c_int32),
                ("reserved", C.c_int32), ("best_E", C.c_double)]


class McStats(C.Structure):
    """goac_mc_stats (device pointers)"""
    _fields_ = [("n_accept_dev", C.c_void_p), ("n_noop_dev", C.c_void_p), ("best_step_dev", C.c_void_p),
                ("steps_dev", C.c_void_p)]


#: name -> (restype, argtypes); every entry point of include/goac.h
SIGNATURES = {
    "goac_last_error": (C.c_char_p, []),
    "goac_version": (_i32, []),
    "goac_ctx_create": (_st, [_i32, _p, C.POINTER(_p)]),
    "goac_ctx_destroy": (_st, [_p]),
    "goac_ctx_set_stream": (_st, [_p, _p]),
    "goac_ctx_synchronize": (_st, [_p]),
    "goac_ctx_set_timing": (_st, [_p, _i32]),
    "goac_ctx_kernel_time": (_st, [_p, _i32, _p, _p]),
    "goac_launch_count": (_i64, []),
    "goac_selftest_wait_timeout": (_st, [_p, _i64]),
    "goac_build_ewald": (_st, [_p, _p, _p, _i32, _d, _p, _d, _d, _p]),
    "goac_problem_create": (_st, [_p, _p, _i32, _p, _p, _p, _i32, _p, _i32, _i32, C.POINTER(_p)]),
    "goac_problem_destroy": (_st, [_p]),
    "goac_problem_info": (_st, [_p, _p, _p]),
    "goac_problem_phi_fix": (_st, [_p, _p]),
    "goac_score": (_st, [_p, _p, _i32, _i32, _p]),
    "goac_problem_exact_info": (_st, [_p, _p, _p, _p]),
    "goac_score_set_shape": (_st, [_p, _i32, _i32, _i32, _i32, _i32]),
    "goac_score_autotune": (_st, [_p, _p, _i32, _i32, _p, _p, _p, _p]),
    "goac_score_host": (_st, [_p, _p, _i32, _i32, _p]),
    "goac_score_host_async": (_st, [_p, _p, _i32, _i32, _p]),
    "goac_score_f64_noalloc": (_st, [_p, _i32, _i32, _p, _i32, _p, _p, _d, _p, _p]),
    "goac_topk_rescore": (_st, [_p, _p, _i32, _p, _i32, _p, _p]),
    "goac_random_configs": (_st, [_p, _i32, _u64, _p]),
    "goac_mc_run": (_st, [_p, _p, _i32, _p, _i64, _u64, _u64, _i32, _p, _p, _p, _p]),
    "goac_mc_run_ex": (_st, [_p, _p, _i32, _p, _i64, _u64, _u64, _i32, _i64, _p, _p, _p, C.POINTER(McStats)]),
    "goac_gd_run": (_st, [_p, _p, _i32, _i32, _p, _p]),
    "goac_hybrid_run": (_st, [_p, _p, _i32, _i32, _p, _i32, _i32, _i64, _i32, _i32, _u32, _u64, _i32, _p]),
    "goac_sa_run": (_st, [_p, _p, _i32, _p, _p, _i64, _i64, _u64, _u64, _i32, _p, _p, _p, _p]),
    "goac_remc_run": (_st, [_p, _p, _i32, _i32, _p, _i32, _i64, _u64, _i32, _p, _p, _p]),
    "goac_batch_mc_run": (_st, [_p, _p, _i32, _p, _p, _p, _i64, _u64, _u64, _i32, _p, _p, _i32, _i32]),
    "goac_batch_mc_autotune": (_st, [_p, _p, _i32, _p, _p, _p, _i64, _i32, _p, _p]),
    "goac_ga_generation": (_st, [_p, _p, _p, _i32, _i32, _u32, _u32, _u64, _p, _p, _p]),
    "goac_ga_run": (_st, [_p, _p, _p, _i32, _i32, _i32, _u32, _u64, _u32, _i32]),
    "goac_ga_run_ex": (_st, [_p, _p, _p, _i32, C.POINTER(GaParams), _u64, _i32, _p, _p, C.POINTER(GaStats)]),
    "goac_ga_run_populations": (_st, [_p, _p, _p, _i32, _i32, _i32, _i32, _u32, _u64, _u32, _i32]),
    "goac_batch_ga_run": (_st, [_p, _p, _i32, _p, _p, _p, _i32, _i32, _u32, _u64, _u32, _i32]),
    "goac_mc_autotune": (_st, [_p, _p, _i32, _p, _i64, _i32, _p, _p, _p]),
    "goac_mc_set_shape": (_st, [_p, _i32, _i32, _i32]),
    "goac_energy_grad": (_st, [_p, _p, _i32, _d, _i32, _p, _p]),
    "goac_round_to_counts": (_st, [_p, _p, _i32, _p]),
    "goac_occupations": (_st, [_p, _p, _i32, _p]),
    "goac_relaxed_descent": (_st, [_p, _p, _i32, _d, _d, _i32, _i32, _p, _p]),
}

for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
