"""ctypes declarations of libnmfkl's C ABI (include/nmfkl.h).

Loading fails loudly when the CUDA library is missing: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

c_i32, c_i64, c_u64, c_f64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENUMERIC", 5: "ETIMEOUT",
                6: "EBUSY", 7: "ENOTCONV", 8: "ECANCELED"}


class Params(ctypes.Structure):
    _fields_ = [("r", c_i32), ("alpha_W", c_f64), ("beta_W", c_f64), ("alpha_F", c_f64),
                ("beta_F", c_f64), ("eps_grad", c_f64), ("eps_div", c_f64), ("eps_x", c_f64),
                ("max_inner", c_i32), ("grad_mode", c_i32), ("break_mode", c_i32),
                ("perm_mode", c_i32), ("seed", c_u64), ("list_mode", c_i32), ("div_mode", c_i32)]


class Counters(ctypes.Structure):
    _fields_ = [("coords", c_i64), ("evals", c_i64), ("steps", c_i64), ("cap_hits", c_i64)]


class BucketInfo(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char_p), ("side", c_i32), ("count", c_i32), ("nnz", c_i64),
                ("max_len", c_i64), ("grid", c_i32), ("block", c_i32), ("smem", c_i64), ("ran_last", c_i32),
                ("list_plan", c_i32)]


class PlanChoice(ctypes.Structure):
    _fields_ = [("list_threshold", c_f64), ("short_kernel", (c_i32 * 4) * 2)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("device", c_i32), ("slots", c_i32), ("mem_budget", c_i64), ("max_pending", c_i32),
                ("max_batch_docs", c_i32), ("max_batch_nnz", c_i64)]


class Request(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("n", c_i64), ("m", c_i64), ("nnz", c_i64), ("colptr", c_vp), ("rowidx", c_vp),
                ("val", c_vp), ("r", c_i32), ("seed", c_u64), ("rel_tol", c_f64), ("max_sweeps", c_i32),
                ("F_out", c_vp), ("W_out", c_vp), ("sweeps_out", c_vp), ("obj_out", c_vp)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("queued_ms", c_f64), ("run_ms", c_f64), ("batch_requests", c_i32),
                ("message", ctypes.c_char * 160)]


class ServerStats(ctypes.Structure):
    _fields_ = [("pending", c_i64), ("mem_in_use", c_i64), ("batches", c_i64), ("batched_requests", c_i64)]


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("nmfkl_default_params", None, [ctypes.POINTER(Params), c_i32]),
    ("nmfkl_status_string", ctypes.c_char_p, [c_i32]),
    ("nmfkl_create", c_i32, [ctypes.POINTER(Params), c_i64, c_i64, c_i32, c_vp, ctypes.POINTER(c_vp)]),
    ("nmfkl_destroy", None, [c_vp]),
    ("nmfkl_last_error", ctypes.c_char_p, [c_vp]),
    ("nmfkl_set_data", c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i32]),
    ("nmfkl_init", c_i32, [c_vp, c_vp, c_vp, c_i32]),
    ("nmfkl_sweep_F", c_i32, [c_vp, c_i64]),
    ("nmfkl_sweep_W", c_i32, [c_vp, c_i64]),
    ("nmfkl_set_wait_limit", c_i32, [c_vp, c_i64]),
    ("nmfkl_sweep_range", c_i32, [c_vp, c_i32, c_i64, c_i64, c_i64, ctypes.POINTER(c_f64)]),
    ("nmfkl_linear_term", c_i32, [c_vp, ctypes.POINTER(c_f64)]),
    ("nmfkl_factor_unit_major", c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_i64),
                                        ctypes.POINTER(c_i32)]),
    ("nmfkl_objective", c_i32, [c_vp, ctypes.POINTER(c_f64), ctypes.POINTER(c_f64)]),
    ("nmfkl_fit", c_i32, [c_vp, c_i64, c_i32, c_f64, c_vp, ctypes.POINTER(c_i32)]),
    ("nmfkl_step", c_i32, [c_vp, c_i64, ctypes.POINTER(c_f64)]),
    ("nmfkl_plan_info", c_i32, [c_vp, c_vp, c_i32]),
    ("nmfkl_get_plan_choice", c_i32, [c_vp, ctypes.POINTER(PlanChoice)]),
    ("nmfkl_set_plan_choice", c_i32, [c_vp, ctypes.POINTER(PlanChoice)]),
    ("nmfkl_autotune", c_i32, [c_vp, c_i64, c_i32, ctypes.c_char_p, ctypes.POINTER(PlanChoice), c_vp,
                               ctypes.POINTER(c_i32)]),
    ("nmfkl_foldin", c_i32, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_f64, c_i32, c_vp, c_vp,
                             c_i32, c_i32]),
    ("nmfkl_get_W", c_i32, [c_vp, c_vp, c_i32]),
    ("nmfkl_get_F", c_i32, [c_vp, c_vp, c_i32]),
    ("nmfkl_state_bytes", c_i64, [c_vp]),
    ("nmfkl_get_state", c_i32, [c_vp, c_i64, c_vp, c_i64]),
    ("nmfkl_set_state", c_i32, [c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]),
    ("nmfkl_get_counters", c_i32, [c_vp, ctypes.POINTER(Counters), c_i32]),
    ("nmfkl_set_timing", c_i32, [c_vp, c_i32]),
    ("nmfkl_set_metrics", c_i32, [c_vp, ctypes.c_char_p]),
    ("nmfkl_kernel_times", c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_i32]),
    ("nmfkl_debug_perm", c_i32, [c_vp, c_i64, c_i32, c_i64, c_vp, c_vp]),
    ("nmfkl_server_default_cfg", None, [ctypes.POINTER(ServerCfg)]),
    ("nmfkl_server_create", c_i32, [ctypes.POINTER(ServerCfg), ctypes.POINTER(Params), c_i64, c_vp,
                                    ctypes.POINTER(c_vp)]),
    ("nmfkl_server_submit", c_i32, [c_vp, ctypes.POINTER(Request), ctypes.POINTER(c_u64)]),
    ("nmfkl_server_poll", c_i32, [c_vp, c_u64, ctypes.POINTER(Result)]),
    ("nmfkl_server_wait", c_i32, [c_vp, c_u64, ctypes.POINTER(Result)]),
    ("nmfkl_server_stats", c_i32, [c_vp, ctypes.POINTER(ServerStats)]),
    ("nmfkl_server_cancel", c_i32, [c_vp, c_u64]),
    ("nmfkl_server_destroy", None, [c_vp]),
    ("nmfkl_sweep_F_noalloc", c_i32, [ctypes.POINTER(Params), c_i64, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp,
                                      c_vp, c_i64, c_vp]),
]

_lib = None


def library_path() -> str:
    return _build.library_path()


def load(build_if_missing: bool = False):
    """Loads libnmfkl.so; raises if it is absent (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build_cuda()
        else:
            raise RuntimeError("libnmfkl.so is not built (%s); run __graft_entry__.build() or "
                               "paper_1604_04026_gb300._build.build_cuda()" % path)
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
