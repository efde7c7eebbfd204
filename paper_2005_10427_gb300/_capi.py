"""ctypes declarations of include/qsd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

MAX_ORDER = 8

QSD_OK = 0
STATUS_NAMES = {
    0: "QSD_OK", 1: "QSD_ERR_INVALID_ARGUMENT", 2: "QSD_ERR_UNSUPPORTED",
    3: "QSD_ERR_OUT_OF_MEMORY", 4: "QSD_ERR_CUDA", 5: "QSD_ERR_UNSORTED_INPUT",
    6: "QSD_ERR_COORD_OUT_OF_RANGE", 7: "QSD_ERR_TIMEOUT", 8: "QSD_ERR_BUDGET",
    9: "QSD_ERR_WORKSPACE_TOO_SMALL",
}


class Coords(ctypes.Structure):
    _fields_ = [("buf", ctypes.c_void_p * 2), ("stride", ctypes.c_int64),
                ("selector", ctypes.c_int)]


class Values(ctypes.Structure):
    _fields_ = [("buf", ctypes.c_void_p * 2), ("elem_bytes", ctypes.c_int),
                ("selector", ctypes.c_int)]


class PlanOptions(ctypes.Structure):
    _fields_ = [("validate", ctypes.c_int), ("digit_bits", ctypes.c_int),
                ("local_capacity", ctypes.c_int), ("no_skip", ctypes.c_int),
                ("tile", ctypes.c_int), ("chunk_tiles", ctypes.c_int),
                ("global_groups", ctypes.c_int), ("top_k", ctypes.c_int),
                ("key_index", ctypes.c_int), ("first_digit_bits", ctypes.c_int)]


_A = ctypes.c_int * MAX_ORDER


class PlanInfo(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("input_mode_order", _A), ("target_perm", _A),
                ("num_calls", ctypes.c_int), ("num_bucketed_calls", ctypes.c_int),
                ("call_prefix_len", _A), ("call_mode", _A), ("num_groups", ctypes.c_int),
                ("group_prefix_len", _A), ("group_num_keys", _A), ("group_key_bits", _A),
                ("group_digit_passes", _A), ("local_capacity", ctypes.c_int),
                ("group_key_index", _A)]


class ProfileRecord(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 32), ("group", ctypes.c_int), ("pass_", ctypes.c_int),
                ("entries", ctypes.c_int64), ("algo_bytes", ctypes.c_int64),
                ("ms", ctypes.c_float)]


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("nnz", ctypes.c_int64),
                ("in_", ctypes.c_void_p), ("in_stride", ctypes.c_int64),
                ("in_vals", ctypes.c_void_p), ("out", ctypes.c_void_p * 2),
                ("out_stride", ctypes.c_int64), ("out_vals", ctypes.c_void_p * 2)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("digit_bits", ctypes.c_int), ("local_capacity", ctypes.c_int),
                ("tile", ctypes.c_int), ("chunk_tiles", ctypes.c_int),
                ("no_graph", ctypes.c_int), ("use_tuned", ctypes.c_int)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("streams", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("val_bytes", ctypes.c_int), ("batch", BatchOptions)]


class ServerResult(ctypes.Structure):
    _fields_ = [("request", ctypes.c_int64), ("tensor", ctypes.c_int), ("status", ctypes.c_int),
                ("coords", ctypes.c_void_p), ("stride", ctypes.c_int64),
                ("vals", ctypes.c_void_p), ("nnz", ctypes.c_int64),
                ("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("released", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("entries_completed", ctypes.c_int64),
                ("queue_depth", ctypes.c_int), ("max_queue_depth", ctypes.c_int),
                ("inflight", ctypes.c_int), ("max_inflight_seen", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t)]


class Csf(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p * MAX_ORDER), ("ptr", ctypes.c_void_p * (MAX_ORDER + 1))]


# (name, restype, argtypes) for every entry point of include/qsd.h
P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
SIGNATURES = [
    ("qsd_plan", I, [I, P, P, P, ctypes.POINTER(P)]),
    ("qsd_plan_ex", I, [I, P, P, P, ctypes.POINTER(PlanOptions), ctypes.POINTER(P)]),
    ("qsd_plan_get_info", I, [P, ctypes.POINTER(PlanInfo)]),
    ("qsd_plan_destroy", None, [P]),
    ("qsd_workspace_bytes", I, [P, I64, ctypes.POINTER(ctypes.c_size_t)]),
    ("qsd_transpose", I, [ctypes.POINTER(Coords), ctypes.POINTER(Values), I64, P, P]),
    ("qsd_transpose_ws", I, [ctypes.POINTER(Coords), ctypes.POINTER(Values), I64, P, P,
                             ctypes.c_size_t, P]),
    ("qsd_transpose_from_ws", I, [P, I64, P, ctypes.POINTER(Coords), ctypes.POINTER(Values),
                                  I64, P, P, ctypes.c_size_t, P]),
    ("qsd_transpose_noalloc", I, [ctypes.POINTER(Coords), ctypes.POINTER(Values), I64, P, P]),
    ("qsd_transpose_host", I, [P, I64, P, P, I64, P, I64, P, ctypes.POINTER(Coords),
                               ctypes.POINTER(Values), P, ctypes.c_size_t, P]),
    ("qsd_transpose_host_async", I, [P, I64, P, P, I64, P, I64, P, ctypes.POINTER(Coords),
                                     ctypes.POINTER(Values), P, ctypes.c_size_t, P]),
    ("qsd_workspace_status", I, [P, P, ctypes.POINTER(I)]),
    ("qsd_get_async_status", I, [P, ctypes.POINTER(I)]),
    ("qsd_exec_create", I, [P, I64, P, ctypes.POINTER(Coords), ctypes.POINTER(Values), I64, P,
                            P, ctypes.c_size_t, ctypes.POINTER(P)]),
    ("qsd_exec_launch", I, [P, P, ctypes.POINTER(I), ctypes.POINTER(I)]),
    ("qsd_exec_destroy", None, [P]),
    ("qsd_debug_set_spin_limit_ns", I, [ctypes.c_uint64]),
    ("qsd_debug_set_stall", I, [I]),
    ("qsd_plan_tune_workspace_bytes", I, [P, I64, ctypes.POINTER(ctypes.c_size_t)]),
    ("qsd_plan_tune", I, [P, P, I64, P, ctypes.POINTER(Coords), ctypes.POINTER(Values), I64, P,
                          ctypes.c_size_t, P, I, ctypes.POINTER(PlanOptions),
                          ctypes.POINTER(ctypes.c_float)]),
    ("qsd_csf_workspace_bytes", I, [I, I64, ctypes.POINTER(ctypes.c_size_t)]),
    ("qsd_csf_build", I, [P, I64, I64, I, P, ctypes.POINTER(Csf), P, P, ctypes.c_size_t, P]),
    ("qsd_transpose_csf_workspace_bytes", I, [P, I64, ctypes.POINTER(ctypes.c_size_t)]),
    ("qsd_transpose_csf_from_ws", I, [P, I64, P, ctypes.POINTER(Coords), ctypes.POINTER(Values),
                                      I64, P, ctypes.POINTER(Csf), P, P, ctypes.c_size_t, P]),
    ("qsd_batch_create", I, [ctypes.POINTER(BatchItem), I, I, ctypes.POINTER(BatchOptions),
                             ctypes.POINTER(P)]),
    ("qsd_batch_workspace_bytes", I, [P, ctypes.POINTER(ctypes.c_size_t)]),
    ("qsd_batch_run", I, [P, P, ctypes.c_size_t, P]),
    ("qsd_batch_result", I, [P, I, ctypes.POINTER(I)]),
    ("qsd_batch_get_options", I, [P, ctypes.POINTER(BatchOptions)]),
    ("qsd_batch_tune", I, [P, P, ctypes.c_size_t, P, I, ctypes.POINTER(BatchOptions)]),
    ("qsd_tune_cache_save", I, [ctypes.c_char_p]),
    ("qsd_tune_cache_load", I, [ctypes.c_char_p]),
    ("qsd_batch_destroy", None, [P]),
    ("qsd_server_create", I, [ctypes.POINTER(ServerOptions), ctypes.POINTER(P)]),
    ("qsd_server_add_tensor", I, [P, I, P, P, P, I64, P, I64, ctypes.POINTER(I)]),
    ("qsd_server_submit", I, [P, I, P, ctypes.c_double, ctypes.POINTER(I64)]),
    ("qsd_server_poll", I, [P, ctypes.POINTER(ServerResult), I, I, ctypes.POINTER(I)]),
    ("qsd_server_copy_result", I, [P, I64, P, I64, P, P]),
    ("qsd_server_release", I, [P, I64]),
    ("qsd_server_get_stats", I, [P, ctypes.POINTER(ServerStats)]),
    ("qsd_server_clock", ctypes.c_double, []),
    ("qsd_server_destroy", None, [P]),
    ("qsd_profile_enable", I, [I]),
    ("qsd_profile_read", I, [ctypes.POINTER(ProfileRecord), I, ctypes.POINTER(I)]),
    ("qsd_profile_reset", I, []),
    ("qsd_status_string", ctypes.c_char_p, [I]),
    ("qsd_version", ctypes.c_char_p, []),
]

_lib = None


def load(path: str) -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libqsd is not built ({path} missing); run build()")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
