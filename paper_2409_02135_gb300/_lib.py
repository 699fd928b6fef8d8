"""ctypes declarations of the C ABI in include/qqa.h.

Loading fails loudly (ImportError / RuntimeError) when libqqa.so is missing or
cannot be loaded: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqqa.so")

QQA_OK = 0
QQA_EINVAL = -1
QQA_ENOMEM = -2
QQA_ECUDA = -3
QQA_ETIMEOUT = -4
QQA_ENONFINITE = -5
QQA_EBUSY = -6
ERROR_NAMES = {QQA_EINVAL: "EINVAL", QQA_ENOMEM: "ENOMEM", QQA_ECUDA: "ECUDA", QQA_ETIMEOUT: "ETIMEOUT",
               QQA_ENONFINITE: "ENONFINITE", QQA_EBUSY: "EBUSY"}

MIS, MAXCUT, MAXCLIQUE = 0, 1, 2
FP32, BF16 = 0, 1
KERNEL_AUTO, KERNEL_DIRECT, KERNEL_STAGED, KERNEL_STREAM, KERNEL_DENSE, KERNEL_PIPE, KERNEL_SCALAR = 0, 1, 2, 3, 4, 5, 6


class qqa_params(ctypes.Structure):
    _fields_ = [
        ("S", ctypes.c_int32), ("steps", ctypes.c_int32), ("round_every", ctypes.c_int32), ("a_ent", ctypes.c_int32),
        ("lr", ctypes.c_float), ("weight_decay", ctypes.c_float), ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
        ("gamma_min", ctypes.c_float), ("gamma_max", ctypes.c_float),
        ("alpha_comm", ctypes.c_float), ("comm_eps", ctypes.c_float), ("temperature", ctypes.c_float),
        ("lam", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class qqa_launch_config(ctypes.Structure):
    _fields_ = [("group_lanes", ctypes.c_int32), ("vec_per_lane", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("kernel_param", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class qqa_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("S", ctypes.c_int32), ("n", ctypes.c_int32),
                ("best_s", ctypes.c_int32), ("feasible", ctypes.c_int32), ("best_obj", ctypes.c_int64),
                ("bytes", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("evaluations", ctypes.c_int32), ("reserved", ctypes.c_int32)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class qqa_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


# every symbol declared in include/qqa.h: name -> (restype, argtypes)
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PU8 = ctypes.POINTER(ctypes.c_uint8)
_PU32 = ctypes.POINTER(ctypes.c_uint32)
_PF = ctypes.POINTER(ctypes.c_float)
_PD = ctypes.POINTER(ctypes.c_double)
_PPARAMS = ctypes.POINTER(qqa_params)
_PCFG = ctypes.POINTER(qqa_launch_config)
_PALLOC = ctypes.POINTER(qqa_allocator)
_PP = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "qqa_last_error": (ctypes.c_char_p, []),
    "qqa_version": (ctypes.c_char_p, []),
    "qqa_default_params": (None, [_PPARAMS]),
    "qqa_launch_count": (ctypes.c_uint64, []),
    "qqa_device_sm_count": (ctypes.c_int, []),
    "qqa_create_problem": (ctypes.c_int, [_I32, _I32, _PI32, _PI32, _PI32, _PALLOC, _P, _PP]),
    "qqa_problem_info": (ctypes.c_int, [_P, _PI32, _PI32, _PI64]),
    "qqa_destroy_problem": (None, [_P]),
    "qqa_run_create_empty": (ctypes.c_int, [_I32, _I32, _I32, _PCFG, _PALLOC, _P, _PP]),
    "qqa_run_add": (ctypes.c_int, [_P, _P, _PPARAMS, _P, _PI32]),
    "qqa_run_remove": (ctypes.c_int, [_P, _I32, _P]),
    "qqa_run_reset": (ctypes.c_int, [_P, _I32, ctypes.c_uint64, _P]),
    "qqa_run_create": (ctypes.c_int, [_PP, _PPARAMS, _I32, _PCFG, _PALLOC, _P, _PP]),
    "qqa_run_destroy": (None, [_P]),
    "qqa_run_config": (ctypes.c_int, [_P, _PCFG]),
    "qqa_autotune": (ctypes.c_int, [_PP, _PPARAMS, _I32, _I32, _PALLOC, _P, _PCFG, _PF]),
    "qqa_run_steps": (ctypes.c_int, [_P, _I32, _P]),
    "qqa_run_eval": (ctypes.c_int, [_P, _P]),
    "qqa_run_sync": (ctypes.c_int, [_P, _P]),
    "qqa_run_result": (ctypes.c_int, [_P, _I32, _PI64, _PI64, _PU8, _PD, _PI32, _PU32, _PI32]),
    "qqa_run_history": (ctypes.c_int, [_P, _I32, _I32, _PI64, _PI32, _PI32]),
    "qqa_run_slot_step": (ctypes.c_int, [_P, _I32, _PI32]),
    "qqa_anneal": (ctypes.c_int, [_PP, _PPARAMS, _I32, _PCFG, _PALLOC, _P, _PP]),
    "qqa_round_eval": (ctypes.c_int, [_P, _P, _PI64, _PI64, _PU8, _PD, _PI32, _PU32]),
    "qqa_run_get_state": (ctypes.c_int, [_P, _I32, _P, _PF, _PF, _PF, _PI32]),
    "qqa_run_set_state": (ctypes.c_int, [_P, _I32, _P, _PF, _PF, _PF, _I32]),
    "qqa_run_step_debug": (ctypes.c_int, [_P, _I32, _P, _PF]),
    "qqa_run_debug_set_status": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, _P]),
    "qqa_round_eval_noalloc": (ctypes.c_int, [_I32, _I32, ctypes.c_int64, _P, _P, _P, _I32, ctypes.c_int64, _P,
                                              ctypes.c_float, _P, _P, _P, _P, _P, _P]),
    "qqa_noalloc_last_error": (ctypes.c_char_p, []),
    "qqa_color_create": (ctypes.c_int, [_I32, _PI32, _PI32, _I32, _PPARAMS, _P, _PP]),
    "qqa_color_destroy": (None, [_P]),
    "qqa_color_steps": (ctypes.c_int, [_P, _I32, _PI32]),
    "qqa_color_sync": (ctypes.c_int, [_P]),
    "qqa_color_step_debug": (ctypes.c_int, [_P, _PF]),
    "qqa_color_debug_set_status": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64]),
    "qqa_color_get_state": (ctypes.c_int, [_P, _PF, _PF, _PF, _PI32]),
    "qqa_color_set_state": (ctypes.c_int, [_P, _PF, _PF, _PF, _I32]),
    "qqa_color_round": (ctypes.c_int, [_P, _PI64, _PI32, _PU8]),
    "qqa_color_info": (ctypes.c_int, [_P, _PI32, _PI32, _PI32, _PI32]),
    "qqa_request_bytes": (ctypes.c_int64, [_I32, ctypes.c_int64, _I32, _I32, _I32]),
    "qqa_server_create": (ctypes.c_int, [ctypes.c_int64, _I32, _I32, _I32, _PCFG, _PALLOC, _PP]),
    "qqa_server_submit": (ctypes.c_int, [_P, _I32, _I32, _PI32, _PI32, _PI32, _PPARAMS, _PI64]),
    "qqa_server_pump": (ctypes.c_int, [_P, _PI32, _PI32, _PI32]),
    "qqa_server_cancel": (ctypes.c_int, [_P, ctypes.c_int64]),
    "qqa_server_poll": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(qqa_request_info)]),
    "qqa_server_result": (ctypes.c_int, [_P, ctypes.c_int64, _PI64, _PI64, _PU8, _PD, _PU32, _PI64]),
    "qqa_server_stats": (ctypes.c_int, [_P, _PI64, _PI32]),
    "qqa_server_destroy": (None, [_P]),
}

_lib = None


class QQAError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"qqa error {ERROR_NAMES.get(code, code)}: {message}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libqqa.so (built by __graft_entry__.build() or paper_2409_02135_gb300._build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libqqa.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != QQA_OK:
        msg = load().qqa_last_error()
        raise QQAError(rc, msg.decode(errors="replace") if msg else "")
    return rc
