"""Loader of libstab.so, the CUDA library behind the C interface in include/stab.h.

The library is built in-tree (``paper_2502_10685_gb300/libstab.so``).  There is
no CPU fallback: if the library cannot be built or loaded, every entry point
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

STAB_OK = 0
ERRORS = {
    -1: "STAB_E_INVAL", -2: "STAB_E_RANGE", -3: "STAB_E_NOMEM", -4: "STAB_E_TIMEOUT",
    -5: "STAB_E_NONFINITE", -6: "STAB_E_CUDA", -7: "STAB_E_STATE", -8: "STAB_E_BUSY",
}


class StabError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        name = ERRORS.get(code, str(code))
        super().__init__("%s failed: %s%s" % (where, name, (" (" + detail + ")") if detail else ""))


class StabGate(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint8), ("q0", ctypes.c_uint8), ("q1", ctypes.c_uint8),
                ("flags", ctypes.c_uint8), ("param", ctypes.c_int32)]


class StabTerm(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("x", ctypes.c_uint64), ("z", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class StabOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("kernel", ctypes.c_int32), ("fuse", ctypes.c_int32),
                ("stream_given", ctypes.c_int32), ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", ctypes.c_void_p)]


class StabBatchItem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("kind", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("thetas", ctypes.c_void_p), ("n_params", ctypes.c_int64),
                ("obs", ctypes.c_void_p), ("n_terms", ctypes.c_int64)]


class StabServerOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("planners", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("iter_chunks", ctypes.c_int32), ("iter_smem_kb", ctypes.c_int32),
                ("iter_max_n", ctypes.c_int32), ("aging_s", ctypes.c_double),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("iter_slice_us", ctypes.c_double)]


class StabRequest(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("kind", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("thetas", ctypes.c_void_p), ("n_params", ctypes.c_int64),
                ("obs", ctypes.c_void_p), ("n_terms", ctypes.c_int64)]


class StabResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("expect", ctypes.c_double), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class StabSparseInfo(ctypes.Structure):
    _fields_ = [("order_final", ctypes.c_int64), ("order_max", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("dense_gates", ctypes.c_int64),
                ("regrows", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class StabPathChoice(ctypes.Structure):
    _fields_ = [("resident", ctypes.c_int32), ("resident_adjoint", ctypes.c_int32),
                ("gen_cut", ctypes.c_double), ("tile_limit", ctypes.c_int64),
                ("tuned", ctypes.c_int32), ("gen_parts", ctypes.c_int32)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libstab.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libstab.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        i32, i64, vp, dp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
        sig = {
            "stab_default_opts": (None, [ctypes.POINTER(StabOpts)]),
            "stab_create": (i32, [i32, ctypes.POINTER(StabOpts), ctypes.POINTER(vp)]),
            "stab_destroy": (i32, [vp]),
            "stab_load_circuit": (i32, [vp, vp, i64, dp, i64]),
            "stab_set_params": (i32, [vp, dp, i32]),
            "stab_run_generators": (i32, [vp]),
            "stab_apply_circuit": (i32, [vp, vp, i64, dp, i64]),
            "stab_get_generators": (i32, [vp, dp, i32]),
            "stab_generators_device": (vp, [vp]),
            "stab_expect": (i32, [vp, vp, i64, dp]),
            "stab_grad": (i32, [vp, vp, i64, dp, dp]),
            "stab_set_observable": (i32, [vp, vp, i64]),
            "stab_expect_async": (i32, [vp, dp]),
            "stab_grad_async": (i32, [vp, dp, dp]),
            "stab_transfer_bytes": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "stab_expect_static": (i32, [i32, vp, i64, dp, i64, vp, i64, dp, vp]),
            "stab_batch_create": (i32, [ctypes.POINTER(StabBatchItem), i64,
                                        ctypes.POINTER(StabOpts), ctypes.POINTER(vp)]),
            "stab_batch_run": (i32, [vp]),
            "stab_apply_batch": (i32, [vp]),
            "stab_serve_submit": (i32, [vp, ctypes.POINTER(StabRequest), ctypes.POINTER(i64)]),
            "stab_serve_poll": (i32, [vp, i64, ctypes.POINTER(ctypes.c_int32)]),
            "stab_batch_expectations": (i32, [vp, dp]),
            "stab_batch_generators": (i32, [vp, i64, dp, i32]),
            "stab_batch_info": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32)]),
            "stab_batch_destroy": (i32, [vp]),
            "stab_request_footprint": (i64, [ctypes.POINTER(StabRequest)]),
            "stab_server_create": (i32, [ctypes.POINTER(StabServerOpts), ctypes.POINTER(vp)]),
            "stab_server_submit": (i32, [vp, ctypes.POINTER(StabRequest), ctypes.POINTER(i64)]),
            "stab_server_wait": (i32, [vp, i64, ctypes.c_double, ctypes.POINTER(StabResult), dp]),
            "stab_server_poll": (i32, [vp, i64, ctypes.POINTER(ctypes.c_int32)]),
            "stab_server_stats": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                        ctypes.POINTER(i64), ctypes.POINTER(i64)]),
            "stab_server_destroy": (i32, [vp]),
            "stab_density_matrix": (i32, [vp, dp, i32]),
            "stab_synchronize": (i32, [vp]),
            "stab_plan_info": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_int32)]),
            "stab_split_info": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
            "stab_launch_count": (i64, [vp]),
            "stab_error_string": (ctypes.c_char_p, [i32]),
            "stab_last_cuda_error": (i32, []),
            "stab_version": (i32, []),
            "stab_selftest_bounded_wait": (i32, [i64]),
            "stab_selftest_plan": (i32, [i32, vp, i64, i64, i32]),
            "stab_selftest_align": (i32, [i32, vp, i64, i64, ctypes.POINTER(i64)]),
            "stab_grad_parts": (i32, [vp, ctypes.POINTER(i32)]),
            "stab_sparse_create": (i32, [i32, i64, ctypes.POINTER(StabOpts), ctypes.POINTER(vp)]),
            "stab_sparse_destroy": (i32, [vp]),
            "stab_sparse_load_circuit": (i32, [vp, vp, i64, dp, i64]),
            "stab_sparse_set_dense_threshold": (i32, [vp, i64]),
            "stab_sparse_expect": (i32, [vp, vp, i64, dp, ctypes.POINTER(StabSparseInfo)]),
            "stab_sparse_generator": (i32, [vp, i32, i64, vp, ctypes.POINTER(i64),
                                            ctypes.POINTER(StabSparseInfo)]),
            "stab_sparse_order_history": (i32, [vp, vp, i64, ctypes.POINTER(i64)]),
            "stab_probe_fp64": (i32, [i32, i64, dp, dp]),
            "stab_probe_pass": (i32, [i32, i32, i64, dp]),
            "stab_path_defaults": (i32, [i32, ctypes.POINTER(StabPathChoice)]),
            "stab_path_lookup": (i32, [ctypes.c_char_p, i32, ctypes.POINTER(StabPathChoice)]),
            "stab_path_store": (i32, [ctypes.c_char_p, i32, ctypes.POINTER(StabPathChoice)]),
            "stab_path_clear": (i32, []),
            "stab_path_save": (i32, [ctypes.c_char_p]),
            "stab_path_load": (i32, [ctypes.c_char_p]),
            "stab_path_tune": (i32, [i32, i32, ctypes.POINTER(StabPathChoice)]),
            "stab_path_current": (i32, [vp, ctypes.POINTER(StabPathChoice)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def check(code: int, where: str) -> None:
    if code != STAB_OK:
        detail = ""
        if code == -6 and _lib is not None:
            detail = "cuda error %d" % _lib.stab_last_cuda_error()
        raise StabError(code, where, detail)
