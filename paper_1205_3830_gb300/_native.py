"""ctypes declarations of librid.so (the C ABI in include/rid.h)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librid.so")

RID_OK, RID_EINVAL, RID_ENOMEM, RID_ECUDA, RID_ERANK, RID_ETIMEOUT, RID_EUNSUPPORTED = range(7)
RID_C128, RID_C64 = 0, 1
RID_FP64_NATIVE, RID_FP64_EMULATED, RID_MIXED_BF16, RID_MIXED_3XTF32 = range(4)

# every symbol include/rid.h declares, with (restype, argtypes)
_c_plan = ctypes.c_void_p
_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
SIGNATURES = {
    "rid_plan_create": (ctypes.c_int, [ctypes.POINTER(_c_plan), _i64, _i64, _i32, _i32, ctypes.c_int,
                                       ctypes.c_int, _u64, _p]),
    "rid_plan_create_probes": (ctypes.c_int, [ctypes.POINTER(_c_plan), _i64, _i64, _i32, _i32, ctypes.c_int,
                                              ctypes.c_int, _u64, _p, _i32, _u64]),
    "rid_plan_destroy": (ctypes.c_int, [_c_plan]),
    "rid_plan_reseed": (ctypes.c_int, [_c_plan, _u64, _u64]),
    "rid_plan_set_stream": (ctypes.c_int, [_c_plan, _p]),
    "rid_plan_footprint": (ctypes.c_int, [_i64, _i64, _i32, _i32, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "rid_plan_omega": (ctypes.c_int, [_c_plan, ctypes.POINTER(_p), ctypes.POINTER(_i64)]),
    "rid_plan_probe_products": (ctypes.c_int, [_c_plan, ctypes.POINTER(_p), ctypes.POINTER(_i64)]),
    "rid_plan_set_omega": (ctypes.c_int, [_c_plan, _p, _i64]),
    "rid_plan_use_srft": (ctypes.c_int, [_c_plan, _u64]),
    "rid_sketch": (ctypes.c_int, [_c_plan, _p, _i64, _p, _i64]),
    "rid_sketch_cols": (ctypes.c_int, [_c_plan, _p, _i64, _p, _i64, _i64, _i64]),
    "rid_select": (ctypes.c_int, [_c_plan, _p, _i64, _p]),
    "rid_solve": (ctypes.c_int, [_c_plan, _p, _i64, _p, _i64]),
    "rid_error": (ctypes.c_int, [_c_plan, _p, _i64, _p, _p, _i64, _i32, _u64,
                                 ctypes.POINTER(ctypes.c_double)]),
    "rid_plan_round_omega": (ctypes.c_int, [_c_plan, _i32]),
    "rid_plan_set_probes": (ctypes.c_int, [_c_plan, _i32, _u64]),
    "rid_error_sketched": (ctypes.c_int, [_c_plan, _p, _p, _i64, ctypes.POINTER(ctypes.c_double)]),
    "rid_sync_status": (ctypes.c_int, [_c_plan]),
    "rid_plan_stats": (ctypes.c_int, [_c_plan, ctypes.POINTER(_i64)]),
    "rid_plan_set_select_grid": (ctypes.c_int, [_c_plan, _i32]),
    "rid_plan_timing": (ctypes.c_int, [_c_plan, _i32, ctypes.POINTER(ctypes.c_double)]),
    "rid_plan_accuracy": (ctypes.c_int, [_c_plan, _p, _i64, ctypes.POINTER(ctypes.c_double)]),
    "rid_batch_workspace": (ctypes.c_int, [_i32, ctypes.POINTER(ctypes.c_size_t)]),
    "rid_batch_run": (ctypes.c_int, [ctypes.c_void_p, _i32, _i32, _u64, _i32, _p, _p, _p, ctypes.c_size_t, _p]),
    "rid_batch_prepare": (ctypes.c_int, [ctypes.c_void_p, _i32, _i32, _p, ctypes.c_size_t, _p]),
    "rid_batch_launch": (ctypes.c_int, [_i32, _i32, _u64, _i32, _p, _p, _p, _p]),
    "rid_batch_tc_create": (ctypes.c_int, [ctypes.POINTER(_p), ctypes.c_void_p, _i32, _i32, _u64, _p, _p, _p]),
    "rid_batch_tc_run": (ctypes.c_int, [_p, _p]),
    "rid_batch_tc_create_tuned": (ctypes.c_int, [ctypes.POINTER(_p), ctypes.c_void_p, _i32, _i32, _u64, _p, _p, _p,
                                                  _p, ctypes.c_size_t, _p]),
    "rid_batch_tc_times": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_double)]),
    "rid_batch_tc_info": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_double)]),
    "rid_batch_tc_destroy": (ctypes.c_int, [_p]),
    "rid_select_noalloc": (ctypes.c_int, [_p, _i64, _i32, _i64, _i32, _p, _p, _p]),
    "rid_selftest_timeouts": (ctypes.c_int, [_p, _p]),
    "rid_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}



class BatchItem(ctypes.Structure):
    """Mirror of rid_batch_item (include/rid.h)."""
    _fields_ = [("m", _i64), ("n", _i64), ("k", _i32), ("l", _i32), ("A", _p), ("lda", _i64), ("Y", _p),
                ("ldy", _i64), ("perm", _p), ("T", _p), ("ldt", _i64), ("seed", _u64)]


_lib = None


class RIDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


def load():
    """Load librid.so (built in-tree by paper_1205_3830_gb300.build).  There is
    no fallback: without the library every call fails loudly."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"native library {LIB_PATH} is missing: run paper_1205_3830_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status):
    return load().rid_status_string(int(status)).decode()


def check(status, where):
    if status != RID_OK:
        raise RIDError(status, where)
