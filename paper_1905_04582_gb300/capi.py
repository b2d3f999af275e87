"""ctypes binding of the C ABI in include/mds.h (argument marshalling only).

Every function here has the name of the C entry point it calls and returns
its status code; nothing is computed in Python.  The shared library is built
in-tree by ``paper_1905_04582_gb300.build`` (or ``__graft_entry__.build()``);
if it is missing, ``lib()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmds.so")

MDS_OK = 0
MDS_ERR_INVALID_ARG = 1
MDS_ERR_STATE = 2
MDS_ERR_CUDA = 3
MDS_ERR_OOM = 4
MDS_ERR_TIMEOUT = 5
MDS_ERR_NONFINITE = 6
MDS_ERR_UNSUPPORTED = 7
MDS_ERR_EXCHANGE = 8

MDS_PREC_FP32C = 0
MDS_PREC_FP64 = 1
MDS_F32 = 0
MDS_F64 = 1
MDS_HOST = 0
MDS_DEVICE = 1
MDS_Y_FULL = 0
MDS_Y_PACKED_UPPER = 1
MDS_MAX_D = 8
MDS_PASS_STRIPS = 0
MDS_PASS_CHUNKS = 1
MDS_PASS_CHUNK_COUNT = 2
MDS_PASS_SM_CHUNKS = 3

STATUS_NAMES = {
    0: "MDS_OK", 1: "MDS_ERR_INVALID_ARG", 2: "MDS_ERR_STATE", 3: "MDS_ERR_CUDA", 4: "MDS_ERR_OOM",
    5: "MDS_ERR_TIMEOUT", 6: "MDS_ERR_NONFINITE", 7: "MDS_ERR_UNSUPPORTED", 8: "MDS_ERR_EXCHANGE",
}

# int (*)(void *user, const double *send, double *recv, int64_t count, int32_t where)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_int32)


class mds_hmc_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("last_dh", ctypes.c_double), ("last_loglik", ctypes.c_double)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_pdbl = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pi32 = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); the public ABI of include/mds.h
SIGNATURES = {
    "mds_create": (_int, [_i64, _i32, _u32, ctypes.POINTER(_vp)]),
    "mds_destroy": (_int, [_vp]),
    "mds_set_stream": (_int, [_vp, _vp]),
    "mds_set_data": (_int, [_vp, _vp, _int, _int, _i64, _int]),
    "mds_set_locations": (_int, [_vp, _vp, _int, _int]),
    "mds_get_locations": (_int, [_vp, _vp, _int, _int]),
    "mds_set_sigma": (_int, [_vp, _dbl]),
    "mds_set_prior": (_int, [_vp, _dbl]),
    "mds_log_likelihood": (_int, [_vp, _pdbl, _pdbl]),
    "mds_gradient": (_int, [_vp, _pdbl, _vp, _int, _int, _pdbl]),
    "mds_set_momentum": (_int, [_vp, _vp, _int, _int]),
    "mds_get_momentum": (_int, [_vp, _vp, _int, _int]),
    "mds_leapfrog": (_int, [_vp, _int, _dbl, _vp, _int, _int, _pdbl]),
    "mds_hmc": (_int, [_vp, _int, _int, _dbl, _u64, _vp, _vp, _vp, _vp, ctypes.POINTER(mds_hmc_stats)]),
    "mds_hmc_enqueue": (_int, [_vp, _int, _int, _dbl, _u64]),
    "mds_get_sigma": (_int, [_vp, _pdbl]),
    "mds_sigma_mh": (_int, [_vp, _int, _dbl, _dbl, _dbl, _u64, _vp, _vp, _vp]),
    "mds_set_heldout": (_int, [_vp, _vp, _i64]),
    "mds_heldout_count": (_int, [_vp, _pi64]),
    "mds_lpd_accumulate": (_int, [_vp]),
    "mds_lpd": (_int, [_vp, _pdbl, _pi64]),
    "mds_lpd_reset": (_int, [_vp]),
    "mds_hmc_collect": (_int, [_vp, _i64, _vp, _vp, _pi64, ctypes.POINTER(mds_hmc_stats)]),
    "mds_problem_size": (_int, [_vp, _pi64, _pi64]),
    "mds_locality_order": (_int, [_i64, _i32, _vp, _vp]),
    "mds_tree_plan_check": (_int, [_i64, _i64, _vp, _vp, _i32, _vp]),
    "mds_reorder": (_int, [_vp]),
    "mds_get_order": (_int, [_vp, _vp]),
    "mds_set_tail_cutoff": (_int, [_vp, _dbl]),
    "mds_far_blocks": (_int, [_vp, _pi64, _pi64]),
    "mds_pair_body_ceiling": (_int, [_vp, _i32, _pdbl]),
    "mds_set_tree_prior": (_int, [_vp, _i64, _vp, _vp, _vp, _vp, _dbl, _dbl]),
    "mds_tree_prior": (_int, [_vp, _pdbl, _vp, _int, _int]),
    "mds_rwmh": (_int, [_vp, _int, _dbl, _u64, _vp, _vp, _vp, _vp, _vp]),
    "mds_get_state": (_int, [_vp, _vp, _pi64]),
    "mds_set_state": (_int, [_vp, _vp, _i64]),
    "mds_set_strip": (_int, [_vp, _i32]),
    "mds_get_strip": (_int, [_vp, _pi32]),
    "mds_shard_range": (_int, [_i64, _i32, _i32, _pi64, _pi64]),
    "mds_set_shard": (_int, [_vp, _i32, _i32, ALLGATHER_FN, _vp, _i32]),
    "mds_shard_sum": (_int, [_i32, _i64, _vp, _vp]),
    "mds_set_pass_shape": (_int, [_vp, _i32, _i32]),
    "mds_get_pass_shape": (_int, [_vp, _pi32, _pi32, _pi32]),
    "mds_set_pass_stamps": (_int, [_vp, _int]),
    "mds_get_pass_span": (_int, [_vp, _pi64, _pdbl]),
    "mds_time_pass": (_int, [_vp, _int, _pdbl]),
    "mds_set_profiling": (_int, [_vp, _int]),
    "mds_get_pass_time": (_int, [_vp, _pi64, _pdbl]),
    "mds_batch_create": (_int, [_i32, _vp, _i32, _vp, _u32, ctypes.POINTER(_vp)]),
    "mds_batch_destroy": (_int, [_vp]),
    "mds_batch_set_stream": (_int, [_vp, _vp]),
    "mds_batch_set_data": (_int, [_vp, _i32, _vp, _int, _int, _i64, _int]),
    "mds_batch_set_sigma": (_int, [_vp, _i32, _dbl]),
    "mds_batch_set_locations": (_int, [_vp, _i32, _i32, _vp, _int, _int]),
    "mds_batch_get_locations": (_int, [_vp, _i32, _i32, _vp, _int, _int]),
    "mds_batch_get_gradient": (_int, [_vp, _i32, _i32, _vp, _int, _int]),
    "mds_batch_evaluate": (_int, [_vp, _vp, _vp]),
    "mds_batch_hmc": (_int, [_vp, _int, _int, _vp, _u64, _vp, _vp]),
    "mds_batch_set_strip": (_int, [_vp, _i32]),
    "mds_batch_reorder": (_int, [_vp]),
    "mds_batch_get_strip": (_int, [_vp, _pi32]),
    "mds_batch_time_pass": (_int, [_vp, _int, _pdbl]),
    "mds_batch_last_error": (ctypes.c_char_p, [_vp]),
    "mds_loglik_grad_noalloc": (_int, [_i64, _i32, _vp, _i64, _vp, _dbl, _vp, _pdbl, _pdbl, _vp]),
    "mds_last_error": (ctypes.c_char_p, [_vp]),
}

_lock = threading.Lock()
_lib = None


def lib():
    """Load libmds.so (built in-tree); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_1905_04582_gb300.build` "
                    "(there is no fallback implementation)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class MDSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, ctx=None):
    if status != MDS_OK:
        msg = lib().mds_last_error(ctx).decode(errors="replace")
        raise MDSError(status, msg)
    return status
