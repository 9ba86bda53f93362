"""ctypes declarations of the C ABI in include/idsketch.h.

Argument marshalling only: every step of the method runs in libidsketch.so.
Loading fails loudly when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libidsketch.so")

ID_OK = 0
ID_ERR_INVALID_ARG = 1
ID_ERR_STATE = 2
ID_ERR_OOM = 3
ID_ERR_CUDA = 4
ID_ERR_RANK_DEFICIENT = 5
ID_ERR_TIMEOUT = 6
ID_ERR_UNSUPPORTED = 7
ID_F32 = 0
ID_F64 = 1
ID_SKETCH_EXACT = 0
ID_SKETCH_BF16 = 1
ID_SKETCH_FP8E4M3 = 2
ID_RANK_TOL_FACTOR = 64.0
ID_NOALLOC_MAX_KN = 131072


class IdConfig(C.Structure):
    _fields_ = [
        ("m", C.c_int64),
        ("n_max", C.c_int64),
        ("k", C.c_int32),
        ("l", C.c_int32),
        ("seed", C.c_uint64),
        ("dtype", C.c_int32),
        ("prec", C.c_int32),
        ("grid", C.c_int32 * 3),
        ("ncomp", C.c_int32),
        ("coarse_stride", C.c_int32 * 3),
        ("want_Y", C.c_int32),
        ("want_coarse", C.c_int32),
        ("window_cols", C.c_int32),
        ("reserved", C.c_int32 * 4),
    ]


ID_BATCH_MAX_PROBLEMS = 1024
ID_BATCH_MAX_COLS = 512


class IdBatchProblem(C.Structure):
    _fields_ = [
        ("d_A", C.c_void_p),
        ("lda", C.c_int64),
        ("m", C.c_int64),
        ("n", C.c_int32),
        ("k", C.c_int32),
        ("l", C.c_int32),
        ("dtype", C.c_int32),
        ("prec", C.c_int32),
        ("reserved", C.c_int32),
        ("seed", C.c_uint64),
    ]


# name -> (restype, argtypes); the exported symbol set of include/idsketch.h
SIGNATURES = {
    "id_sketch_create": (C.c_int, [C.POINTER(IdConfig), C.c_void_p, C.POINTER(C.c_void_p)]),
    "id_sketch_stream_columns": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "id_sketch_flush": (C.c_int, [C.c_void_p]),
    "id_sketch_reset": (C.c_int, [C.c_void_p]),
    "id_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "id_coarse_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "id_factor_restricted": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                       C.c_void_p, C.POINTER(C.c_int32)]),
    "id_reconstruct_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                       C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
    "id_reconstruct_error_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                               C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                               C.POINTER(C.c_double), C.POINTER(C.c_double),
                                               C.c_void_p]),
    "id_sketch_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
    "id_sketch_destroy": (None, [C.c_void_p]),
    "id_set_mesh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "id_single_pass_lift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "id_single_pass_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                       C.c_void_p, C.c_void_p, C.c_int32,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "id_batch_create": (C.c_int, [C.POINTER(IdBatchProblem), C.c_int32, C.c_void_p,
                                  C.POINTER(C.c_void_p)]),
    "id_batch_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "id_batch_tune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "id_batch_wait": (C.c_int, [C.c_void_p, C.c_void_p]),
    "id_batch_destroy": (None, [C.c_void_p]),
    "id_mlp_features": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                  C.c_void_p, C.c_int64, C.c_float, C.c_void_p, C.c_void_p]),
    "id_mlp_forward": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "id_mlp_backward": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "id_mlp_sgd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p]),
    "id_mlp_check": (C.c_int, [C.c_void_p]),
    "id_mlp_propose": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]),
    "id_mlp_propose_stratified": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                            C.c_void_p, C.c_void_p, C.c_void_p]),
    "id_timing_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "id_timing_read": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                 C.POINTER(C.c_int64)]),
    "id_gaussian_fill": (C.c_int, [C.c_int32, C.c_uint64, C.c_int64, C.c_int64, C.c_int32,
                                   C.c_void_p, C.c_void_p]),
    "id_gaussian_table": (C.c_int, [C.POINTER(C.c_uint16)]),
    "id_check_wait": (C.c_int, [C.c_int32, C.c_int32]),
    "id_kernel_launches": (C.c_int64, []),
    "id_last_cuda_error": (C.c_char_p, []),
    "id_status_str": (C.c_char_p, [C.c_int]),
    "id_version": (C.c_int32, []),
}

_LIB = None


def load():
    """Load libidsketch.so (raises if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
            "g.build()'` (nvcc, sm_103a). There is no CPU fallback.")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class IdError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        lib = load()
        msg = lib.id_status_str(status).decode()
        if status == ID_ERR_CUDA:
            msg += f" [{lib.id_last_cuda_error().decode()}]"
        super().__init__(f"{where}: {msg} (status {status})")


def check(status, where, allow=()):
    if status != ID_OK and status not in allow:
        raise IdError(status, where)
    return status
