"""ctypes binding of the C ABI in include/sgks.h (argument marshalling only).

Every function of the header is exposed under the same name.  The library is loaded from
the package directory (built in-tree by ``_build.build``); importing this module fails loudly
if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgks.so")

SGKS_OK, SGKS_BREAKDOWN, SGKS_STOPPED = 0, 1, 2
SGKS_ERR_INVALID, SGKS_ERR_CUDA, SGKS_ERR_NONFINITE = -1, -2, -3
SGKS_ERR_STATE, SGKS_ERR_NOMEM, SGKS_ERR_SKETCH = -4, -5, -6
SGKS_F32, SGKS_F64 = 0, 1
SGKS_OP_DENSE, SGKS_OP_CSR, SGKS_OP_CONV2D = 1, 2, 3
SGKS_REG_FD1, SGKS_REG_GRAD2D, SGKS_REG_LAPLACE2D, SGKS_REG_SPACETIME = 1, 2, 3, 4
SGKS_SKETCH_SPARSE_SIGN, SGKS_SKETCH_GAUSSIAN, SGKS_SKETCH_SRTT = 0, 1, 2
SGKS_PREC_FP64, SGKS_PREC_FP32, SGKS_PREC_FP32X, SGKS_PREC_FP32_PLAIN, SGKS_PREC_FF = 0, 1, 2, 3, 4
(SGKS_BUF_X, SGKS_BUF_Y, SGKS_BUF_W, SGKS_BUF_QA, SGKS_BUF_RA, SGKS_BUF_QL, SGKS_BUF_RL,
 SGKS_BUF_DA, SGKS_BUF_SB, SGKS_BUF_T, SGKS_BUF_AW) = range(1, 12)
(SGKS_APPLY_A, SGKS_APPLY_AT, SGKS_APPLY_L, SGKS_APPLY_LT, SGKS_APPLY_LTL, SGKS_APPLY_SA,
 SGKS_APPLY_SL) = range(1, 8)

ERROR_NAMES = {
    SGKS_OK: "SGKS_OK", SGKS_BREAKDOWN: "SGKS_BREAKDOWN", SGKS_STOPPED: "SGKS_STOPPED",
    SGKS_ERR_INVALID: "SGKS_ERR_INVALID", SGKS_ERR_CUDA: "SGKS_ERR_CUDA",
    SGKS_ERR_NONFINITE: "SGKS_ERR_NONFINITE", SGKS_ERR_STATE: "SGKS_ERR_STATE",
    SGKS_ERR_NOMEM: "SGKS_ERR_NOMEM", SGKS_ERR_SKETCH: "SGKS_ERR_SKETCH",
}


class sgks_op(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("val_dtype", C.c_int32), ("m", C.c_int64), ("n", C.c_int64),
        ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
        ("t_row_ptr", C.c_void_p), ("t_col", C.c_void_p), ("t_val", C.c_void_p),
        ("dense", C.c_void_p), ("ld", C.c_int64),
        ("nx", C.c_int32), ("ny", C.c_int32), ("kh", C.c_int32), ("kw", C.c_int32),
        ("psf", C.c_void_p),
    ]


class sgks_reg(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nt", C.c_int32)]


class sgks_options(C.Structure):
    _fields_ = [
        ("max_iters", C.c_int32), ("ell", C.c_int32), ("n_refine", C.c_int32),
        ("precision", C.c_int32), ("sketch_kind", C.c_int32), ("zeta", C.c_int32),
        ("cgs_passes", C.c_int32), ("flags", C.c_int32),
        ("gauss_SA", C.c_void_p), ("gauss_SL", C.c_void_p), ("x_true", C.c_void_p),
        ("srtt_signs_A", C.c_void_p), ("srtt_rows_A", C.c_void_p), ("srtt_signs_L", C.c_void_p),
        ("srtt_rows_L", C.c_void_p),
    ]


class sgks_report(C.Structure):
    _fields_ = [
        ("iters_done", C.c_int32), ("status", C.c_int32), ("subspace_dim", C.c_int32),
        ("reserved", C.c_int32), ("rc_last", C.c_double), ("rre_last", C.c_double),
        ("rre0", C.c_double), ("rc", C.POINTER(C.c_double)), ("rre", C.POINTER(C.c_double)),
    ]


_SIGNATURES = {
    "sgks_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(sgks_op), C.POINTER(sgks_reg), C.c_void_p,
                              C.c_double, C.c_int32, C.c_uint64, C.POINTER(sgks_options), C.c_void_p]),
    "sgks_reset": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgks_step": (C.c_int, [C.c_void_p]),
    "sgks_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.POINTER(sgks_report)]),
    "sgks_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "sgks_last_error": (C.c_char_p, [C.c_void_p]),
    "sgks_destroy": (None, [C.c_void_p]),
    "sgks_get_buffer": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "sgks_get_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "sgks_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "sgks_sparse_sign_rows": (C.c_int, [C.c_uint64, C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "sgks_csr_transpose": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgks_csr_transpose_noalloc": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgks_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(sgks_op), C.POINTER(sgks_reg),
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_double), C.POINTER(C.c_void_p), C.c_int32,
                                    C.c_uint64, C.POINTER(sgks_options), C.c_void_p]),
    "sgks_batch_reset": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "sgks_batch_step": (C.c_int, [C.c_void_p]),
    "sgks_batch_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_void_p),
                                   C.POINTER(sgks_report)]),
    "sgks_batch_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "sgks_batch_get_x": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "sgks_batch_layout": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "sgks_batch_profile_steps": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "sgks_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "sgks_batch_config": (C.c_char_p, [C.c_void_p, C.c_int32]),
    "sgks_batch_destroy": (None, [C.c_void_p]),
    "sgks_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "sgks_set_lambda": (C.c_int, [C.c_void_p, C.c_double]),
    "sgks_kernel_launches": (C.c_int64, []),
    "sgks_profile_steps": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double)]),
    "sgks_profile_graph": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double)]),
    "sgks_time_class": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
}
SGKS_PROFILE_CLASSES = 8
PROFILE_CLASS_NAMES = ["gradient_append", "sketch_column", "qr_append", "stacked_solve", "combine_refine",
                       "gradient_refine", "refine_solve", "combine"]
SGKS_FLAG_GLOBAL_SMALL = 1
SGKS_FLAG_RECORD = 2
SGKS_FLAG_GKS = 4
SGKS_FLAG_AUTOTUNE = 8
SGKS_FLAG_NO_TILES = 16
SGKS_FLAG_BW_HOST = 32
SGKS_BATCH_PROFILE_CLASSES = 10
BATCH_PROFILE_CLASS_NAMES = ["gradient_append", "apply_column", "qr_append", "stacked_solve", "combine_refine",
                             "gradient_refine", "refine_solve", "combine", "sketch_gather", "sketch_l"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libsgks.so and declare the ABI; raises if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2606_18073_gb300._build.build() "
                           "(the sGKS path has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGNATURES)


class SGKSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code, handle=None):
    if code < 0:
        lib = load()
        msg = lib.sgks_last_error(handle)
        raise SGKSError(code, msg.decode() if msg else "")
    return code


def check_batch(code, handle=None):
    if code < 0:
        lib = load()
        msg = lib.sgks_batch_last_error(handle)
        raise SGKSError(code, msg.decode() if msg else "")
    return code
