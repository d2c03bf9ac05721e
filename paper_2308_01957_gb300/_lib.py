"""ctypes binding of libastrophot_gb300 (include/astrophot_gb300.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libastrophot_gb300.so")

AP_OK, AP_ERR_ARG, AP_ERR_CUDA, AP_ERR_NOT_SPD, AP_ERR_NONFINITE, AP_ERR_TIMEOUT, AP_ERR_STATE, AP_ERR_NOMEM = range(8)
AP_SERSIC, AP_EXPONENTIAL, AP_GAUSSIAN, AP_MOFFAT, AP_SKY_FLAT, AP_SKY_PLANE, AP_PSF_STAR = range(7)
AP_PREC_MIXED, AP_PREC_F64 = 0, 1
AP_SHIFT_LANCZOS3, AP_SHIFT_BILINEAR = 1, 2

EXPORTED = (
    "ap_create", "ap_destroy", "ap_strerror", "ap_get_error", "ap_set_problem", "ap_get_layout", "ap_render",
    "ap_eval", "ap_normal_eq", "ap_get_jtwj_nnz", "ap_get_jtwj_structure", "ap_copy_jtwj", "ap_lm_solve",
    "ap_lm_iterate", "ap_lm_continue", "ap_get_status", "ap_get_state", "ap_get_launch_count", "ap_set_timing", "ap_get_timing",
    "ap_lm_solve_noalloc", "ap_get_jcol_mode", "ap_eval_adaptive", "ap_get_adaptive_layout", "ap_get_conv_variant",
    "ap_measure_pipe", "ap_eval_shifted",
)


class ApOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("quad_order", C.c_int), ("device", C.c_int),
                ("tile_w", C.c_int), ("tile_h", C.c_int), ("jcol_mode", C.c_int),
                ("conv_variant", C.c_int), ("gram_tc_min", C.c_int)]


class ApImageDesc(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("A", C.c_double * 4), ("origin", C.c_double * 2),
                ("data_dev", C.c_void_p), ("variance_dev", C.c_void_p), ("mask_dev", C.c_void_p),
                ("psf_dev", C.c_void_p), ("K", C.c_int), ("group", C.c_int), ("psf_live", C.c_int),
                ("psf_pidx", C.c_int * 2), ("psf_pfix", C.c_double * 2)]


class ApSourceDesc(C.Structure):
    _fields_ = [("type", C.c_int), ("image", C.c_int), ("win", C.c_int * 4), ("psf_convolve", C.c_int),
                ("pidx", C.c_int * 8), ("pfix", C.c_double * 8)]


class ApError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {_strerror(code)}" + (f" ({detail})" if detail else ""))


_lib = None


def load() -> C.CDLL:
    """Load the library (once).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2308_01957_gb300.build.build() (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "ap_create": (i, [C.POINTER(vp), C.POINTER(ApOptions)]),
        "ap_destroy": (None, [vp]),
        "ap_strerror": (C.c_char_p, [i]),
        "ap_get_error": (C.c_char_p, [vp]),
        "ap_set_problem": (i, [vp, C.POINTER(ApImageDesc), i, C.POINTER(ApSourceDesc), i, i, vp]),
        "ap_get_layout": (i, [vp, C.POINTER(i), C.POINTER(i)]),
        "ap_render": (i, [vp, vp, C.POINTER(vp), vp]),
        "ap_eval": (i, [vp, vp, vp, vp, vp]),
        "ap_normal_eq": (i, [vp, vp, vp, vp]),
        "ap_get_jtwj_nnz": (i, [vp, C.POINTER(i64)]),
        "ap_get_jtwj_structure": (i, [vp, vp, vp]),
        "ap_copy_jtwj": (i, [vp, vp, vp]),
        "ap_lm_solve": (i, [vp, vp, vp, vp]),
        "ap_lm_iterate": (i, [vp, vp, vp, vp, i, vp, vp]),
        "ap_lm_continue": (i, [vp, vp, vp, vp, i, vp, vp]),
        "ap_get_status": (i, [vp, C.POINTER(i), vp]),
        "ap_get_state": (i, [vp, vp, C.POINTER(i64), vp]),
        "ap_get_launch_count": (i, [vp, C.POINTER(i), C.POINTER(i)]),
        "ap_get_jcol_mode": (i, [vp, C.POINTER(i), C.POINTER(d), C.POINTER(d), C.POINTER(i), C.POINTER(i)]),
        "ap_set_timing": (i, [vp, i]),
        "ap_lm_solve_noalloc": (i, [i, vp, vp, vp, vp, vp, vp, vp, vp]),
        "ap_get_timing": (i, [vp, C.c_char_p, i, C.POINTER(d), C.POINTER(i), i, C.POINTER(i)]),
        "ap_eval_adaptive": (i, [vp, vp, d, vp, C.POINTER(vp), vp, vp, vp]),
        "ap_get_adaptive_layout": (i, [vp, C.POINTER(i64), vp]),
        "ap_get_conv_variant": (i, [vp, C.POINTER(i), C.POINTER(i), vp, vp]),
        "ap_measure_pipe": (i, [i, i, C.POINTER(d), C.POINTER(d), vp]),
        "ap_eval_shifted": (i, [vp, vp, i, vp, C.POINTER(vp), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _strerror(code: int) -> str:
    try:
        return load().ap_strerror(code).decode()
    except Exception:
        return f"status {code}"


def check(code: int, where: str, ctx=None) -> None:
    if code != AP_OK:
        detail = load().ap_get_error(ctx).decode() if ctx else ""
        raise ApError(code, where, detail)
