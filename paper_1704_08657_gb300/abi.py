"""ctypes binding of the libdwt2 C ABI (include/dwt2.h), same names.

Argument marshalling only: every step of the transform runs in the CUDA
kernels of libdwt2.so.  Importing this module loads the in-tree library and
fails loudly if it has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# DWT2_LIBRARY=checked loads the range-checked build (libdwt2_checked.so)
LIB_PATH = os.path.join(_PKG, "libdwt2_checked.so" if os.environ.get("DWT2_LIBRARY") == "checked" else "libdwt2.so")

DWT2_CDF97, DWT2_CDF53_INT, DWT2_DD137 = 0, 1, 2
DWT2_F32, DWT2_F16, DWT2_BF16, DWT2_I32 = 0, 1, 2, 3
DWT2_NONSEP, DWT2_NONSEP_REDUCED, DWT2_SEP_LIFTING, DWT2_POLYCONV, DWT2_CONV, DWT2_NONSEP_CONV = 0, 1, 2, 3, 4, 5
DWT2_SYMMETRIC = 0
DWT2_OK = 0
DWT2_ERR_INVALID_ARG = -1
DWT2_ERR_UNSUPPORTED = -2
DWT2_ERR_LEVELS_TOO_DEEP = -3
DWT2_ERR_MISALIGNED = -4
DWT2_ERR_CUDA = -5
DWT2_ERR_TIMEOUT = -6
DWT2_ERR_DEVICE_CHECK = -7
DWT2_ERR_TOO_LARGE = -8
DWT2_FLAG_PERSISTENT = 0x1
DWT2_TESTONLY_DROP_SIGNAL = 0x100  # test-only failure injection

# the functions the header declares (checked by the CPU test suite)
EXPORTS = ("dwt2_plan", "dwt2_workspace_bytes", "dwt2_forward", "dwt2_inverse", "dwt2_adjoint", "dwt2_adjoint_l1", "dwt2_adjoint_l1_dev",
           "dwt2_autotune", "dwt2_status", "dwt2_profile", "dwt2_profile_read", "dwt2_forward_noalloc",
           "dwt2_noalloc_status", "dwt2_band_rows", "dwt2_band_rects", "dwt2_band_stitch", "dwt2_checked", "dwt2_destroy",
           "dwt2_strerror")


class dwt2_image_desc(ctypes.Structure):
    _fields_ = [("offset_elems", ctypes.c_int64), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("pitch_elems", ctypes.c_int64)]


class Dwt2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {dwt2_strerror(code)} ({code})")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdwt2.so (or, with DWT2_LIBRARY=checked, libdwt2_checked.so;
    built by paper_1704_08657_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    lib.dwt2_checked.argtypes = []
    lib.dwt2_checked.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.dwt2_plan.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(dwt2_image_desc),
                              ctypes.c_uint]
    lib.dwt2_plan.restype = ctypes.c_int
    lib.dwt2_workspace_bytes.argtypes = [vp]
    lib.dwt2_workspace_bytes.restype = ctypes.c_size_t
    for name in ("dwt2_forward", "dwt2_inverse", "dwt2_adjoint"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, vp, vp, vp]
        f.restype = ctypes.c_int
    lib.dwt2_adjoint_l1.argtypes = [vp, vp, vp, ctypes.c_float, vp, vp]
    lib.dwt2_adjoint_l1.restype = ctypes.c_int
    lib.dwt2_adjoint_l1_dev.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp, vp]
    lib.dwt2_adjoint_l1_dev.restype = ctypes.c_int
    lib.dwt2_autotune.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
    lib.dwt2_autotune.restype = ctypes.c_int
    lib.dwt2_status.argtypes = [vp, vp]
    lib.dwt2_status.restype = ctypes.c_int
    lib.dwt2_profile.argtypes = [vp, ctypes.c_int]
    lib.dwt2_profile.restype = ctypes.c_int
    lib.dwt2_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.dwt2_profile_read.restype = ctypes.c_int
    lib.dwt2_forward_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int64, vp, vp, vp]
    lib.dwt2_forward_noalloc.restype = ctypes.c_int
    lib.dwt2_noalloc_status.argtypes = [vp]
    lib.dwt2_noalloc_status.restype = ctypes.c_int
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.dwt2_band_rows.argtypes = [ctypes.c_int] * 5 + [i32p]
    lib.dwt2_band_rows.restype = ctypes.c_int
    lib.dwt2_band_rects.argtypes = [ctypes.c_int] * 6 + [i32p, ctypes.c_int]
    lib.dwt2_band_rects.restype = ctypes.c_int
    lib.dwt2_band_stitch.argtypes = [ctypes.c_int] * 7 + [vp, ctypes.c_int64, vp, ctypes.c_int64, vp]
    lib.dwt2_band_stitch.restype = ctypes.c_int
    lib.dwt2_destroy.argtypes = [vp]
    lib.dwt2_destroy.restype = None
    lib.dwt2_strerror.argtypes = [ctypes.c_int]
    lib.dwt2_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


# --- same-name wrappers ------------------------------------------------------

def dwt2_strerror(code: int) -> str:
    return load().dwt2_strerror(int(code)).decode()


def dwt2_plan(wavelet: int, levels: int, boundary: int, in_dtype: int, coef_dtype: int, scheme: int,
              images, flags: int = 0) -> int:
    """Returns the plan handle; images is a list of (offset_elems, h, w, pitch_elems)."""
    arr = (dwt2_image_desc * len(images))(*[dwt2_image_desc(int(o), int(h), int(w), int(p))
                                            for (o, h, w, p) in images])
    out = ctypes.c_void_p()
    rc = load().dwt2_plan(ctypes.byref(out), int(wavelet), int(levels), int(boundary), int(in_dtype),
                          int(coef_dtype), int(scheme), len(images), arr, int(flags))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_plan")
    return out.value


def dwt2_workspace_bytes(plan: int) -> int:
    return int(load().dwt2_workspace_bytes(ctypes.c_void_p(plan)))


def _call(name, plan, a, b, ws, stream):
    rc = getattr(load(), name)(ctypes.c_void_p(plan), ctypes.c_void_p(a), ctypes.c_void_p(b),
                               ctypes.c_void_p(ws), ctypes.c_void_p(stream))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, name)


def dwt2_forward(plan: int, in_ptr: int, coef_ptr: int, ws_ptr: int = 0, stream: int = 0) -> None:
    _call("dwt2_forward", plan, in_ptr, coef_ptr, ws_ptr, stream)


def dwt2_inverse(plan: int, coef_ptr: int, out_ptr: int, ws_ptr: int = 0, stream: int = 0) -> None:
    _call("dwt2_inverse", plan, coef_ptr, out_ptr, ws_ptr, stream)


def dwt2_adjoint(plan: int, gcoef_ptr: int, gin_ptr: int, ws_ptr: int = 0, stream: int = 0) -> None:
    _call("dwt2_adjoint", plan, gcoef_ptr, gin_ptr, ws_ptr, stream)


def dwt2_adjoint_l1(plan: int, coef_ptr: int, gin_ptr: int, scale: float, ws_ptr: int = 0, stream: int = 0) -> None:
    rc = load().dwt2_adjoint_l1(ctypes.c_void_p(plan), ctypes.c_void_p(coef_ptr), ctypes.c_void_p(gin_ptr),
                                ctypes.c_float(scale), ctypes.c_void_p(ws_ptr), ctypes.c_void_p(stream))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_adjoint_l1")


def dwt2_adjoint_l1_dev(plan: int, coef_ptr: int, gin_ptr: int, scale_dev_ptr: int, scale: float, ws_ptr: int = 0,
                        stream: int = 0) -> None:
    rc = load().dwt2_adjoint_l1_dev(ctypes.c_void_p(plan), ctypes.c_void_p(coef_ptr), ctypes.c_void_p(gin_ptr),
                                    ctypes.c_void_p(scale_dev_ptr), ctypes.c_float(scale), ctypes.c_void_p(ws_ptr),
                                    ctypes.c_void_p(stream))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_adjoint_l1_dev")


def dwt2_autotune(plan: int, in_ptr: int, coef_ptr: int, ws_ptr: int = 0, stream: int = 0,
                  choice: int = -1) -> int:
    """Time the candidate configurations (choice < 0) or apply one; returns the choice."""
    c = ctypes.c_int(int(choice))
    rc = load().dwt2_autotune(ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(coef_ptr),
                              ctypes.c_void_p(ws_ptr), ctypes.c_void_p(stream), ctypes.byref(c))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_autotune")
    return int(c.value)


def dwt2_status(plan: int, stream: int = 0) -> int:
    return int(load().dwt2_status(ctypes.c_void_p(plan), ctypes.c_void_p(stream)))


def dwt2_profile(plan: int, enable: bool = True) -> None:
    rc = load().dwt2_profile(ctypes.c_void_p(plan), int(bool(enable)))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_profile")


def dwt2_profile_read(plan: int, n: int):
    """Mean milliseconds of each of the first n levels over the profiled calls."""
    arr = (ctypes.c_float * max(n, 1))()
    rc = load().dwt2_profile_read(ctypes.c_void_p(plan), arr, int(n))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_profile_read")
    return [float(arr[i]) for i in range(n)]


def dwt2_forward_noalloc(wavelet: int, levels: int, scheme: int, coef_dtype: int, h: int, w: int,
                         pitch_elems: int, in_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    """Forward pyramid of one image without any device allocation (the
    intermediate bands use the library's static scratch); returns the code."""
    return int(load().dwt2_forward_noalloc(int(wavelet), int(levels), int(scheme), int(coef_dtype), int(h),
                                           int(w), int(pitch_elems), ctypes.c_void_p(in_ptr),
                                           ctypes.c_void_p(coef_ptr), ctypes.c_void_p(stream)))


def dwt2_noalloc_status(stream: int = 0) -> int:
    """Synchronise the stream, return and clear dwt2_forward_noalloc's status word."""
    return int(load().dwt2_noalloc_status(ctypes.c_void_p(stream)))


def dwt2_band_rows(wavelet: int, levels: int, h: int, n_bands: int, band: int):
    """(own0, own1, in0, in1): the input rows band `band` of `n_bands` owns and
    the rows it transforms (host only)."""
    r = (ctypes.c_int32 * 4)()
    rc = load().dwt2_band_rows(int(wavelet), int(levels), int(h), int(n_bands), int(band), r)
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_band_rows")
    return tuple(int(v) for v in r)


def dwt2_band_rects(wavelet: int, levels: int, h: int, w: int, n_bands: int, band: int):
    """The band's copy rectangles (src_row, dst_row, rows, col0, cols) (host only)."""
    n = load().dwt2_band_rects(int(wavelet), int(levels), int(h), int(w), int(n_bands), int(band), None, 0)
    if n < 0:
        raise Dwt2Error(n, "dwt2_band_rects")
    buf = (ctypes.c_int32 * (5 * max(n, 1)))()
    n = load().dwt2_band_rects(int(wavelet), int(levels), int(h), int(w), int(n_bands), int(band), buf, n)
    if n < 0:
        raise Dwt2Error(n, "dwt2_band_rects")
    return [tuple(int(buf[5 * i + k]) for k in range(5)) for i in range(n)]


def dwt2_band_stitch(wavelet: int, levels: int, coef_dtype: int, h: int, w: int, n_bands: int, band: int,
                     band_coef_ptr: int, band_pitch: int, coef_ptr: int, pitch: int, stream: int = 0) -> None:
    rc = load().dwt2_band_stitch(int(wavelet), int(levels), int(coef_dtype), int(h), int(w), int(n_bands),
                                 int(band), ctypes.c_void_p(band_coef_ptr), int(band_pitch),
                                 ctypes.c_void_p(coef_ptr), int(pitch), ctypes.c_void_p(stream))
    if rc != DWT2_OK:
        raise Dwt2Error(rc, "dwt2_band_stitch")


def dwt2_destroy(plan: int) -> None:
    load().dwt2_destroy(ctypes.c_void_p(plan))


def raw_call(name: str, plan: int, a: int, b: int, ws: int = 0, stream: int = 0) -> int:
    """Call a transform entry point and return its code without raising."""
    return int(getattr(load(), name)(ctypes.c_void_p(plan), ctypes.c_void_p(a), ctypes.c_void_p(b),
                                     ctypes.c_void_p(ws), ctypes.c_void_p(stream)))
