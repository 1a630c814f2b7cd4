"""The oracle: a plain CPU reference of the 2-D DWT (FP64 and int64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library does
not import it and shares no code with it.

``dwt2ref.c`` computes the separable lifting scheme of Barina et al.
(arXiv:1704.08657, Background section: Eq. 2 and the separable lifting scheme
"S_U^V | S_U^H | T_P^V | T_P^H") for CDF 9/7 and DD 13/7 in FP64 and the
reversible integer CDF 5/3 in int64, multi-level, Mallat layout, whole-sample
symmetric boundary.
``polyphase.py`` holds the paper's 4x4 polyphase matrices over Laurent
polynomials (Background, Proposed Schemes, Optimization Approach, Table 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwt2ref.c")
_LIB = os.path.join(_HERE, "libdwt2ref.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "invalid argument", -3: "levels too deep", -8: "out of memory"}


def build(force: bool = False) -> str:
    """Compile dwt2ref.c into libdwt2ref.so with gcc (OpenMP when available).

    -O3 without -ffast-math: ISO C11 mode keeps every floating-point operation
    as written (no contraction into fused multiply-adds, no reassociation), so
    the optimisation level changes the speed of the oracle, not its values.
    The build is portable (no -march=native): the same source runs on the
    host of the GPU machine, an Arm machine."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int64)
            L = ctypes.c_long
            for name, p in (("dwt2ref_forward_f64", dp), ("dwt2ref_inverse_f64", dp),
                            ("dwt2ref_adjoint_f64", dp), ("dwt2ref_forward_i64", ip),
                            ("dwt2ref_inverse_i64", ip), ("dwt2ref_forward_dd137_f64", dp),
                            ("dwt2ref_inverse_dd137_f64", dp)):
                f = getattr(lib, name)
                f.argtypes = [p, p, L, L, ctypes.c_int]
                f.restype = ctypes.c_int
            lib.dwt2ref_threads.restype = ctypes.c_int
            lib.dwt2ref_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _call(name: str, x: np.ndarray, levels: int, dtype) -> np.ndarray:
    lib = _load()
    if x.ndim != 2:
        raise ValueError("expected a 2-D array")
    src = np.ascontiguousarray(x, dtype=dtype)
    out = np.empty_like(src)
    ctype = ctypes.c_double if dtype == np.float64 else ctypes.c_int64
    p = ctypes.POINTER(ctype)
    rc = getattr(lib, name)(src.ctypes.data_as(p), out.ctypes.data_as(p),
                            src.shape[0], src.shape[1], int(levels))
    if rc != 0:
        raise ValueError(f"{name}: {ERRORS.get(rc, rc)} (shape {src.shape}, levels {levels})")
    return out


def forward97(x: np.ndarray, levels: int = 1) -> np.ndarray:
    """CDF 9/7 forward pyramid in FP64, Mallat layout (same shape as x)."""
    return _call("dwt2ref_forward_f64", x, levels, np.float64)


def inverse97(c: np.ndarray, levels: int = 1) -> np.ndarray:
    """Inverse of :func:`forward97`."""
    return _call("dwt2ref_inverse_f64", c, levels, np.float64)


def adjoint97(g: np.ndarray, levels: int = 1) -> np.ndarray:
    """Transpose of :func:`forward97` applied to a coefficient-domain array."""
    return _call("dwt2ref_adjoint_f64", g, levels, np.float64)


def forward137(x: np.ndarray, levels: int = 1) -> np.ndarray:
    """DD 13/7 forward pyramid in FP64, Mallat layout (no scaling step)."""
    return _call("dwt2ref_forward_dd137_f64", x, levels, np.float64)


def inverse137(c: np.ndarray, levels: int = 1) -> np.ndarray:
    """Inverse of :func:`forward137`."""
    return _call("dwt2ref_inverse_dd137_f64", c, levels, np.float64)


def forward53i(x: np.ndarray, levels: int = 1) -> np.ndarray:
    """Reversible integer CDF 5/3 forward pyramid in int64, Mallat layout."""
    return _call("dwt2ref_forward_i64", x, levels, np.int64)


def inverse53i(c: np.ndarray, levels: int = 1) -> np.ndarray:
    """Inverse of :func:`forward53i` (exact)."""
    return _call("dwt2ref_inverse_i64", c, levels, np.int64)


def threads() -> int:
    """Threads the oracle's loops use (1 when built without OpenMP)."""
    return int(_load().dwt2ref_threads())


def set_threads(n: int) -> None:
    _load().dwt2ref_set_threads(int(n))


def band_slices(h: int, w: int, levels: int):
    """Mallat band rectangles: list of (level, name, row slice, col slice).

    Level 1 is the finest.  Names: 'HL' (even row, odd column), 'LH' (odd row,
    even column), 'HH', and 'LL' for the coarsest low-low band.
    """
    out = []
    for lev in range(1, levels + 1):
        hl, wl = (h + 1) // 2, (w + 1) // 2
        out.append((lev, "HL", slice(0, hl), slice(wl, w)))
        out.append((lev, "LH", slice(hl, h), slice(0, wl)))
        out.append((lev, "HH", slice(hl, h), slice(wl, w)))
        h, w = hl, wl
    out.append((levels, "LL", slice(0, h), slice(0, w)))
    return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
