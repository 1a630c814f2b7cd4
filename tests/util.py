"""Shared helpers for the GPU parity tests (tolerances, band errors)."""
from __future__ import annotations

import numpy as np

from oracle import band_slices


def band_errors(got: np.ndarray, ref: np.ndarray, levels: int):
    """Per band: (level, name, max abs error, max |ref| in the band)."""
    out = []
    for lev, name, rs, cs in band_slices(ref.shape[0], ref.shape[1], levels):
        g, r = got[rs, cs].astype(np.float64), ref[rs, cs].astype(np.float64)
        if r.size == 0:
            continue
        out.append((lev, name, float(np.abs(g - r).max()), float(np.abs(r).max())))
    return out


def assert_fp32_close(got: np.ndarray, ref: np.ndarray, levels: int, x_max: float, what: str = ""):
    """FP32 lifting vs the FP64 oracle.

    Criterion: a level-k band, divided by 2^k
    (the DC gain of k levels, so that every band lives on the input's [0, 255]
    scale), must be within 1e-3 * x_max / 255 of the oracle; equivalently the
    raw error is at most 1e-3 * 2^k * x_max / 255.
    """
    for lev, name, err, bmax in band_errors(got, ref, levels):
        tol = 1e-3 * (2.0 ** lev) * max(x_max, 1e-30) / 255.0
        assert err <= tol, f"{what} level {lev} {name}: max abs err {err:.3e} > {tol:.3e} (band max {bmax:.3e})"


def assert_lowp_close(got: np.ndarray, ref: np.ndarray, levels: int, rel: float, what: str = ""):
    """FP16 / BF16 storage: per band max |q - ref| / max |ref band| <= rel."""
    for lev, name, err, bmax in band_errors(got, ref, levels):
        assert err <= rel * max(bmax, 1e-30), f"{what} level {lev} {name}: rel err {err / max(bmax, 1e-30):.3e} > {rel}"


def assert_dd_close(got: np.ndarray, ref: np.ndarray, levels: int, x_max: float, what: str = ""):
    """FP32 DD 13/7 lifting vs the FP64 oracle.  The transform has no scaling
    step (low-pass DC gain 1), so every band stays on the input's scale: each
    band within 1e-3 * x_max / 255 of the oracle."""
    for lev, name, err, bmax in band_errors(got, ref, levels):
        tol = 1e-3 * max(x_max, 1e-30) / 255.0
        assert err <= tol, f"{what} level {lev} {name}: max abs err {err:.3e} > {tol:.3e} (band max {bmax:.3e})"
