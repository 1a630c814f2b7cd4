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


U32 = 2.0 ** -24  # unit roundoff of FP32


def fp32_bounds(lev: int, name: str, bmax: float, x_max: float):
    """(absolute bound, relative bound) of one band for FP32 lifting.

    The values a level-k band is computed from have the magnitude of the
    level's input, 2^(k-1) x_max (the low-low DC gain is 2 per level), and
    every FP32 operation rounds at that scale, so the error of a level-k band
    is a multiple of u * 2^k * x_max (u = 2^-24).  Measured over every parity
    test and the 16384^2 bench workload (all six schemes, one to six levels):
    at most 17 such units in a detail band and 33 in the coarsest low-low band
    (which carries the rounding of every level before it).  Bounds: 24 units
    for detail bands, 48 for the low-low band -- and, per band, at most 1e-4
    of the band's own largest magnitude plus 4 units (measured at most half
    of that), which holds a band of small values to its own scale.
    """
    unit = U32 * (2.0 ** lev) * max(x_max, 1e-30)
    return (48.0 if name == "LL" else 24.0) * unit, 1e-4 * bmax + 4.0 * unit


def assert_fp32_close(got: np.ndarray, ref: np.ndarray, levels: int, x_max: float, what: str = ""):
    """FP32 lifting vs the FP64 oracle, band by band: the absolute bound in
    units of u * 2^k * x_max and the relative bound of fp32_bounds."""
    for lev, name, err, bmax in band_errors(got, ref, levels):
        tol_a, tol_r = fp32_bounds(lev, name, bmax, x_max)
        assert err <= tol_a, f"{what} level {lev} {name}: max abs err {err:.3e} > {tol_a:.3e} (band max {bmax:.3e})"
        assert err <= tol_r, (f"{what} level {lev} {name}: max abs err {err:.3e} > {tol_r:.3e} = 1e-4 of the band max "
                              f"{bmax:.3e} + 4 units")


def report_band_errors(got: np.ndarray, ref: np.ndarray, levels: int, x_max: float, what: str = ""):
    """Print, per band, the max abs error, the max relative error (against the
    band's largest magnitude) and the error in units of u * 2^k * x_max."""
    print(f"\n{what}: per-band errors against the FP64 oracle")
    print(f"{'level':>5} {'band':>4} {'max abs':>11} {'max rel':>11} {'units':>7}")
    for lev, name, err, bmax in band_errors(got, ref, levels):
        unit = U32 * (2.0 ** lev) * max(x_max, 1e-30)
        print(f"{lev:>5} {name:>4} {err:11.3e} {err / max(bmax, 1e-30):11.3e} {err / unit:7.2f}")


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
