"""Seeded synthetic inputs for the 2-D DWT workloads.

This module holds input recipes only -- no wavelet arithmetic -- and imports
nothing from the rest of the package, so the tests can feed the same arrays to
the GPU library and to the CPU oracle.  All generators use numpy's PCG64.

The paper (arXiv:1704.08657, Evaluation) measures throughput against image
resolution on unnamed images; these recipes stand in for them:

  uniform(h, w, seed)        i.i.d. integers in [0, 255] cast to float32
  gradient(h, w, seed)       0.5*u + 63.75*(i/(h-1) + j/(w-1)), in [0, 255]
  noisy(h, w, seed)          u + N(0, 10^2), unclipped
  batch_shapes(n, seed)      sides 2*round(exp(U(ln 64, ln 2048))/2)
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(h: int, w: int, seed: int = 1) -> np.ndarray:
    """i.i.d. uniform integers in [0, 255] as float32, shape (h, w)."""
    return _rng(seed).integers(0, 256, size=(h, w), dtype=np.int16).astype(np.float32)


def gradient(h: int, w: int, seed: int = 2) -> np.ndarray:
    """Uniform noise at half amplitude plus a smooth diagonal ramp, in [0, 255]."""
    x = uniform(h, w, seed)
    x *= np.float32(0.5)
    ri = np.arange(h, dtype=np.float32) / np.float32(max(h - 1, 1))
    cj = np.arange(w, dtype=np.float32) / np.float32(max(w - 1, 1))
    x += np.float32(63.75) * ri[:, None]
    x += np.float32(63.75) * cj[None, :]
    return x


def noisy(h: int, w: int, seed: int = 3) -> np.ndarray:
    """Uniform [0, 255] integers plus Gaussian noise of sigma 10 (unclipped)."""
    rng = _rng(seed)
    x = rng.integers(0, 256, size=(h, w), dtype=np.int16).astype(np.float32)
    x += rng.standard_normal(size=(h, w), dtype=np.float32) * np.float32(10.0)
    return x


def to_int(x: np.ndarray, clip: bool = False) -> np.ndarray:
    """Round a float image to int32 (optionally clipped to [0, 255])."""
    if clip:
        x = np.clip(x, 0, 255)
    return np.rint(x).astype(np.int32)


def batch_shapes(n: int = 512, seed: int = 4, lo: int = 64, hi: int = 2048) -> List[Tuple[int, int]]:
    """(h, w) pairs with each side log-uniform in [lo, hi], rounded to even."""
    rng = _rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=(n, 2))
    sides = 2 * np.rint(np.exp(u) / 2).astype(np.int64)
    sides = np.clip(sides, lo, hi)
    return [(int(a), int(b)) for a, b in sides]


def batch_pack(shapes: List[Tuple[int, int]], seed: int = 5, align_elems: int = 4):
    """Pack uniform images into one flat float32 buffer.

    Returns (buffer, descs) with descs[i] = (offset_elems, h, w, pitch_elems);
    pitches and offsets are rounded up to ``align_elems`` elements.
    """
    rng = _rng(seed)
    descs = []
    off = 0
    for h, w in shapes:
        pitch = (w + align_elems - 1) // align_elems * align_elems
        descs.append((off, h, w, pitch))
        off += h * pitch
        off = (off + align_elems - 1) // align_elems * align_elems
    buf = np.zeros(off, dtype=np.float32)
    for (o, h, w, p) in descs:
        img = rng.integers(0, 256, size=(h, w), dtype=np.int16).astype(np.float32)
        buf[o:o + h * p].reshape(h, p)[:, :w] = img
    return buf, descs
