"""PyTorch-facing helpers over the libdwt2 C ABI.

PyTorch provides device memory and streams only; every transform step runs in
the CUDA kernels of libdwt2.so (see ``abi``).  A ``Plan`` wraps one C plan and
owns a workspace tensor; ``DWT2Function`` exposes the forward transform to
autograd with the hand-written adjoint kernel as its backward.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import List, Optional, Sequence, Tuple

import torch

from . import abi

WAVELETS = {"cdf97": abi.DWT2_CDF97, "cdf53": abi.DWT2_CDF53_INT, "dd137": abi.DWT2_DD137}
SCHEMES = {"nonsep": abi.DWT2_NONSEP, "reduced": abi.DWT2_NONSEP_REDUCED, "sep": abi.DWT2_SEP_LIFTING,
           "polyconv": abi.DWT2_POLYCONV, "conv": abi.DWT2_CONV,
           "nsconv": abi.DWT2_NONSEP_CONV}
DTYPES = {torch.float32: abi.DWT2_F32, torch.float16: abi.DWT2_F16, torch.bfloat16: abi.DWT2_BF16,
          torch.int32: abi.DWT2_I32}


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def round_up(v: int, m: int) -> int:
    return (v + m - 1) // m * m


class Plan:
    """One transform plan (wavelet, levels, scheme, dtypes, image layout).

    ``images`` is a list of (offset_elems, h, w, pitch_elems); for a single
    image use ``Plan.single(h, w, ...)``.  Buffers passed to the transform
    calls are flat or 2-D CUDA tensors addressed by those offsets and pitches.
    """

    def __init__(self, images: Sequence[Tuple[int, int, int, int]], levels: int, wavelet: str = "cdf97",
                 scheme: str = "nonsep", coef_dtype: torch.dtype = torch.float32, flags: int = 0,
                 device: Optional[torch.device] = None):
        self.images = [tuple(int(v) for v in d) for d in images]
        self.levels = int(levels)
        self.wavelet = wavelet
        self.scheme = scheme
        self.in_dtype = torch.int32 if wavelet == "cdf53" else torch.float32
        self.coef_dtype = coef_dtype
        self.flags = int(flags)
        self.tuned: Optional[int] = None
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.handle = abi.dwt2_plan(WAVELETS[wavelet], self.levels, abi.DWT2_SYMMETRIC,
                                        DTYPES[self.in_dtype], DTYPES[coef_dtype], SCHEMES[scheme],
                                        self.images, flags)
        self.ws_bytes = abi.dwt2_workspace_bytes(self.handle)
        self._ws: Optional[torch.Tensor] = None
        self.n_elems = max(o + h * p for (o, h, w, p) in self.images)

    @classmethod
    def single(cls, h: int, w: int, levels: int, pitch: Optional[int] = None, **kw) -> "Plan":
        return cls([(0, h, w, pitch if pitch is not None else w)], levels, **kw)

    @property
    def workspace(self) -> torch.Tensor:
        if self._ws is None:
            self._ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def _check(self, t: torch.Tensor, dtype: torch.dtype, name: str):
        if not t.is_cuda or t.dtype != dtype:
            raise TypeError(f"{name}: expected a CUDA {dtype} tensor, got {t.dtype} on {t.device}")
        if t.storage_offset() < 0 or t.untyped_storage().nbytes() < (t.storage_offset() + self.n_elems) * t.element_size():
            raise ValueError(f"{name}: buffer smaller than the plan's layout")

    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        self._check(x, self.in_dtype, "x")
        if out is None:
            out = torch.empty_like(x, dtype=self.coef_dtype)
        self._check(out, self.coef_dtype, "out")
        abi.dwt2_forward(self.handle, x.data_ptr(), out.data_ptr(), self.workspace.data_ptr(),
                         _stream_handle(stream))
        return out

    def inverse(self, c: torch.Tensor, out: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        self._check(c, self.coef_dtype, "coef")
        if out is None:
            out = torch.empty_like(c, dtype=self.in_dtype)
        self._check(out, self.in_dtype, "out")
        abi.dwt2_inverse(self.handle, c.data_ptr(), out.data_ptr(), self.workspace.data_ptr(),
                         _stream_handle(stream))
        return out

    def adjoint(self, g: torch.Tensor, out: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        self._check(g, torch.float32, "coef_grad")
        if out is None:
            out = torch.empty_like(g)
        self._check(out, torch.float32, "out")
        abi.dwt2_adjoint(self.handle, g.data_ptr(), out.data_ptr(), self.workspace.data_ptr(),
                         _stream_handle(stream))
        return out

    def adjoint_l1(self, coef: torch.Tensor, scale: float, out: Optional[torch.Tensor] = None,
                   stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """Gradient of scale * sum|detail coefficients| w.r.t. the image, where
        coef = forward(image) (dwt2_adjoint_l1)."""
        self._check(coef, torch.float32, "coef")
        if out is None:
            out = torch.empty_like(coef)
        self._check(out, torch.float32, "out")
        abi.dwt2_adjoint_l1(self.handle, coef.data_ptr(), out.data_ptr(), float(scale), self.workspace.data_ptr(),
                            _stream_handle(stream))
        return out

    def coarsest_ll(self):
        """(offset, h, w, pitch) of every image's coarsest low-low band."""
        out = []
        for (o, h, w, p) in self.images:
            for _ in range(self.levels):
                h, w = (h + 1) // 2, (w + 1) // 2
            out.append((o, h, w, p))
        return out

    def n_detail(self) -> int:
        """Number of detail coefficients over all images and levels."""
        return sum(h * w for (_, h, w, _) in self.images) - sum(h * w for (_, h, w, _) in self.coarsest_ll())

    def tune_key(self) -> str:
        """Cache key of this plan's autotuning choice on this GPU and driver."""
        h = hashlib.sha256(repr(self.images).encode()).hexdigest()[:16]
        return "|".join([torch.cuda.get_device_name(self.device), str(torch.version.cuda), self.wavelet, self.scheme,
                         str(self.coef_dtype), str(self.levels), str(self.flags), h])

    def autotune(self, x: torch.Tensor, out: Optional[torch.Tensor] = None,
                 stream: Optional[torch.cuda.Stream] = None, cache: Optional[str] = None) -> int:
        """Pick the fastest launch configuration for this plan (dwt2_autotune).

        With ``cache`` (a JSON file, default $DWT2_TUNE_CACHE) an earlier choice
        for the same GPU, driver and plan is applied without timing, and a new
        choice is written back.  ``out`` is overwritten.
        """
        self._check(x, self.in_dtype, "x")
        if out is None:
            out = torch.empty_like(x, dtype=self.coef_dtype)
        cache = cache if cache is not None else os.environ.get("DWT2_TUNE_CACHE")
        key = self.tune_key()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        choice = int(table.get(key, -1))
        choice = abi.dwt2_autotune(self.handle, x.data_ptr(), out.data_ptr(), self.workspace.data_ptr(),
                                   _stream_handle(stream), choice)
        if cache and table.get(key) != choice:
            table[key] = choice
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        self.tuned = choice
        return choice

    def status(self, stream: Optional[torch.cuda.Stream] = None) -> int:
        return abi.dwt2_status(self.handle, _stream_handle(stream))

    def close(self):
        if getattr(self, "handle", None):
            abi.dwt2_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class DWT2Function(torch.autograd.Function):
    """coef = W(x) with backward dL/dx = W^T(dL/dcoef) from the adjoint kernel."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.forward(x.contiguous() if x.stride(-1) != 1 else x)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return ctx.plan.adjoint(g.contiguous()), None


def dwt2(x: torch.Tensor, plan: Plan) -> torch.Tensor:
    return DWT2Function.apply(x, plan)


def _abs_sum_images(c: torch.Tensor, regions) -> torch.Tensor:
    flat = c.reshape(-1)
    tot = torch.zeros((), dtype=torch.float64, device=c.device)
    for (o, h, w, p) in regions:
        tot = tot + flat[o:o + h * p].view(h, p)[:, :w].abs().sum(dtype=torch.float64)
    return tot


class L1DetailLoss(torch.autograd.Function):
    """mean |detail coefficients| of W(x) (every level, the coarsest LL
    excluded).  The backward is one dwt2_adjoint_l1 call: the sign of the
    coefficients is taken inside the adjoint kernel."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: Plan) -> torch.Tensor:
        c = plan.forward(x)
        ctx.plan = plan
        ctx.save_for_backward(c)
        n = plan.n_detail()
        total = _abs_sum_images(c, plan.images) - _abs_sum_images(c, plan.coarsest_ll())
        return (total / n).to(torch.float32)

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        (c,) = ctx.saved_tensors
        plan = ctx.plan
        # the upstream gradient stays on the device: the kernels read it, so
        # the backward neither synchronises nor leaves CUDA-graph capture
        g = gout.detach().to(device=c.device, dtype=torch.float32).reshape(1).contiguous()
        out = torch.empty_like(c)
        plan._check(out, torch.float32, "out")
        abi.dwt2_adjoint_l1_dev(plan.handle, c.data_ptr(), out.data_ptr(), g.data_ptr(), 1.0 / plan.n_detail(),
                                plan.workspace.data_ptr(), _stream_handle(None))
        ctx.keep = g  # alive until the kernels that read it have been queued after it
        return out, None


def l1_detail_loss(x: torch.Tensor, plan: Plan) -> torch.Tensor:
    return L1DetailLoss.apply(x, plan)


def band_rows(h: int, levels: int, n_bands: int, wavelet: str = "cdf97") -> List[Tuple[int, int, int, int]]:
    """(own0, own1, in0, in1) of every row band of an image of h rows
    (dwt2_band_rows)."""
    return [abi.dwt2_band_rows(WAVELETS[wavelet], levels, h, n_bands, b) for b in range(n_bands)]


class BandPlan:
    """Forward transform of one row band of an h x w image (dwt2_band_rows):
    a single-image plan over the band's rows [in0, in1) and the copy of the
    coefficients it owns into the image's Mallat layout (dwt2_band_stitch).
    Bands exchange no data: each can run on its own GPU from its own rows of
    the image."""

    def __init__(self, h: int, w: int, levels: int, n_bands: int, band: int, pitch: Optional[int] = None,
                 wavelet: str = "cdf97", scheme: str = "nonsep", coef_dtype: torch.dtype = torch.float32,
                 device: Optional[torch.device] = None):
        self.h, self.w, self.levels = h, w, levels
        self.n_bands, self.band = n_bands, band
        self.pitch = pitch if pitch is not None else w
        self.wavelet, self.coef_dtype = wavelet, coef_dtype
        self.own0, self.own1, self.in0, self.in1 = abi.dwt2_band_rows(WAVELETS[wavelet], levels, h, n_bands, band)
        self.plan = Plan.single(self.in1 - self.in0, w, levels, pitch=self.pitch, wavelet=wavelet, scheme=scheme,
                                coef_dtype=coef_dtype, device=device)
        self.band_coef = torch.empty((self.in1 - self.in0) * self.pitch, dtype=coef_dtype, device=self.plan.device)

    def forward_rows(self, x_rows: torch.Tensor, coef: torch.Tensor,
                     stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """x_rows: the image rows [in0, in1) (pitch elements each); coef: the
        whole image's coefficient buffer, of which the owned rectangles are
        written."""
        self.plan._check(x_rows, self.plan.in_dtype, "x_rows")
        st = _stream_handle(stream)
        abi.dwt2_forward(self.plan.handle, x_rows.data_ptr(), self.band_coef.data_ptr(),
                         self.plan.workspace.data_ptr(), st)
        abi.dwt2_band_stitch(WAVELETS[self.wavelet], self.levels, DTYPES[self.coef_dtype], self.h, self.w,
                             self.n_bands, self.band, self.band_coef.data_ptr(), self.pitch, coef.data_ptr(),
                             self.pitch, st)
        return coef

    def forward(self, x: torch.Tensor, coef: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
        """x: the whole image (h rows of pitch elements)."""
        rows = x.reshape(-1)[self.in0 * self.pitch:self.in1 * self.pitch]
        return self.forward_rows(rows, coef, stream)

    def close(self):
        self.plan.close()


def band_slices(h: int, w: int, levels: int) -> List[Tuple[int, str, slice, slice]]:
    """Mallat band rectangles (level, name, rows, cols); level 1 is the finest."""
    out = []
    for lev in range(1, levels + 1):
        hl, wl = (h + 1) // 2, (w + 1) // 2
        out.append((lev, "HL", slice(0, hl), slice(wl, w)))
        out.append((lev, "LH", slice(hl, h), slice(0, wl)))
        out.append((lev, "HH", slice(hl, h), slice(wl, w)))
        h, w = hl, wl
    out.append((levels, "LL", slice(0, h), slice(0, w)))
    return out
