"""Fused level pairs: levels l and l+1 in one launch, the low-low band between
them kept in a ring of rows in shared memory.

The fused kernel runs the same row pipelines on the same values as the
per-level launches, so its coefficients must equal theirs bit for bit; they
are also checked against the oracle.  Sizes cover odd and even sides at both
levels (the mirror rows of the bottom edge differ between the two), ragged
last blocks and segments, several blocks across and down, the smallest
eligible input (64 x 64), every scheme and coefficient type, and a guard band
that must stay untouched.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import synth
from paper_1704_08657_gb300.dwt import Plan
from tests.test_gpu_parity import SENT, _guard_ok, _padded
from tests.util import assert_fp32_close, assert_lowp_close

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 2), (66, 130, 2), (131, 67, 3), (512, 512, 5), (1000, 764, 4), (1030, 1094, 2),
          (2048, 2048, 5), (4097, 200, 4), (200, 4095, 4), (1535, 2173, 6)]


def _forward(x, levels, scheme, coef_dtype, wavelet, fuse_seg, fuse_pairs, monkeypatch):
    h, w = x.shape
    in_dt = torch.float32 if wavelet == "cdf97" else torch.int32
    xin, pitch = _padded(x, in_dt)
    out = torch.full_like(xin, SENT, dtype=coef_dtype)
    monkeypatch.setenv("DWT2_FUSE_SEG", str(fuse_seg))
    monkeypatch.setenv("DWT2_FUSE_PAIRS", str(fuse_pairs))
    plan = Plan.single(h, w, levels, pitch=pitch, wavelet=wavelet, scheme=scheme, coef_dtype=coef_dtype)
    plan.forward(xin, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert _guard_ok(out, h, w), "forward wrote outside the coefficient region"
    return out[:h, :w].cpu()


@pytest.mark.parametrize("h,w,levels", SHAPES)
@pytest.mark.parametrize("scheme", ["reduced", "nonsep", "sep"])
def test_fused_equals_per_level_and_oracle(h, w, levels, scheme, monkeypatch):
    x = synth.gradient(h, w, seed=h + w)
    fused = _forward(x, levels, scheme, torch.float32, "cdf97", 16, 9, monkeypatch)
    per = _forward(x, levels, scheme, torch.float32, "cdf97", 0, 0, monkeypatch)
    assert torch.equal(fused, per), "fused and per-level coefficients differ"
    ref = oracle.forward97(x.astype(np.float64), levels)
    assert_fp32_close(fused.numpy(), ref, levels, 255.0, f"fused {scheme} {h}x{w}")


@pytest.mark.parametrize("seg", [2, 3, 7, 24, 48, 1000])
def test_fused_segment_heights(seg, monkeypatch):
    # short, odd and whole-height segments (one block column per segment row)
    h, w, levels = 771, 1286, 3
    x = synth.noisy(h, w, seed=seg)
    fused = _forward(x, levels, "reduced", torch.float32, "cdf97", seg, 1, monkeypatch)
    per = _forward(x, levels, "reduced", torch.float32, "cdf97", 0, 0, monkeypatch)
    assert torch.equal(fused, per)


@pytest.mark.parametrize("dtype,rel", [(torch.float16, 1e-3), (torch.bfloat16, 8e-3)])
def test_fused_low_precision_storage(dtype, rel, monkeypatch):
    h, w, levels = 1000, 1502, 4
    x = synth.uniform(h, w, seed=3)
    fused = _forward(x, levels, "reduced", dtype, "cdf97", 16, 2, monkeypatch)
    per = _forward(x, levels, "reduced", dtype, "cdf97", 0, 0, monkeypatch)
    assert torch.equal(fused, per)
    assert_lowp_close(fused.float().numpy(), oracle.forward97(x.astype(np.float64), levels), levels, rel, "fused")


@pytest.mark.parametrize("scheme", ["nonsep", "sep"])
@pytest.mark.parametrize("h,w", [(64, 64), (1001, 763), (2048, 1030)])
def test_fused_int53_exact(scheme, h, w, monkeypatch):
    x = synth.to_int(synth.noisy(h, w, seed=7))
    levels = 4
    fused = _forward(x, levels, scheme, torch.int32, "cdf53", 16, 2, monkeypatch)
    assert np.array_equal(fused.numpy().astype(np.int64), oracle.forward53i(x.astype(np.int64), levels))


def test_fused_batch_of_images(monkeypatch):
    # a multi-image plan fuses each image's level pair when every image is eligible
    shapes = [(64, 64), (300, 517), (1024, 96), (130, 2050)]
    buf, descs = synth.batch_pack(shapes, seed=2)
    xd = torch.from_numpy(buf.astype(np.float32)).cuda()
    outs = []
    for fuse in (16, 0):
        monkeypatch.setenv("DWT2_FUSE_SEG", str(fuse))
        plan = Plan(descs, 3, scheme="nonsep")
        outs.append(plan.forward(xd, torch.zeros_like(xd)))
        torch.cuda.synchronize()
        assert plan.status() == 0
    assert torch.equal(outs[0], outs[1])
