"""Inter-level overlap of the single-image forward pyramid.

Every level after the first is launched as a programmatic dependent of the
previous one and waits only for the previous level's segments it reads (per-
segment completion counters, bounded waits).  The coefficients must equal
those of launches that wait for the whole previous grid, bit for bit, for
every scheme, coefficient type and tuned configuration; a dropped completion
signal must surface as DWT2_ERR_TIMEOUT without hanging.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import abi, synth
from paper_1704_08657_gb300.dwt import Plan
from tests.test_gpu_parity import _padded
from tests.util import assert_dd_close, assert_fp32_close

pytestmark = pytest.mark.gpu


def _run(x, levels, scheme, coef_dtype, overlap, monkeypatch, choice=None, wavelet="cdf97"):
    """x: host array; odd widths get a padded pitch (a multiple of 4)."""
    monkeypatch.setenv("DWT2_LEVEL_OVERLAP", "1" if overlap else "0")
    h, w = x.shape
    xin, pitch = _padded(x, torch.int32 if wavelet == "cdf53" else torch.float32, guard_rows=0)
    plan = Plan.single(h, w, levels, pitch=pitch, scheme=scheme, coef_dtype=coef_dtype, wavelet=wavelet)
    out = torch.full_like(xin, float("nan") if coef_dtype != torch.int32 else 0, dtype=coef_dtype)
    if choice is not None:
        assert abi.dwt2_autotune(plan.handle, xin.data_ptr(), out.data_ptr(), plan.workspace.data_ptr(), 0,
                                 choice) == choice
    c = plan.forward(xin, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return c[:, :w].cpu()


@pytest.mark.parametrize("h,w,levels", [(2048, 2048, 5), (1031, 2050, 6), (300, 4100, 4), (4099, 130, 5),
                                        (66, 66, 3), (5000, 3000, 5)])
@pytest.mark.parametrize("scheme", ["reduced", "sep", "conv", "nsconv"])
def test_overlap_equals_grid_waits(h, w, levels, scheme, monkeypatch):
    x = synth.gradient(h, w, seed=h ^ w)
    a = _run(x, levels, scheme, torch.float32, True, monkeypatch)
    b = _run(x, levels, scheme, torch.float32, False, monkeypatch)
    assert not torch.isnan(a).any(), "coefficients left unwritten"
    assert torch.equal(a, b)
    if h * w <= 4_200_000:
        assert_fp32_close(a.numpy(), oracle.forward97(x.astype(np.float64), levels), levels, 255.0)


@pytest.mark.parametrize("choice", [0, 1, 2 | (10 << 6) | (21 << 12) | (31 << 18), 31 * (1 + 64 + 4096 + 262144)])
def test_overlap_with_tuned_segment_heights(choice, monkeypatch):
    # segment heights 2..32 and the four configurations, mixed across levels
    x = synth.uniform(3001, 2222, seed=5)
    a = _run(x, 5, "reduced", torch.float16, True, monkeypatch, choice)
    b = _run(x, 5, "reduced", torch.float16, False, monkeypatch, choice)
    assert not torch.isnan(a).any()
    assert torch.equal(a, b)


def test_overlap_int53(monkeypatch):
    x = synth.to_int(synth.noisy(1500, 1700, seed=3))
    a = _run(x, 5, "nonsep", torch.int32, True, monkeypatch, wavelet="cdf53")
    assert np.array_equal(a.numpy().astype(np.int64), oracle.forward53i(x.astype(np.int64), 5))


def test_dropped_segment_signal_times_out(monkeypatch):
    monkeypatch.setenv("DWT2_TIMEOUT_MS", "30")
    monkeypatch.setenv("DWT2_LEVEL_OVERLAP", "1")
    h = w = 1024
    x = torch.from_numpy(synth.uniform(h, w, seed=1)).cuda()
    plan = Plan.single(h, w, 3, flags=abi.DWT2_TESTONLY_DROP_SIGNAL)
    plan.forward(x)
    assert plan.status() == abi.DWT2_ERR_TIMEOUT
    assert plan.status() == 0
    ok = Plan.single(h, w, 3)
    c = ok.forward(x)
    assert ok.status() == 0
    assert_fp32_close(c.cpu().numpy(), oracle.forward97(x.cpu().numpy().astype(np.float64), 3), 3, 255.0)


@pytest.mark.parametrize("h,w,levels", [(2048, 2048, 5), (1031, 2052, 6), (300, 4100, 4), (66, 66, 3)])
@pytest.mark.parametrize("scheme", ["nonsep", "reduced", "sep"])
def test_overlap_dd137(h, w, levels, scheme, monkeypatch):
    # three warm-up rows: a unit waits for one more row of the previous level
    x = synth.gradient(h, w, seed=h + w)
    a = _run(x, levels, scheme, torch.float32, True, monkeypatch, wavelet="dd137")
    b = _run(x, levels, scheme, torch.float32, False, monkeypatch, wavelet="dd137")
    assert not torch.isnan(a).any(), "coefficients left unwritten"
    assert torch.equal(a, b)
    assert_dd_close(a.numpy(), oracle.forward137(x.astype(np.float64), levels), levels, 255.0)
