"""Row bands of one image on one GPU: every band runs its own plan over its
rows (own rows plus halo) and stitches the coefficients it owns into one
buffer.  The stitched pyramid must equal the whole-image GPU pyramid bit for
bit (the same kernels do the same arithmetic on every owned coefficient) and
the oracle within the usual bound.  Two to four bands, two to five levels,
odd heights, every wavelet."""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import synth
from paper_1704_08657_gb300.dwt import BandPlan, Plan, round_up
from tests.util import assert_dd_close, assert_fp32_close, assert_lowp_close

pytestmark = pytest.mark.gpu

CASES = [(1000, 520, 2, 2), (2049, 700, 5, 2), (777, 301, 3, 3), (4097, 1500, 5, 4), (130, 250, 2, 2)]


def _banded(x, levels, n, pitch, **kw):
    h, w = x.shape[0], kw.pop("w")
    dt = kw.get("coef_dtype", torch.float32)
    coef = torch.full((h * pitch,), float("nan") if dt.is_floating_point else -7, dtype=dt, device="cuda")
    for b in range(n):
        bp = BandPlan(h, w, levels, n, b, pitch=pitch, **kw)
        bp.forward(x.reshape(-1), coef)
        torch.cuda.synchronize()
        assert bp.plan.status() == 0
        bp.close()
    return coef.view(h, pitch)


def _whole(x, levels, pitch, **kw):
    h, w = x.shape[0], kw.pop("w")
    p = Plan.single(h, w, levels, pitch=pitch, **kw)
    c = p.forward(x)
    torch.cuda.synchronize()
    assert p.status() == 0
    return c.view(h, pitch)


def _input(h, w, pitch, dtype=torch.float32, seed=1):
    x = synth.gradient(h, w, seed=seed)
    buf = torch.zeros((h, pitch), dtype=dtype, device="cuda")
    buf[:, :w] = torch.from_numpy(synth.to_int(x) if dtype == torch.int32 else x).to(dtype).cuda()
    return x, buf


@pytest.mark.parametrize("scheme", ["reduced", "sep"])
@pytest.mark.parametrize("h,w,levels,n", CASES)
def test_bands_cdf97(h, w, levels, n, scheme):
    pitch = round_up(w, 4)
    x, xd = _input(h, w, pitch, seed=h + w)
    got = _banded(xd, levels, n, pitch, w=w, scheme=scheme)
    whole = _whole(xd, levels, pitch, w=w, scheme=scheme)
    assert not torch.isnan(got[:, :w]).any(), "coefficients left unwritten"
    assert torch.equal(got[:, :w], whole[:, :w])
    assert_fp32_close(got[:, :w].cpu().numpy(), oracle.forward97(x.astype(np.float64), levels), levels, 255.0)


@pytest.mark.parametrize("h,w,levels,n", CASES[:3])
def test_bands_fp16_storage(h, w, levels, n):
    pitch = round_up(w, 4)
    x, xd = _input(h, w, pitch, seed=7)
    got = _banded(xd, levels, n, pitch, w=w, scheme="reduced", coef_dtype=torch.float16)
    whole = _whole(xd, levels, pitch, w=w, scheme="reduced", coef_dtype=torch.float16)
    assert torch.equal(got[:, :w], whole[:, :w])
    assert_lowp_close(got[:, :w].float().cpu().numpy(), oracle.forward97(x.astype(np.float64), levels), levels, 1e-3)


@pytest.mark.parametrize("h,w,levels,n", CASES)
def test_bands_int53_bit_exact(h, w, levels, n):
    pitch = round_up(w, 4)
    x, xd = _input(h, w, pitch, torch.int32, seed=3)
    got = _banded(xd, levels, n, pitch, w=w, wavelet="cdf53", scheme="nonsep", coef_dtype=torch.int32)
    ref = oracle.forward53i(synth.to_int(x).astype(np.int64), levels)
    assert np.array_equal(got[:, :w].cpu().numpy().astype(np.int64), ref)


@pytest.mark.parametrize("h,w,levels,n", CASES[:4])
def test_bands_dd137(h, w, levels, n):
    pitch = round_up(w, 4)
    x, xd = _input(h, w, pitch, seed=5)
    got = _banded(xd, levels, n, pitch, w=w, wavelet="dd137", scheme="nonsep")
    whole = _whole(xd, levels, pitch, w=w, wavelet="dd137", scheme="nonsep")
    assert torch.equal(got[:, :w], whole[:, :w])
    assert_dd_close(got[:, :w].cpu().numpy(), oracle.forward137(x.astype(np.float64), levels), levels, 255.0)
