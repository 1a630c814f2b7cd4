"""The bench workload at full size, in the launch configuration bench.py times.

16384 x 16384 FP32 gradient image (seed 2), five levels, each scheme autotuned
per level exactly as bench.py does, every coefficient compared with the FP64
oracle (the C oracle transforms the whole image in a few seconds on the host
cores); FP16 storage and the integer 5/3 path at the same size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import synth
from paper_1704_08657_gb300.dwt import Plan
from tests.util import assert_dd_close, assert_fp32_close, assert_lowp_close, report_band_errors

pytestmark = pytest.mark.gpu

N, LEVELS = 16384, 5


@pytest.fixture(scope="module")
def image():
    x = synth.gradient(N, N, seed=2)
    return x, oracle.forward97(x.astype(np.float64), LEVELS)


@pytest.mark.parametrize("scheme", ["reduced", "sep", "nonsep", "polyconv", "conv", "nsconv"])
def test_bench_workload_matches_oracle(image, scheme):
    x, ref = image
    xd = torch.from_numpy(x).cuda()
    plan = Plan.single(N, N, LEVELS, scheme=scheme)
    out = torch.empty_like(xd)
    plan.autotune(xd, out)
    out.fill_(float("nan"))
    plan.forward(xd, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    report_band_errors(got, ref, LEVELS, 255.0, f"16384^2 {scheme} FP32")
    assert_fp32_close(got, ref, LEVELS, 255.0, f"16384^2 {scheme}")
    plan.close()


def test_bench_workload_fp16_storage(image):
    x, ref = image
    xd = torch.from_numpy(x).cuda()
    plan = Plan.single(N, N, LEVELS, scheme="reduced", coef_dtype=torch.float16)
    out = torch.empty_like(xd, dtype=torch.float16)
    plan.autotune(xd, out)
    c = plan.forward(xd, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    report_band_errors(c.float().cpu().numpy(), ref, LEVELS, 255.0, "16384^2 reduced FP16 storage")
    assert_lowp_close(c.float().cpu().numpy(), ref, LEVELS, 1e-3, "16384^2 fp16")
    plan.close()


@pytest.mark.parametrize("scheme", ["nonsep", "sep"])
def test_int53_full_size_bit_exact(scheme):
    x = synth.to_int(synth.gradient(N, N, seed=2))
    ref = oracle.forward53i(x.astype(np.int64), LEVELS)
    xd = torch.from_numpy(x).cuda()
    plan = Plan.single(N, N, LEVELS, wavelet="cdf53", scheme=scheme, coef_dtype=torch.int32)
    out = torch.empty_like(xd)
    plan.autotune(xd, out)
    c = plan.forward(xd, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = c.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, ref), f"{int((got != ref).sum())} coefficients differ"
    back = plan.inverse(c)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), x)
    plan.close()


@pytest.mark.parametrize("scheme", ["nonsep", "reduced"])
def test_dd137_full_size(scheme):
    x = synth.gradient(N, N, seed=2)
    ref = oracle.forward137(x.astype(np.float64), LEVELS)
    xd = torch.from_numpy(x).cuda()
    plan = Plan.single(N, N, LEVELS, wavelet="dd137", scheme=scheme)
    out = torch.empty_like(xd)
    plan.autotune(xd, out)
    out.fill_(float("nan"))
    plan.forward(xd, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert_dd_close(got, ref, LEVELS, 255.0, f"16384^2 dd137 {scheme}")
    back = plan.inverse(out)
    torch.cuda.synchronize()
    assert float((back - xd).abs().max()) <= 2e-3
    plan.close()
