"""dwt2_forward_noalloc against the oracle and against dwt2_forward, through
the C ABI.

dwt2_forward_noalloc serves callers that cannot allocate device memory when
they transform (code that runs during a CUDA graph capture that forbids
cudaMalloc, real-time pipelines with no allocation after start-up, plug-ins
whose host owns all device memory): it keeps the intermediate low-low bands in
a static device array of the library instead of a caller workspace and needs
no plan.  Every wavelet, coefficient type and scheme it accepts, at one and
five levels, must match the FP64 / int64 oracle within the bounds of the other
parity tests (integer 5/3 bit for bit) and the planned forward bit for bit, on
two calls in a row (the second call finds the first call's data left in the
shared array), and its status word must read clear.

The file name sorts last so that a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import abi, build, synth
from paper_1704_08657_gb300.dwt import Plan, round_up
from tests.util import assert_fp32_close, assert_lowp_close

pytestmark = pytest.mark.gpu

SCHEMES = {"nonsep": abi.DWT2_NONSEP, "reduced": abi.DWT2_NONSEP_REDUCED, "sep": abi.DWT2_SEP_LIFTING}
DT = {torch.float32: abi.DWT2_F32, torch.float16: abi.DWT2_F16, torch.bfloat16: abi.DWT2_BF16,
      torch.int32: abi.DWT2_I32}
CASES = ([("cdf97", s, d) for d in (torch.float32, torch.float16, torch.bfloat16) for s in ("nonsep", "reduced", "sep")]
         + [("cdf53", s, torch.int32) for s in ("nonsep", "sep")])


def _image(h, w, pitch, seed, integer):
    x = synth.uniform(h, w, seed=seed)
    if integer:
        x = synth.to_int(x)
    buf = torch.zeros((h, pitch), dtype=torch.int32 if integer else torch.float32, device="cuda")
    buf[:, :w] = torch.from_numpy(x).cuda()
    return x, buf


@pytest.mark.parametrize("levels", [1, 5])
@pytest.mark.parametrize("wavelet,scheme,cdt", CASES)
def test_noalloc_matches_oracle_on_two_calls(wavelet, scheme, cdt, levels):
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    integer = wavelet == "cdf53"
    # an odd width with a pitch wider than round4(w), then an even size
    for call, (h, w, pitch, seed) in enumerate(((1001, 763, 772, 21), (640, 1000, 1000, 22))):
        x, xd = _image(h, w, pitch, seed, integer)
        got = torch.full((h, pitch), -1, dtype=cdt, device="cuda")
        rc = abi.dwt2_forward_noalloc(abi.DWT2_CDF53_INT if integer else abi.DWT2_CDF97, levels, SCHEMES[scheme],
                                      DT[cdt], h, w, pitch, xd.data_ptr(), got.data_ptr(), stream)
        assert rc == abi.DWT2_OK, abi.dwt2_strerror(rc)
        assert abi.dwt2_noalloc_status(stream) == abi.DWT2_OK
        g = got[:, :w].cpu()
        assert (got[:, w:].cpu() == -1).all(), "wrote past the image width"
        if integer:
            ref = oracle.forward53i(x.astype(np.int64), levels)
            assert np.array_equal(g.numpy().astype(np.int64), ref), f"call {call}"
        else:
            ref = oracle.forward97(x.astype(np.float64), levels)
            if cdt == torch.float32:
                assert_fp32_close(g.numpy(), ref, levels, 255.0, f"noalloc call {call}")
            else:
                assert_lowp_close(g.float().numpy(), ref, levels, 1e-3 if cdt == torch.float16 else 8e-3,
                                  f"noalloc call {call}")
        # the planned forward computes the same coefficients, bit for bit
        plan = Plan.single(h, w, levels, pitch=pitch, wavelet=wavelet, scheme=scheme, coef_dtype=cdt)
        planned = plan.forward(xd)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert torch.equal(planned[:, :w].cpu(), g)
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    x = torch.zeros(16, device="cuda")
    # level-1 low-low band of 8192 x 8192 needs 64 MiB, more than the 32 MiB scratch
    rc = abi.dwt2_forward_noalloc(abi.DWT2_CDF97, 2, abi.DWT2_NONSEP, abi.DWT2_F32, 8192, 8192, 8192,
                                  x.data_ptr(), x.data_ptr(), 0)
    assert rc == abi.DWT2_ERR_TOO_LARGE
    assert "noalloc" in abi.dwt2_strerror(rc)
    # the documented limit: 5176 x 5176 fits at any depth, 5180 x 5180 does not
    big = torch.zeros(5180 * 5180, device="cuda")
    out = torch.zeros_like(big)
    rc = abi.dwt2_forward_noalloc(abi.DWT2_CDF97, 5, abi.DWT2_NONSEP, abi.DWT2_F32, 5180, 5180, 5180,
                                  big.data_ptr(), out.data_ptr(), 0)
    assert rc == abi.DWT2_ERR_TOO_LARGE
    rc = abi.dwt2_forward_noalloc(abi.DWT2_CDF97, 5, abi.DWT2_NONSEP, abi.DWT2_F32, 5176, 5176, 5176,
                                  big.data_ptr(), out.data_ptr(), 0)
    assert rc == abi.DWT2_OK
    assert abi.dwt2_noalloc_status(0) == abi.DWT2_OK
