"""dwt2_forward_noalloc against dwt2_forward, through the C ABI.

dwt2_forward_noalloc serves callers that cannot allocate device memory when
they transform (code that runs during a CUDA graph capture that forbids
cudaMalloc, real-time pipelines with no allocation after start-up, plug-ins
whose host owns all device memory): it keeps the intermediate low-low bands in
a static device array of the library instead of a caller workspace and needs
no plan.  Its output must match the planned forward within the FP32 tolerance
of the other parity tests, on two calls in a row (the second call finds the
first call's data left in the shared array).

The file name sorts last so that a run that stops at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_1704_08657_gb300 import abi, build, synth
from paper_1704_08657_gb300.dwt import Plan, round_up
from tests.util import assert_fp32_close

pytestmark = pytest.mark.gpu


def _image(h, w, seed):
    pitch = round_up(w, 4)
    x = torch.zeros((h, pitch), dtype=torch.float32, device="cuda")
    x[:, :w] = torch.from_numpy(synth.uniform(h, w, seed=seed)).cuda()
    return x, pitch


def test_noalloc_matches_planned_forward_on_two_calls():
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    h, w, levels = 1000, 764, 5
    for call, seed in enumerate((21, 22)):
        x, pitch = _image(h, w, seed)
        plan = Plan.single(h, w, levels, pitch=pitch, scheme="reduced")
        ref = plan.forward(x)
        got = torch.full_like(x, -1.0)
        rc = abi.dwt2_forward_noalloc(abi.DWT2_CDF97, levels, abi.DWT2_NONSEP_REDUCED, abi.DWT2_F32, h, w, pitch,
                                      x.data_ptr(), got.data_ptr(), stream)
        assert rc == abi.DWT2_OK, abi.dwt2_strerror(rc)
        torch.cuda.synchronize()
        g = got[:, :w].cpu().numpy().astype(np.float64)
        r = ref[:, :w].cpu().numpy().astype(np.float64)
        assert_fp32_close(g, r, levels, 255.0, f"noalloc call {call}")
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    x = torch.zeros(16, device="cuda")
    # level-1 low-low band of 8192 x 8192 needs 64 MiB, more than the 32 MiB scratch
    rc = abi.dwt2_forward_noalloc(abi.DWT2_CDF97, 2, abi.DWT2_NONSEP, abi.DWT2_F32, 8192, 8192, 8192,
                                  x.data_ptr(), x.data_ptr(), 0)
    assert rc == abi.DWT2_ERR_TOO_LARGE
    assert "noalloc" in abi.dwt2_strerror(rc)
