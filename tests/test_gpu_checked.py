"""The range-checked build (libdwt2_checked.so, DWT2_CHECKED): the parity
suite of small, odd and ragged shapes for every wavelet, scheme and dtype, the
grouped and persistent batches, the adjoint and the no-alloc entry, run
against the oracle through the checked library, where every global access of
the transform kernels is first tested against its buffer.  Every plan's status
word must stay DWT2_OK (a tripped check reads DWT2_ERR_DEVICE_CHECK), so the
kernels' index arithmetic stays inside its buffers on all these shapes.

The library is chosen per process (DWT2_LIBRARY=checked), so the suites run
in a child pytest process.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# node ids run in the child process: the whole parity suite, the batched and
# persistent paths, the adjoint's gradients and the no-alloc entry
CHECKED_SUITES = [
    "tests/test_gpu_checked.py::test_checked_library_is_loaded",
    "tests/test_gpu_parity.py",
    "tests/test_gpu_persistent.py::test_persistent_single_image",
    "tests/test_gpu_persistent.py::test_batch_inverse_adjoint_and_l1",
    "tests/test_gpu_persistent.py::test_grouped_batch_equals_single_image_plans",
    "tests/test_gpu_grad.py::test_l1_gradient_matches_oracle_transpose",
    "tests/test_zz_no_alloc.py",
]


def test_checked_library_is_loaded():
    """In the child process: the checked build is the one loaded."""
    if os.environ.get("DWT2_LIBRARY") != "checked":
        pytest.skip("runs in the checked child process")
    from paper_1704_08657_gb300 import abi
    assert abi.load().dwt2_checked() == 1
    assert abi.LIB_PATH.endswith("libdwt2_checked.so")


def test_parity_suites_under_the_checked_build():
    if os.environ.get("DWT2_LIBRARY") == "checked":
        pytest.skip("the parent process runs the child")
    from paper_1704_08657_gb300 import build
    build.build(checked=True)  # a no-op when build() made it already
    env = dict(os.environ, DWT2_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *CHECKED_SUITES], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "skipped" not in r.stdout.split("\n")[-2], tail
