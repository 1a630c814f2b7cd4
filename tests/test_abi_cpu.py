"""The C ABI library on the CPU: it builds, loads, exports every function the
header declares, and validates plans before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_1704_08657_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "dwt2.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dwt2_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_function(lib):
    names = _declared_functions()
    assert set(names) == set(abi.EXPORTS)
    for n in names:
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_checked_build_exports_the_same_functions(lib):
    """libdwt2_checked.so (DWT2_CHECKED, built by build_all() or by its GPU
    test) exports every declared function and says it is the checked build;
    the normal library says it is not (a child process loads the checked one:
    the library is chosen per process)."""
    import subprocess
    import sys
    assert lib.dwt2_checked() == 0
    if not build.up_to_date(checked=True):
        pytest.skip("libdwt2_checked.so not built here (build.build_all())")
    code = ("from paper_1704_08657_gb300 import abi; l = abi.load(); "
            "[getattr(l, n) for n in abi.EXPORTS]; print(l.dwt2_checked(), abi.LIB_PATH)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, DWT2_LIBRARY="checked"), timeout=300)
    assert r.returncode == 0, r.stderr
    flag, path = r.stdout.split()
    assert flag == "1" and path.endswith("libdwt2_checked.so")


def test_strerror_names_every_code(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert abi.dwt2_strerror(code) and abi.dwt2_strerror(code) != "unknown error"
    assert abi.dwt2_strerror(-99) == "unknown error"


@pytest.mark.parametrize("args,code", [
    ((abi.DWT2_CDF97, 0, 0, 0, 0, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_INVALID_ARG),          # levels 0
    ((abi.DWT2_CDF97, 1, 1, 0, 0, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_INVALID_ARG),          # boundary
    ((7, 1, 0, 0, 0, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_INVALID_ARG),                        # wavelet
    ((abi.DWT2_CDF97, 1, 0, 0, 0, 9, [(0, 16, 16, 16)]), abi.DWT2_ERR_INVALID_ARG),          # scheme
    ((abi.DWT2_CDF97, 1, 0, 0, 0, 0, [(0, 16, 16, 8)]), abi.DWT2_ERR_INVALID_ARG),           # pitch < w
    ((abi.DWT2_CDF97, 1, 0, 0, 0, 0, [(0, 16, 16, 18)]), abi.DWT2_ERR_MISALIGNED),           # pitch % 4
    ((abi.DWT2_CDF97, 1, 0, 0, 0, 0, [(2, 16, 16, 16)]), abi.DWT2_ERR_MISALIGNED),           # offset % 4
    ((abi.DWT2_CDF97, 5, 0, 0, 0, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_LEVELS_TOO_DEEP),      # 16->8->4->2->1
    ((abi.DWT2_CDF97, 2, 0, 0, 0, 0, [(0, 3, 16, 16)]), abi.DWT2_ERR_LEVELS_TOO_DEEP),       # 3->2->1 ok? no: 2 levels ok
    ((abi.DWT2_CDF97, 1, 0, abi.DWT2_I32, 0, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_CDF97, 1, 0, 0, abi.DWT2_I32, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_CDF53_INT, 1, 0, abi.DWT2_I32, abi.DWT2_I32, abi.DWT2_NONSEP_REDUCED, [(0, 16, 16, 16)]),
     abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_CDF53_INT, 1, 0, abi.DWT2_F32, abi.DWT2_F32, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_CDF97, 1, 0, 0, 0, 6, [(0, 16, 16, 16)]), abi.DWT2_ERR_INVALID_ARG),          # past NONSEP_CONV
    ((abi.DWT2_CDF53_INT, 1, 0, abi.DWT2_I32, abi.DWT2_I32, abi.DWT2_POLYCONV, [(0, 16, 16, 16)]),
     abi.DWT2_ERR_UNSUPPORTED),                                                             # floor: lifting only
    ((abi.DWT2_CDF53_INT, 1, 0, abi.DWT2_I32, abi.DWT2_I32, abi.DWT2_CONV, [(0, 16, 16, 16)]),
     abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_CDF53_INT, 1, 0, abi.DWT2_I32, abi.DWT2_I32, abi.DWT2_NONSEP_CONV, [(0, 16, 16, 16)]),
     abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_DD137, 1, 0, 0, 0, abi.DWT2_POLYCONV, [(0, 16, 16, 16)]), abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_DD137, 1, 0, 0, 0, abi.DWT2_CONV, [(0, 16, 16, 16)]), abi.DWT2_ERR_UNSUPPORTED),
    ((abi.DWT2_DD137, 1, 0, abi.DWT2_I32, abi.DWT2_I32, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_UNSUPPORTED),
    ((3, 1, 0, 0, 0, 0, [(0, 16, 16, 16)]), abi.DWT2_ERR_INVALID_ARG),                       # no such wavelet
])
def test_plan_validation(lib, args, code):
    wav, lv, bd, idt, cdt, sch, imgs = args
    if code == abi.DWT2_ERR_LEVELS_TOO_DEEP and imgs[0][1] == 3:
        # 3 -> 2 -> 1: two levels are legal (inputs 3 and 2); three are not
        args = (wav, 3, bd, idt, cdt, sch, imgs)
        wav, lv, bd, idt, cdt, sch, imgs = args
    with pytest.raises(abi.Dwt2Error) as e:
        abi.dwt2_plan(wav, lv, bd, idt, cdt, sch, imgs)
    assert e.value.code == code


def test_dd137_has_no_persistent_form(lib):
    with pytest.raises(abi.Dwt2Error) as e:
        abi.dwt2_plan(abi.DWT2_DD137, 1, 0, 0, 0, abi.DWT2_NONSEP, [(0, 16, 16, 16)], abi.DWT2_FLAG_PERSISTENT)
    assert e.value.code == abi.DWT2_ERR_UNSUPPORTED


@pytest.mark.parametrize("scheme", [abi.DWT2_POLYCONV, abi.DWT2_CONV, abi.DWT2_NONSEP_CONV])
def test_filter_bank_schemes_have_no_persistent_form(lib, scheme):
    with pytest.raises(abi.Dwt2Error) as e:
        abi.dwt2_plan(abi.DWT2_CDF97, 1, 0, 0, 0, scheme, [(0, 16, 16, 16)], abi.DWT2_FLAG_PERSISTENT)
    assert e.value.code == abi.DWT2_ERR_UNSUPPORTED


def test_null_arguments(lib):
    assert lib.dwt2_plan(None, 0, 1, 0, 0, 0, 0, 0, None, 0) == abi.DWT2_ERR_INVALID_ARG
    for n in ("dwt2_forward", "dwt2_inverse", "dwt2_adjoint"):
        assert abi.raw_call(n, 0, 0, 0) == abi.DWT2_ERR_INVALID_ARG
    assert lib.dwt2_workspace_bytes(None) == 0
    lib.dwt2_destroy(None)
