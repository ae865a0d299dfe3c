"""C ABI checks that need no GPU: the library builds, loads, exports every entry point that
include/dmk.h declares, and rejects invalid plans before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2606_27134_b300 import build, dmk

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dmk.h")


def declared():
    txt = open(HDR).read()
    return sorted(set(re.findall(r"^\s*(?:dmk_status_t|const char\*)\s+(dmk_\w+)\s*\(", txt, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    lib = dmk.load()
    for code in range(9):
        assert lib.dmk_status_string(code)
    assert dmk.status_string(0) == "ok"


@pytest.mark.parametrize("args,code", [
    (("laplace", 3, (1, 1, 1), 1e-2), 1),          # tol outside the table range
    (("laplace", 5, (1, 1, 1), 1e-6), 1),          # D out of range
    (("laplace", 3, (1, -1, 1), 1e-6), 1),         # negative length
    (("laplace", 3, (1, 1, 2000), 1e-6), 4),       # more than 1024 cubes in the tiling
    (("laplace", 3, (1, 40, 30), 1e-6), 4),        # the same with padded axes (42 x 32 cubes)
])
def test_invalid_plans_rejected_before_device(args, code):
    kernel, D, L, tol = args
    with pytest.raises(dmk.DmkError) as e:
        dmk.Plan(kernel, D, L, tol)
    assert e.value.status == code
    assert dmk.last_plan_error()


def test_plan_info_of_non_exact_tilings():
    """Sec. 4.1.1: a periodic length that the cube side does not divide is tiled by
    ceil(L_i / s) cubes plus one padding cube on each side (L = [1, 1.3, 1.7]: 1 x 4 x 4)."""
    info = dmk.plan_info("laplace", 3, [1, 1.3, 1.7], 1e-6)
    assert info["M"] == [1, 4, 4] and info["s"] == 1.0
    info = dmk.plan_info("rotlet", 2, [2, 1.3, 0.7], 1e-6)
    assert info["M"] == [4, 1, 1] and info["s"] == 1.3      # s = 1.3; axis 0 padded: ceil(2 / 1.3) + 2


def test_bad_precision_and_leaf_size():
    lib = dmk.load()
    h = ctypes.c_void_p()
    L = (ctypes.c_double * 3)(1, 1, 1)
    assert lib.dmk_plan_ex(0, 3, L, 1e-6, 7, 250, None, ctypes.byref(h)) == 1
    assert lib.dmk_plan_ex(0, 3, L, 1e-6, 1, 0, None, ctypes.byref(h)) == 1
    assert lib.dmk_plan_ex(0, 3, None, 1e-6, 1, 250, None, ctypes.byref(h)) == 1
    assert lib.dmk_destroy(None) == 0


def test_peaks_library_exports_its_entry_point():
    path = build.build_peaks()
    lib = ctypes.CDLL(path)
    assert hasattr(lib, "dmk_peak_measure")


def test_stats_struct_matches_header():
    """dmk_stats_t as ctypes lays it out (the binding) against the header's field list."""
    txt = open(HDR).read()
    body = txt[txt.index("typedef struct {", txt.index("DMK_ERR_TIMEOUT")):txt.index("} dmk_stats_t;")]
    names = re.findall(r"^\s*(?:int32_t|int64_t|float)\s+(\w+)", body, re.M)
    assert names == [f for f, _ in dmk.Stats._fields_]
    assert ctypes.sizeof(dmk.Stats) == 112
