"""The C-ABI library: it builds, loads, exports every symbol the header
declares, and rejects bad arguments before touching a GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2007_04457_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = []
    for h in HEADERS:
        text = open(h).read()
        names += re.findall(r"^MGARD_API\s+[^(]*?\b(mgard_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = gbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("mgard_plan_create", "mgard_decompose", "mgard_recompose",
                     "mgard_workspace_bytes", "mgard_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} is declared in include/ but not exported"


def test_status_strings(lib):
    lib.mgard_status_string.restype = ctypes.c_char_p
    assert lib.mgard_status_string(0) == b"MGARD_OK"
    assert lib.mgard_status_string(3) == b"MGARD_ERR_WORKSPACE"
    assert lib.mgard_status_string(99) == b"MGARD_ERR_UNKNOWN"


def _create(lib, dims, nlevels=-1, dtype=0, coords=None):
    lib.mgard_plan_create.restype = ctypes.c_int
    d = (ctypes.c_int64 * len(dims))(*dims)
    out = ctypes.c_void_p()
    rc = lib.mgard_plan_create(len(dims), d, nlevels, coords, dtype, ctypes.byref(out))
    return rc, out.value


def test_plan_create_rejects_bad_shapes_without_gpu(lib):
    lib.mgard_last_error.restype = ctypes.c_char_p
    assert _create(lib, [10, 10], nlevels=1)[0] == 2  # (n-1) not divisible by 2
    assert b"divisible" in lib.mgard_last_error()
    assert _create(lib, [17, 17], nlevels=5)[0] == 2  # 16 not divisible by 32
    assert _create(lib, [1, 1])[0] == 2             # nothing left after squeezing
    assert _create(lib, [5, 5, 5, 5])[0] == 2       # 4 dims
    assert _create(lib, [17], dtype=7)[0] == 1      # unknown dtype
    assert _create(lib, [17], nlevels=-2)[0] == 1


def test_plan_create_rejects_bad_coordinates(lib):
    xs = (ctypes.c_double * 5)(0.0, 0.5, 0.4, 0.7, 1.0)  # not increasing
    arr = (ctypes.POINTER(ctypes.c_double) * 1)(ctypes.cast(xs, ctypes.POINTER(ctypes.c_double)))
    assert _create(lib, [5], coords=arr)[0] == 1


def test_null_arguments(lib):
    lib.mgard_decompose.restype = ctypes.c_int
    assert lib.mgard_decompose(None, None, None, 0, None) == 1
    lib.mgard_recompose_classes.restype = ctypes.c_int
    assert lib.mgard_recompose_classes(None, 1, None, None, 0, None) == 1
    lib.mgard_plan_destroy.restype = ctypes.c_int
    assert lib.mgard_plan_destroy(None) == 0
    lib.mgard_workspace_bytes.restype = ctypes.c_size_t
    assert lib.mgard_workspace_bytes(None) == 0
    lib.mgard_probe_fp64_peak.restype = ctypes.c_int
    assert lib.mgard_probe_fp64_peak(None, None) == 1
    for name in ("mgard_quantize", "mgard_dequantize"):
        getattr(lib, name).restype = ctypes.c_int
        assert getattr(lib, name)(None, None, None, None, None) == 1
    for name in ("mgard_decompose_quantize", "mgard_dequantize_recompose"):
        getattr(lib, name).restype = ctypes.c_int
        assert getattr(lib, name)(None, None, None, None, None, ctypes.c_size_t(0), None) == 1
