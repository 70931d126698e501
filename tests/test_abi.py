"""The C-ABI library loads without a GPU and exports what include/mbir.h declares;
host-side argument validation needs no device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2108_01438_gb300 import mbir, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mbir_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(mbir.LIB_PATH):
        from paper_2108_01438_gb300 import build
        build.build()
    return mbir.lib()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(mbir.exported_symbols()) | declared
    assert set(mbir.exported_symbols()) <= declared


def test_status_strings(lib):
    for code in range(-6, 1):
        assert lib.mbir_status_string(code).decode()
    assert lib.mbir_status_string(12345).decode() == "unknown status"


def _create(lib, d, **over):
    g, keep = mbir.make_geometry(d)
    for k, v in over.items():
        setattr(g, k, v)
    h = C.c_void_p()
    rc = lib.mbir_plan_create(C.byref(g), None, C.byref(h))
    return rc, h


@pytest.mark.parametrize("field,value,code", [
    ("nx", 0, -1), ("nz", -3, -1), ("m", 0, -1), ("dx_um", 0.0, -1), ("dz_um", -1.0, -1),
    ("precision", 7, -1), ("kb_width", 5, -2), ("kb_width", 10, -2), ("kb_oversamp", 1.5, -2),
    ("nx", 11, -2), ("nx", 8192, -2), ("nz", 4, -2), ("nz", 11 * 8, -2), ("na", float("nan"), -1),
])
def test_plan_rejects_bad_geometry_on_host(lib, field, value, code):
    d = workloads.geometry(16, 32, 24)
    rc, h = _create(lib, d, **{field: value})
    assert rc == code and not h.value


def test_plan_rejects_non_monotone_wavenumbers(lib):
    d = workloads.geometry(16, 32, 24)
    k = np.array(d["k"])
    k[5], k[6] = k[6], k[5]
    d["k"] = k
    rc, h = _create(lib, d)
    assert rc == -1


def test_null_arguments(lib):
    assert lib.mbir_forward(None, None, None, None, None) == -1
    assert lib.mbir_adjoint(None, None, None, None, None) == -1
    h = C.c_void_p()
    assert lib.mbir_plan_create(None, None, C.byref(h)) == -1
    lib.mbir_plan_destroy(None)
