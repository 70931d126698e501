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
    ("nx", 2053, -2), ("nx", 8192, -2), ("nz", 4, -2), ("nz", 11 * 8, -2), ("na", float("nan"), -1),
])
def test_plan_rejects_bad_geometry_on_host(lib, field, value, code):
    d = workloads.geometry(16, 32, 24)
    rc, h = _create(lib, d, **{field: value})
    assert rc == code and not h.value


@pytest.mark.parametrize("ny,dy,over,code", [
    (1, 2.0, {}, -1), (0, 2.0, {}, -1), (4, float("nan"), {}, -1), (2053, 2.0, {}, -2), (5000, 2.0, {}, -2),
    (2048, 2.0, {"size": (1024, 1024, 1024)}, -2), (8, 2.0, {"kb_width": 5}, -2),
])
def test_volume_plan_rejects_bad_sizes_on_host(lib, ny, dy, over, code):
    """A second lateral axis: ny >= 2 with the width rule of nx, the volume below
    2^31 elements; checked before any device work."""
    over = dict(over)
    g, keep = mbir.make_geometry(workloads.geometry(*over.pop("size", (16, 32, 24))))
    for k, v in over.items():
        setattr(g, k, v)
    h = C.c_void_p()
    assert lib.mbir_volume_plan_create(C.byref(g), ny, dy, None, C.byref(h)) == code
    assert not h.value


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


# ctypes type of each C field type used in include/mbir.h
_CTYPE = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "size_t": C.c_size_t}


def _c_structs():
    """{typedef name: [(field, C type text), ...]} of the header's plain structs."""
    text = open(os.path.join(ROOT, "include", "mbir.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const )?\w+\s*\**)\s*(.*)", decl)
            ctype, names = m.group(1).replace(" ", ""), m.group(2)
            for n in names.split(","):
                n = n.strip()
                stars = len(n) - len(n.lstrip("*"))
                fields.append((n.lstrip("*"), ctype + "*" * stars))
        out[name] = fields
    return out


@pytest.mark.parametrize("cname,pyname", [
    ("mbir_geometry", "Geometry"), ("mbir_solve_opts", "SolveOpts"), ("mbir_solve_info", "SolveInfo"),
    ("mbir_lambda_search_info", "LambdaSearchInfo"), ("mbir_tuning", "Tuning"),
    ("mbir_profile_entry", "ProfileEntry"),
])
def test_binding_structs_match_the_header(cname, pyname):
    """Field order, count and type of every ctypes struct equal the C declaration
    (a field added on one side only would shift every later one)."""
    cf = _c_structs()[cname]
    pf = getattr(mbir, pyname)._fields_
    assert len(cf) == len(pf), (cname, [f for f, _ in cf], [f for f, _ in pf])
    for (cn, ct), (pn, pt) in zip(cf, pf):
        if ct.endswith("*"):
            assert pt is C.c_char_p or issubclass(pt, C._Pointer) or pt is C.c_void_p, (cname, cn, pt)
        else:
            assert pt is _CTYPE[ct], (cname, cn, ct, pt)
        assert pn.replace("lam", "lambda") == cn or pn == cn, (cname, cn, pn)
    assert C.sizeof(getattr(mbir, pyname)) >= 8 * (len(pf) // 2)


def test_new_entry_points_validate_on_the_host(lib):
    """NULL plans and arguments are refused before any device work."""
    assert lib.mbir_adjoint_hilbert(None, None, None, None, None) == -1
    assert lib.mbir_isam_interpolated(None, None, None, None, None) == -1
    r = C.c_double()
    assert lib.mbir_ncc(None, None, None, C.byref(r), None) == -1
    info = mbir.LambdaSearchInfo()
    o = mbir.SolveOpts()
    assert lib.mbir_lambda_search(None, None, None, None, C.byref(o), -3.0, 0.0, 5, None, C.byref(info), None) == -1
    assert lib.mbir_prox_tv(None, None, 0.5, 5, None, None) == -1
