"""The C-ABI library loads and exports every symbol that include/*.h declares,
and the host-side argument checks work without a GPU (no compute calls)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ucp_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    from paper_0709_3331_gb300 import build as b
    b.build()
    from paper_0709_3331_gb300 import ucp
    return ucp.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 15
    for nm in sorted(names):
        assert hasattr(L, nm), nm
    from paper_0709_3331_gb300 import ucp
    assert set(ucp.EXPORTS) <= names


def test_strerror(L):
    for code in range(0, -7, -1):
        assert L.ucp_strerror(code)
    assert L.ucp_strerror(-99) == b"unknown error"


def test_create_rejects_bad_params_before_touching_the_device(L):
    from paper_0709_3331_gb300.ucp import ucp_params
    h = C.c_void_p()
    for kw in (dict(n=0), dict(leaf_cap=0), dict(leaf_cap=5000), dict(precision=7),
               dict(m=(0.0, 1.0)), dict(n=1 << 40)):
        p = ucp_params()
        p.n, p.leaf_cap, p.precision = 16, 4, 0
        p.q[0], p.q[1], p.m[0], p.m[1] = 1.0, -1.0, 1000.0, 1.0
        for k, v in kw.items():
            if k == "m":
                p.m[0], p.m[1] = v
            else:
                setattr(p, k, v)
        assert L.ucp_create(C.byref(h), C.byref(p)) == -1
    assert L.ucp_create(None, None) == -1


def test_binding_rejects_wrong_dtypes():
    from paper_0709_3331_gb300.ucp import _ptr
    with pytest.raises(TypeError):
        _ptr(np.zeros((4, 3), dtype=np.float32), np.float64)
    with pytest.raises(TypeError):
        _ptr(np.zeros((4, 3))[:, :2], np.float64)
    p, dev = _ptr(np.zeros((4, 3)), np.float64)
    assert dev == 0 and p


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_0709_3331_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert not re.search(r"(from|import)\s+oracle|liboracle|ucp_oracle", src), f


def test_walk_shape_count_matches_header():
    from paper_0709_3331_gb300 import ucp
    src = open(os.path.join(ROOT, "include", "ucp.h")).read()
    m = re.search(r"#define UCP_WALK_SHAPES (\d+)", src)
    assert m and int(m.group(1)) == ucp.UCP_WALK_SHAPES
    cu = open(os.path.join(ROOT, "paper_0709_3331_gb300", "csrc", "ucp_walk.cu")).read()
    tab = re.search(r"kShapes\[\]\[3\] = \{(.*?)\};", cu, flags=re.S).group(1)
    rows = tuple((int(a), int(b), int(c)) for a, b, c in
                 re.findall(r"\{(\d+), (\d+), (\d+)\}", tab))
    assert rows == ucp.WALK_SHAPE_TABLE and len(rows) == ucp.UCP_WALK_SHAPES


def test_walk_shape_rejects_null_context(L):
    L.ucp_set_walk_shape.argtypes = [C.c_void_p, C.c_int]
    assert L.ucp_set_walk_shape(None, 0) == -1
