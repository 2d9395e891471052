"""The C-ABI library loads and exports every entry point include/*.h
declares; argument checks that need no device return their status codes."""
import ctypes
import re
from pathlib import Path

import pytest

import paper_2501_12349_b300 as fp
from paper_2501_12349_b300 import _build

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return fp.lib()


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(fp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    assert fp.fp_status_string(0) == "ok"
    assert "invalid" in fp.fp_status_string(-1)
    o = fp.fp_opts_default()
    assert o.bbox_tol == 0.1 and o.M == 0 and o.newton_tol == 1e-10 and o.max_iter == 50
    assert o.dist_tol == 1e-10 and o.precision == fp.FP_F64 and o.point_order == fp.FP_ORDER_CELL


def test_argument_checks_without_device(lib):
    h = ctypes.c_void_p()
    # NULL coordinates, bad dimension pairs, unsupported order
    assert lib.fp_setup(None, 3, 3, 4, 10, None, None, ctypes.byref(h)) == fp.FP_EINVAL
    assert lib.fp_setup(ctypes.c_void_p(8), 2, 3, 4, 10, None, None, ctypes.byref(h)) == fp.FP_EINVAL
    assert lib.fp_setup(ctypes.c_void_p(8), 3, 3, 9, 10, None, None, ctypes.byref(h)) == fp.FP_EUNSUPPORTED
    assert lib.fp_setup(ctypes.c_void_p(8), 3, 3, 4, 0, None, None, ctypes.byref(h)) == fp.FP_EINVAL
    assert lib.fp_setup(ctypes.c_void_p(8), 3, 3, 4, 10, None, None, None) == fp.FP_EINVAL
    assert lib.fp_findpts(None, None, 0, None, None, None, None, None) == fp.FP_EINVAL
    assert lib.fp_eval(None, None, None, None, 0, None, 1, None, None) == fp.FP_EINVAL
    assert lib.fp_free(None) == fp.FP_EINVAL
    assert lib.fp_set_precision(None, 0) == fp.FP_EINVAL
    assert lib.fp_set_point_order(None, fp.FP_ORDER_CELL) == fp.FP_EINVAL
    assert lib.fp_findpts_host(None, None, 10, None, None, None, None, None, 0, None, 0, None) == fp.FP_EINVAL


def test_header_constants_match_binding():
    """Every integer #define FP_* of the header has the same value in the binding."""
    text = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "findpts.h").read_text(), flags=re.S)
    seen = 0
    for name, expr in re.findall(r"^#define (FP_\w+)[ \t]+([-0-9() <]+?)[ \t]*$", text, flags=re.M):
        if hasattr(fp, name):
            assert getattr(fp, name) == eval(expr), name
            seen += 1
    assert seen >= 15 and fp.FP_NSTATS == 16
