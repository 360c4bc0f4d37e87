"""The C ABI library builds, loads and exports every entry point declared in
include/mes.h; argument validation runs on the host before anything is
enqueued (no GPU needed for these calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2104_04726_gb300 import _lib
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "mes.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mes_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "mes_tucker_als" in names and "mes_colour_convert" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2104_04726_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_opts_struct_matches_header(lib):
    from paper_2104_04726_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "mes.h")).read()
    body = src[src.index("typedef struct mes_als_opts"):src.index("} mes_als_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\*?\s*\b(\w+);", body)
    assert [f for f, _ in _lib.MesAlsOpts._fields_] == fields


def test_version(lib):
    assert lib.mes_version().decode().startswith("mes ")


def _i64(v):
    return (ctypes.c_int64 * len(v))(*v)


def test_validation_without_gpu(lib):
    fake = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    assert lib.mes_colour_convert(None, 4, 4, 1, 0, ctypes.c_float(2.2), fake, None, None) == 1
    assert lib.mes_colour_convert(fake, 0, 4, 1, 0, ctypes.c_float(2.2), fake, None, None) == 1
    assert lib.mes_colour_convert(fake, 4, 4, 1, 7, ctypes.c_float(2.2), fake, None, None) == 1
    assert lib.mes_colour_convert(fake, 4, 4, 1, 1, ctypes.c_float(0.0), fake, None, None) == 1
    facs = (ctypes.c_void_p * 4)(16, 16, 16, 16)
    # rank above the mode size
    st = lib.mes_tucker_als(fake, 4, _i64([8, 6, 3, 2]), _i64([9, 2, 1, 1]), 5, 0.0, fake, facs, None, None, None)
    assert st == 2
    # rank above the product of the other ranks
    st = lib.mes_tucker_als(fake, 4, _i64([8, 6, 3, 2]), _i64([5, 2, 1, 2]), 5, 0.0, fake, facs, None, None, None)
    assert st == 2
    assert b"product of the other ranks" in lib.mes_last_error()
    # order out of range, max_iters, small mode too large
    assert lib.mes_tucker_als(fake, 1, _i64([8]), _i64([2]), 5, 0.0, fake, facs, None, None, None) == 1
    assert lib.mes_tucker_als(fake, 4, _i64([8, 6, 3, 2]), _i64([2, 2, 1, 1]), 0, 0.0, fake, facs, None, None, None) == 1
    assert lib.mes_tucker_als(fake, 3, _i64([8, 6, 40]), _i64([2, 2, 2]), 3, 0.0, fake, facs, None, None, None) == 1
    assert lib.mes_quantize_core(fake, 2, _i64([4, 4]), 1, fake, fake, 0, None) == 1
    assert lib.mes_quantize_core(fake, 2, _i64([4, 4]), 17, fake, fake, 0, None) == 1
    assert lib.mes_quantize_core(None, 2, _i64([4, 4]), 8, fake, fake, 0, None) == 1
    assert lib.mes_reconstruct(fake, facs, 4, _i64([8, 6, 3, 2]), _i64([2, 2, 1, 1]), fake, fake, None, None) == 1
