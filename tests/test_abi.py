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
    assert lib.mes_reconstruct(fake, facs, 4, _i64([8, 6, 3, 2]), _i64([2, 2, 1, 1]), fake, fake, None, 0, None) == 1
    assert lib.mes_reconstruct(fake, facs, 4, _i64([8, 6, 3, 2]), _i64([2, 2, 1, 1]), fake, None, None, 9, None) == 1


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a tiny C program."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    out_dir = os.path.join(ROOT, "paper_2104_04726_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, f"layout_{struct}.c")
    exe = os.path.join(out_dir, f"layout_{struct}")
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    with open(src, "w") as fh:
        fh.write('#include <stddef.h>\n#include <stdio.h>\n#include "mes.h"\nint main(void) {\n'
                 f'  printf("%zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    vals = [int(x) for x in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("struct,cls", [("mes_als_opts", "MesAlsOpts"), ("mes_problem", "MesProblem"),
                                        ("mes_serve_stats", "MesServeStats")])
def test_struct_layout_matches_c(struct, cls):
    from paper_2104_04726_gb300 import _lib
    C = getattr(_lib, cls)
    names = [f for f, _ in C._fields_]
    size, offs = _c_layout(struct, names)
    assert size == ctypes.sizeof(C)
    assert offs == [getattr(C, f).offset for f in names]


def test_batch_and_server_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.mes_batch_create(0, ctypes.byref(h)) == 1
    assert lib.mes_batch_create(65, ctypes.byref(h)) == 1
    assert lib.mes_batch_run(None, None, 1, None, None) == 1
    assert lib.mes_batch_launch(None, None) == 1
    assert lib.mes_serve_create(0, 2, ctypes.byref(h)) == 1
    assert lib.mes_serve_create(1 << 30, 0, ctypes.byref(h)) == 1
    assert lib.mes_serve_submit(None, None, None) == 1
    assert lib.mes_batch_destroy(None) == 0 and lib.mes_serve_destroy(None) == 0


def test_workspace_size_query_without_gpu(lib):
    import paper_2104_04726_gb300 as mes
    a = mes.tucker_als_workspace_size([64, 48, 3, 6], [16, 12, 3, 6])
    b = mes.tucker_als_workspace_size([128, 96, 3, 6], [16, 12, 3, 6])
    c = mes.tucker_als_workspace_size([64, 48, 3, 6], [16, 12, 3, 6], "tf32")
    assert 0 < a < b
    # the TF32 form keeps a rounded copy of T and of the two large factors
    assert c - a >= 64 * 48 * 18 * 4
    n = ctypes.c_size_t()
    assert lib.mes_tucker_als_workspace_size(4, _i64([8, 6, 3, 2]), _i64([9, 2, 1, 1]), None, ctypes.byref(n)) == 2
    assert lib.mes_tucker_als_workspace_size(4, _i64([8, 6, 3, 2]), _i64([2, 2, 1, 1]), None, None) == 1


def test_init_option_validated_without_gpu(lib):
    from paper_2104_04726_gb300 import _lib
    n = ctypes.c_size_t()
    dims, ranks = _i64([8, 6, 3, 2]), _i64([2, 2, 1, 1])
    for init, want in ((0, 0), (1, 0), (2, 1), (-1, 1)):
        o = _lib.MesAlsOpts()
        o.init = init
        assert lib.mes_tucker_als_workspace_size(4, dims, ranks, ctypes.byref(o), ctypes.byref(n)) == want, init
    # both starts use the same workspace
    o0, o1 = _lib.MesAlsOpts(), _lib.MesAlsOpts()
    o1.init = 1
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    lib.mes_tucker_als_workspace_size(4, dims, ranks, ctypes.byref(o0), ctypes.byref(a))
    lib.mes_tucker_als_workspace_size(4, dims, ranks, ctypes.byref(o1), ctypes.byref(b))
    assert a.value == b.value


def test_colour_invert_validation_without_gpu(lib):
    bogus = ctypes.c_void_p(16)
    g = ctypes.c_float(2.2)
    assert lib.mes_colour_invert(None, 4, 4, 1, 0, g, bogus, None, None, None, None) == 1
    assert lib.mes_colour_invert(bogus, 4, 4, 1, 0, g, None, None, None, None, None) == 1
    assert lib.mes_colour_invert(bogus, 0, 4, 1, 0, g, bogus, None, None, None, None) == 1
    assert lib.mes_colour_invert(bogus, 4, 4, 1, 3, g, bogus, None, None, None, None) == 1
    assert lib.mes_colour_invert(bogus, 4, 4, 1, 2, ctypes.c_float(0.0), bogus, None, None, None, None) == 1
    assert lib.mes_colour_invert(bogus, 4, 4, 1, 2, g, bogus, None, bogus, None, None) == 1   # ref8 without sse8
    assert lib.mes_colour_invert(bogus, 4, 4, 1, 2, g, None, None, None, bogus, None) == 1    # sse8 without ref8
    assert lib.mes_colour_convert(bogus, 4, 4, 1, 3, g, bogus, None, None) == 1


def test_rate_bits_counts_core_scales_and_factors():
    import paper_2104_04726_gb300 as mes
    dims, ranks = [64, 48, 3, 6], [16, 12, 3, 6]
    factors = 64 * 16 + 48 * 12 + 3 * 3 + 6 * 6
    assert mes.rate_bits(dims, ranks, 8) == 16 * 12 * 18 * 8 + 18 * 32 + factors * 16
    assert mes.rate_bits(dims, ranks, 0) == 16 * 12 * 18 * 32 + factors * 16
    assert mes.rate_bits(dims, ranks, 4, factor_bits=8) == 16 * 12 * 18 * 4 + 18 * 32 + factors * 8


def test_quantiser_plane_count_cannot_wrap(lib):
    """Ranks whose product would overflow int64 are rejected before anything
    is enqueued (e.g. (1, 1, 2^62, 2) wraps to a negative plane count), by
    both quantiser entry points and the dequantiser; so are plane counts just
    above each entry point's limit (4096 without allocation, 65535 with)."""
    fake = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    for ranks in ([1, 1, 1 << 62, 2], [1, 1, 2, 1 << 62], [3, 5, 1 << 40, 1 << 40], [1 << 40, 1 << 30],
                  [2, 2, 65536]):
        assert lib.mes_quantize_core(fake, len(ranks), _i64(ranks), 8, fake, fake, 0, None) == 1, ranks
        assert lib.mes_dequantize_core(fake, fake, len(ranks), _i64(ranks), fake, None) == 1, ranks
        assert lib.mes_quantize_core_noalloc(fake, len(ranks), _i64(ranks), 8, fake, fake, None) == 1, ranks
    assert lib.mes_quantize_core_noalloc(fake, 3, _i64([2, 2, 4097]), 8, fake, fake, None) == 1
    assert b"4096 planes" in lib.mes_last_error()
