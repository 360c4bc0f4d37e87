"""The quantiser entry point that allocates nothing (for callers that must not
call the device allocator while they run, e.g. a serving loop with a fixed
memory budget).  It must give exactly what mes_quantize_core gives, call
after call, although every call reuses the same fixed device array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2104_04726_gb300 import _lib
    return _lib


def _i64(v):
    return (ctypes.c_int64 * len(v))(*v)


def _quant(lib, fn, core, ranks, bits):
    q = torch.empty(core.shape, dtype=torch.int16, device="cuda")
    P = int(np.prod(ranks[2:])) if len(ranks) > 2 else 1
    sc = torch.empty((P,), dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = lib.load()
    if fn == "alloc":
        rc = L.mes_quantize_core(ctypes.c_void_p(core.data_ptr()), len(ranks), _i64(ranks), bits,
                                 ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(sc.data_ptr()), 0, st)
    else:
        rc = L.mes_quantize_core_noalloc(ctypes.c_void_p(core.data_ptr()), len(ranks), _i64(ranks), bits,
                                         ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(sc.data_ptr()), st)
    lib.check(rc, fn)
    torch.cuda.synchronize()
    return q.cpu().numpy(), sc.cpu().numpy()


def test_matches_allocating_quantiser_on_consecutive_calls(lib):
    rng = np.random.default_rng(77)
    ranks = (48, 40, 3, 10)
    # first call on large values, second on values 1000x smaller: stale
    # per-plane maxima left in the shared array would show in the second call
    for call, scale in enumerate((1e3, 1.0)):
        core_np = (rng.standard_normal(ranks[::-1]) * scale).astype(np.float32)
        core = torch.from_numpy(core_np).cuda()
        q_ref, s_ref = _quant(lib, "alloc", core, ranks, 12)
        q, s = _quant(lib, "noalloc", core, ranks, 12)
        assert np.array_equal(s, s_ref), call
        assert np.array_equal(q, q_ref), call


def test_rejects_more_planes_than_its_fixed_scratch(lib):
    core = torch.zeros((4097, 2, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.MesError) as e:
        _quant(lib, "noalloc", core, (2, 2, 4097), 8)
    assert e.value.name == "MES_ERR_INVALID_ARG"


@pytest.mark.parametrize("ranks", [(8, 8, 4096), (37, 29)])
def test_largest_plane_count_and_order_two_core(lib, ranks):
    """Exactly 4096 planes, where the fixed scratch is used to its last word,
    and an order-2 core (one plane, no trailing modes): the same codes and
    scales as the allocating quantiser, on two calls in a row."""
    rng = np.random.default_rng(sum(ranks))
    for call in range(2):
        core_np = (rng.standard_normal(ranks[::-1]) * (10.0 ** (2 - 2 * call))).astype(np.float32)
        core = torch.from_numpy(core_np).cuda()
        q_ref, s_ref = _quant(lib, "alloc", core, ranks, 10)
        q, s = _quant(lib, "noalloc", core, ranks, 10)
        assert np.array_equal(s, s_ref), (ranks, call)
        assert np.array_equal(q, q_ref), (ranks, call)
