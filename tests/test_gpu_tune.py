"""Tile autotuner of the tensor-core products: in a fresh process with
MES_TUNE=1 and MES_TUNE_CACHE=<file>, every product shape is timed over its
candidate tile widths and split-K factors on first use, the results stay
correct, the choices are written to the cache, and a second process that
loads the cache gives the same results bit for bit."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import ctypes, sys
    import numpy as np
    import torch
    sys.path.insert(0, %r)
    from paper_2104_04726_gb300 import _lib
    lib = _lib.load()
    out = []
    for impl, (M, N, K, b) in [(1, (384, 256, 1920, 1)), (2, (256, 512, 1024, 3)), (3, (200, 384, 640, 1))]:
        rng = np.random.default_rng(M + N + K)
        A = rng.standard_normal((b, M, K)).astype(np.float32)
        B = rng.standard_normal((b, N, K)).astype(np.float32)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        for rep in range(2):
            dC = torch.full((b, M, N), float("nan"), device="cuda")
            st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            _lib.check(lib.mes_gemm_selftest(impl, ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                             ctypes.c_void_p(dC.data_ptr()), M, N, K, b, st), "selftest")
            torch.cuda.synchronize()
            C = dC.cpu().numpy()
            if impl == 2:
                A_, B_ = torch.from_numpy(A).bfloat16().float().numpy(), torch.from_numpy(B).bfloat16().float().numpy()
            else:
                A_, B_ = A, B
            want = np.einsum("bmk,bnk->bmn", A_.astype(np.float64), B_.astype(np.float64))
            tol = 8e-3 * np.sqrt(K) if impl == 1 else 6 * 2.0 ** -24 * K + 3e-6 * np.sqrt(K) + 1e-6
            assert np.isfinite(C).all() and np.abs(C - want).max() < tol, (impl, np.abs(C - want).max(), tol)
            out.append(C.tobytes())
    np.save(sys.argv[1], np.frombuffer(b"".join(out), dtype=np.uint8))
""") % ROOT


def _child(tmp_path, name, cache):
    env = dict(os.environ, MES_TUNE="1", MES_TUNE_CACHE=str(cache))
    res = tmp_path / name
    r = subprocess.run([sys.executable, "-c", CHILD, str(res)], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return (tmp_path / (name + ".npy")).read_bytes()


def test_autotuner_caches_and_reproduces(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    cache = tmp_path / "tune.txt"
    first = _child(tmp_path, "a", cache)
    lines = [ln for ln in cache.read_text().splitlines() if " = " in ln]
    assert len(lines) >= 3, lines
    for ln in lines:
        bn, splits = (int(x) for x in ln.split(" = ")[1].split())
        assert bn in (128, 256) and splits >= 1
    second = _child(tmp_path, "b", cache)
    assert first == second
    assert len([ln for ln in cache.read_text().splitlines() if " = " in ln]) == len(lines)
