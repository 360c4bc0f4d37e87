"""The matrix-product kernels in isolation, through the C ABI test hook:
CUDA-core FP32, tcgen05 kind::tf32 and kind::f16 (BF16), the three-term TF32 and six-term BF16 splits, against numpy.

Tolerances follow the arithmetic of each kind, for N(0,1) inputs (partial
sums grow like sqrt(k)): sequential FP32 accumulation of K products has an
error of about 2^-24 * K / sqrt(2) per output, so the max over all outputs
stays below 6 * 2^-24 * K; kind::tf32 keeps 10 explicit mantissa bits of each
input (relative error up to 2^-10 per operand, about 2e-3 per product), a
random sum of K of them stays below 8e-3 * sqrt(K); kind::f16 on
BF16-rounded inputs is compared with the product of the same rounded inputs,
so only the FP32 accumulation differs (6 * 2^-24 * K).  The three-term TF32
split (impl 3) represents each operand as hi + lo to ~2^-22 relative and drops
the lo*lo term, about 3 * 2^-22 per product: a random sum of K of them has a
standard deviation near 4e-7 * sqrt(K), and the largest of up to 17 million
outputs (8192 x 512 x 4) lies some 6 deviations out, on top of partial sums
accumulated inside the tensor core rather than in sequential IEEE order, so
the bound is 8e-6 * sqrt(K) on top of the FP32 accumulation bound."""
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


def _bf16(a):
    return torch.from_numpy(a).to(torch.bfloat16).float().numpy()


def _run(lib, impl, A, B):
    batch, M, K = A.shape
    N = B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.full((batch, M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.load().mes_gemm_selftest(impl, ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                      ctypes.c_void_p(dC.data_ptr()), M, N, K, batch, st)
    lib.check(rc, "mes_gemm_selftest")
    torch.cuda.synchronize()
    return dC.cpu().numpy()


# the last two give every CTA of the persistent kernel several tiles (more
# tiles than SMs), with ragged M and K, for both tile widths (N = 512 -> 256,
# N = 384 -> 128 wide tiles), so the accumulator hand-off between tiles runs
SHAPES = [(128, 128, 32, 1), (256, 256, 128, 1), (200, 300, 100, 1), (384, 512, 1920, 2),
          (128, 128, 4096, 1), (1000, 72, 648, 3), (8192, 512, 128, 4), (6000, 384, 200, 3)]


@pytest.mark.parametrize("M,N,K,batch", SHAPES)
@pytest.mark.parametrize("impl", [0, 1, 2, 3, 4])
def test_gemm_kernels(lib, impl, M, N, K, batch):
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((batch, M, K)).astype(np.float32)
    B = rng.standard_normal((batch, N, K)).astype(np.float32)
    u = 2.0 ** -24
    if impl == 2:
        Ar, Br = _bf16(A), _bf16(B)
        tol = 6 * u * K + 1e-6
    elif impl == 1:
        Ar, Br = A, B
        tol = 8e-3 * np.sqrt(K)
    elif impl == 3:
        Ar, Br = A, B
        tol = 6 * u * K + 8e-6 * np.sqrt(K) + 1e-6
    elif impl == 4:
        # six-term BF16 split: ~3 * 2^-24 per product; measured, its largest
        # error follows the three-term product's at small K (both limited by
        # the partial sums inside the tensor core) and stays at or below the
        # CUDA-core kernel's at K >= 1920, so it takes the same bound
        Ar, Br = A, B
        tol = 6 * u * K + 8e-6 * np.sqrt(K) + 1e-6
    else:
        Ar, Br = A, B
        tol = 6 * u * K + 1e-6
    if impl in (2, 4) and (K * 2) % 16:
        # BF16 rows of K elements are not a multiple of 16 bytes: the tensor
        # map cannot address them and the call must say so
        with pytest.raises(lib.MesError) as e:
            _run(lib, impl, A, B)
        assert e.value.name == "MES_ERR_INVALID_ARG"
        return
    want = np.einsum("bmk,bnk->bmn", Ar.astype(np.float64), Br.astype(np.float64))
    got = _run(lib, impl, A, B)
    assert np.isfinite(got).all()
    err = np.abs(got - want).max()
    print(f"impl {impl} {M}x{N}x{K}x{batch}: max error {err:.3e} (bound {tol:.3e})")
    assert err < tol, (impl, M, N, K, err, tol)
