"""The factorization and solve of one CholeskyQR pass (the r x r Cholesky
and the right-side triangular solve of the factor update after Eq. 8) in
isolation, through the C ABI test hook, against float64 numpy.

Every kernel form is reached: the one-CTA factorization (r <= 128), the
8-CTA shared-memory cluster (128 < r <= 512) and the cluster through L2
(r > 512); the wide solve (r <= 384, whole and ragged row blocks, float4
and scalar paths) and the narrow one (r > 384).

Bounds.  With A = D^-1 H D^-1 (unit diagonal) the computed factor
satisfies L L^T = A + E with |E| <= gamma_{r+1} |L| |L^T| (Higham, Thm 10.3),
and the entries of |L| |L^T| are at most 1 for a unit diagonal, so
max |L L^T - A| <= (r + 1) u (u = 2^-24); the gate is twice that.  The
solve V L^T = W D^-1 is backward stable row by row (the 32 x 32 diagonal
blocks are applied as their computed inverses, well conditioned here), so
its residual is gated at 4 r u relative to |V| |L^T| plus 32 u cond(L_kk)
for the largest condition number of a 32 x 32 diagonal block (they are
applied as computed inverses), and its forward error against the float64
solution at cond(L) times that."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24
MES_ERR_NONFINITE = 6


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2104_04726_gb300 import _lib
    return _lib


def _spd(r, cond, rng):
    """H = D0 Q diag(lam) Q^T D0: eigenvalues log-spaced over `cond`, rows
    scaled by 10^U(-2, 2) so the equilibration matters."""
    Q, _ = np.linalg.qr(rng.standard_normal((r, r)))
    lam = np.logspace(0.0, -np.log10(cond), r)
    d0 = 10.0 ** rng.uniform(-2, 2, r)
    H = (Q * lam) @ Q.T
    return (d0[:, None] * H * d0[None, :]).astype(np.float32)


def _run(lib, H, W):
    r, s = H.shape[0], W.shape[0]
    dH = torch.from_numpy(np.asfortranarray(H).ravel(order="F").copy()).cuda()
    dW = torch.from_numpy(np.asfortranarray(W).ravel(order="F").copy()).cuda()
    dL = torch.zeros(r * r, dtype=torch.float32, device="cuda")
    dd = torch.full((r,), float("nan"), dtype=torch.float32, device="cuda")
    dV = torch.full((s * r,), float("nan"), dtype=torch.float32, device="cuda")
    restarts = ctypes.c_int(-1)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.load().mes_solve_selftest(ctypes.c_void_p(dH.data_ptr()), r, ctypes.c_void_p(dW.data_ptr()), s,
                                       ctypes.c_void_p(dL.data_ptr()), ctypes.c_void_p(dd.data_ptr()),
                                       ctypes.c_void_p(dV.data_ptr()), ctypes.byref(restarts), st)
    torch.cuda.synchronize()
    L = np.tril(dL.cpu().numpy().astype(np.float64).reshape(r, r, order="F"))
    V = dV.cpu().numpy().astype(np.float64).reshape(s, r, order="F")
    return rc, L, dd.cpu().numpy().astype(np.float64), V, restarts.value


CASES = [(1, 5), (33, 100), (128, 1000), (129, 64), (200, 777), (256, 11520), (384, 7680), (385, 500),
         (512, 2048), (513, 96), (700, 300)]


@pytest.mark.parametrize("r,s", CASES)
def test_factor_and_solve_against_float64(lib, r, s):
    rng = np.random.default_rng(1000 * r + s)
    H = _spd(r, 1e3, rng)
    W = rng.standard_normal((s, r)).astype(np.float32)
    rc, L, dinv, V, restarts = _run(lib, H, W)
    lib.check(rc, "mes_solve_selftest")
    assert restarts == 0
    H64 = H.astype(np.float64)
    d_ref = 1.0 / np.sqrt(np.diag(H64))
    assert np.max(np.abs(dinv / d_ref - 1.0)) <= 8 * U
    A = dinv[:, None] * H64 * dinv[None, :]
    res_L = np.max(np.abs(L @ L.T - A))
    assert res_L <= 2 * (r + 1) * U, res_L
    Wd = W.astype(np.float64) * dinv[None, :]
    L64 = np.linalg.cholesky(A)
    # the diagonal blocks are applied as computed inverses: each adds about
    # 32 u cond(L_kk) relative to the block's part of the solution
    kb = max(np.linalg.cond(L64[k:k + 32, k:k + 32]) for k in range(0, r, 32))
    tol = 4 * r * U + 32 * kb * U
    res_V = np.linalg.norm(V @ L.T - Wd) / (np.linalg.norm(np.abs(V) @ np.abs(L.T)) + 1e-300)
    assert res_V <= tol, (res_V, tol)
    V64 = np.linalg.solve(L64, Wd.T).T
    fwd = np.linalg.norm(V - V64) / np.linalg.norm(V64)
    assert fwd <= np.linalg.cond(L64) * tol, fwd


def test_nonpositive_diagonal_is_reported(lib):
    H = np.eye(40, dtype=np.float32)
    H[5, 5] = -1.0
    W = np.ones((10, 40), dtype=np.float32)
    rc, *_ = _run(lib, H, W)
    assert rc == MES_ERR_NONFINITE


def test_indefinite_matrix_raises_the_shift(lib):
    """A unit-diagonal matrix with a negative eigenvalue: the factorization
    meets a pivot below its floor, raises its diagonal shift and restarts;
    the count comes back and the outputs stay finite."""
    H = np.eye(40)
    B = np.array([[1.0, 0.9, 0.9], [0.9, 1.0, -0.9], [0.9, -0.9, 1.0]])
    assert np.linalg.eigvalsh(B)[0] < 0
    H[10:13, 10:13] = B
    W = np.ones((64, 40), dtype=np.float32)
    rc, L, dinv, V, restarts = _run(lib, H.astype(np.float32), W)
    lib.check(rc, "mes_solve_selftest")
    assert restarts >= 1
    assert np.all(np.isfinite(L)) and np.all(np.isfinite(V))
