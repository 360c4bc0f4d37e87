"""Tucker-ALS (HOOI) of Section III-B, written from the paper's definitions.

Notation follows the paper: the stack tensor T in R^{s_1 x ... x s_N}, the
core Q in R^{R_1 x ... x R_N} and the factors S^(n) in R^{s_n x R_n} with
orthonormal columns, so that T ~= Q x_1 S^(1) x_2 ... x_N S^(N) (Eq. 1,
element-wise Eq. 2).

* Initialisation: truncated HOSVD (Eq. 3 to Eq. 7).  Eq. 3 and Eq. 4 are
  garbled in the text (they take "the SVD of the mode-r unfolding of Q"); the
  reading used is the standard one: S^(r) holds the leading k_r left singular
  vectors of the mode-r unfolding of T, and the truncated core is
  T x_1 S^(1)T ... x_N S^(N)T (Eq. 5 and Eq. 7).  The singular vectors are
  taken as eigenvectors of the unfolding's Gram, as the paper does for the
  sweeps (text after Eq. 8).
* Interlaced initialisation (st_hosvd): the paper's cheaper alternative to
  T-HOSVD; mode n's factor comes from the tensor already truncated in modes
  1..n-1.  Pinned by the exact error identity of sequential projections.
* Sweep: for n = 1..N in order, Y^(n) = T x_{i != n} S^(i)T (Eq. 8), and
  S^(n) = the R_n leading left singular vectors of Y^(n)_(n), computed as the
  leading eigenvectors of the Gram Y^(n)_(n) Y^(n)_(n)^T.
* Core and fit (the paper is silent on the stopping rule): after mode N the
  core is Q = Y^(N) x_N S^(N)T; with orthonormal factors
  ||T - T_hat||^2 = ||T||^2 - ||Q||^2, so fit = 1 - sqrt(max(||T||^2 -
  ||Q||^2, 0)) / ||T||.  Stop when a sweep after the first changes the fit
  by less than tol, or after max_iters sweeps.
* Sign convention (not in the paper; makes the factors unique when the
  eigenvalues are simple): in every column of S^(n) the entry of largest
  magnitude (lowest index on ties) is positive; the core is recomputed from
  the signed factors.

Tensors are numpy arrays of shape (s_1, ..., s_N); memory order is
irrelevant here.
"""
from __future__ import annotations

import dataclasses
import numpy as np


def unfold(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding T_(n): rows indexed by mode n, columns by the rest."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1)


def mode_product(T: np.ndarray, A: np.ndarray, n: int) -> np.ndarray:
    """(T x_n A)(i_1..j..i_N) = sum_{i_n} T(i_1..i_n..i_N) A(j, i_n)."""
    out = np.tensordot(A, T, axes=(1, n))      # new mode first
    return np.moveaxis(out, 0, n)


def multi_mode_product(T: np.ndarray, mats, skip=None, transpose=False) -> np.ndarray:
    """T x_1 M_1 x_2 ... x_N M_N, skipping mode `skip`; M_n^T if transpose."""
    out = T
    for n, M in enumerate(mats):
        if n == skip or M is None:
            continue
        out = mode_product(out, M.T if transpose else M, n)
    return out


def leading_eigvecs(G: np.ndarray, r: int):
    """The r eigenvectors of symmetric G with the largest eigenvalues,
    in descending eigenvalue order, and those eigenvalues."""
    w, V = np.linalg.eigh(G)
    order = np.argsort(-w, kind="stable")[:r]
    return V[:, order], w[order]


def gram(M: np.ndarray) -> np.ndarray:
    return M @ M.T


def fix_signs(U: np.ndarray) -> np.ndarray:
    """Flip each column so its largest-magnitude entry (first on ties) is > 0."""
    U = U.copy()
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s


def core_of(T: np.ndarray, factors) -> np.ndarray:
    """Q = T x_1 S^(1)T ... x_N S^(N)T (Eq. 5 / Eq. 7)."""
    return multi_mode_product(T, factors, transpose=True)


def reconstruct(core: np.ndarray, factors) -> np.ndarray:
    """T_hat = Q x_1 S^(1) ... x_N S^(N) (Eq. 1)."""
    return multi_mode_product(core, factors, transpose=False)


def fit_from_norms(norm2_T: float, norm2_Q: float) -> float:
    return 1.0 - np.sqrt(max(norm2_T - norm2_Q, 0.0)) / np.sqrt(norm2_T)


def thosvd(T: np.ndarray, ranks):
    """Truncated HOSVD (Eq. 6, Eq. 7): leading k_r left singular vectors of
    each unfolding, via the Gram eigenvectors."""
    factors = []
    for n, r in enumerate(ranks):
        Tn = unfold(T, n)
        U, _ = leading_eigvecs(gram(Tn), r)
        factors.append(U)
    return factors


def st_hosvd(T: np.ndarray, ranks):
    """Interlaced (sequentially truncated) HOSVD, which the paper offers as
    the cheaper way to the initial factors (end of the initialisation
    subsection, after Eq. 7).  Modes are taken in the order 1..N; each mode's
    factor holds the leading r_n eigenvectors of the Gram of the tensor
    already truncated in the earlier modes, and the tensor is then truncated
    in that mode:  S^(n) from G_(n) G_(n)^T,  G <- G x_n S^(n)T.
    Returns the factors and, per mode, the energy that step drops (trace of
    the Gram minus its kept eigenvalues)."""
    G = np.asarray(T, dtype=np.float64)
    factors, dropped = [], []
    for n, r in enumerate(ranks):
        Gn = gram(unfold(G, n))
        U, lead = leading_eigvecs(Gn, r)
        factors.append(U)
        dropped.append(float(np.trace(Gn) - np.sum(lead)))
        G = mode_product(G, U.T, n)
    return factors, dropped


@dataclasses.dataclass
class TuckerResult:
    core: np.ndarray
    factors: list
    fit: float
    iters: int
    fit_history: list


def hooi(T: np.ndarray, ranks, max_iters: int, tol: float,
         init_factors=None) -> TuckerResult:
    """Tucker-ALS / HOOI (Section III-B), T-HOSVD initialised."""
    T = np.asarray(T, dtype=np.float64)
    N = T.ndim
    ranks = tuple(int(r) for r in ranks)
    assert len(ranks) == N
    norm2_T = float(np.sum(T * T))
    if init_factors is None:
        factors = thosvd(T, ranks)
    else:
        factors = [np.asarray(U, dtype=np.float64).copy() for U in init_factors]
    history = []
    core = None
    it = 0
    for it in range(1, max_iters + 1):
        Y = None
        for n in range(N):
            Y = multi_mode_product(T, factors, skip=n, transpose=True)   # Eq. 8
            U, _ = leading_eigvecs(gram(unfold(Y, n)), ranks[n])
            factors[n] = U
        core = mode_product(Y, factors[N - 1].T, N - 1)
        fit = fit_from_norms(norm2_T, float(np.sum(core * core)))
        history.append(fit)
        if it > 1 and abs(history[-1] - history[-2]) < tol:
            break
    factors = [fix_signs(U) for U in factors]
    core = core_of(T, factors)
    fit = fit_from_norms(norm2_T, float(np.sum(core * core)))
    return TuckerResult(core=core, factors=factors, fit=fit, iters=it,
                        fit_history=history)


def relative_error(T: np.ndarray, T_hat: np.ndarray) -> float:
    return float(np.linalg.norm((T - T_hat).ravel()) / np.linalg.norm(T.ravel()))


def psnr(T: np.ndarray, T_hat: np.ndarray) -> float:
    """PSNR of the reconstructed stack in its working colour space, peak =
    max(T) - min(T) of the input (the paper reports PSNR of decoded views,
    Figs. 3 and 4; this is the in-scope part of that measurement)."""
    peak = float(T.max() - T.min())
    mse = float(np.mean((T - T_hat) ** 2))
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(peak * peak / mse)


def element(core: np.ndarray, factors, idx) -> float:
    """One entry of the Tucker model, Eq. 2:
    T_hat(t_1..t_N) = sum_{q_1..q_N} Q(q_1..q_N) prod_r S^(r)(t_r, q_r)."""
    out = np.asarray(core, dtype=np.float64)
    for U, t in zip(factors, idx):
        # contract the leading mode with row t of its factor
        out = np.tensordot(np.asarray(U, dtype=np.float64)[t], out, axes=(0, 0))
    return float(out)
