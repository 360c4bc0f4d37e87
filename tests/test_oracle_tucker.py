"""Pins of the oracle's Tucker-ALS / HOOI (Section III-B) against facts fixed
by the mathematics rather than by the oracle: brute-force mode products,
Eckart-Young for order 2 (checked with numpy's SVD), exactness at full
multilinear rank, the HOSVD all-orthogonality property, recovery of planted
low-rank tensors, orthonormal factors, the energy identity, monotone fit,
a least-squares core for fixed factors, local optimality and a 2x2 angle
enumeration."""
import itertools

import numpy as np
import pytest

from oracle import tucker


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _orthonormal(n, r, rng):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def test_mode_product_brute_force():
    T = _rand((3, 4, 2, 5), 1)
    for n, rows in itertools.product(range(4), ("wide", "square")):
        m = 6 if rows == "wide" else T.shape[n]
        A = _rand((m, T.shape[n]), 10 + n)
        got = tucker.mode_product(T, A, n)
        shape = list(T.shape)
        shape[n] = m
        want = np.zeros(shape)
        for idx in itertools.product(*[range(s) for s in shape]):
            acc = 0.0
            for i in range(T.shape[n]):
                src = list(idx)
                src[n] = i
                acc += T[tuple(src)] * A[idx[n], i]
            want[idx] = acc
        np.testing.assert_allclose(got, want, atol=1e-12)


def test_unfold_columns_are_fibres():
    T = _rand((3, 4, 2), 2)
    for n in range(3):
        Tn = tucker.unfold(T, n)
        assert Tn.shape[0] == T.shape[n]
        # the Gram of the unfolding is sum over all fibres, independent of order
        want = np.zeros((T.shape[n], T.shape[n]))
        for idx in itertools.product(*[range(s) for m, s in enumerate(T.shape) if m != n]):
            sl = list(idx)
            sl.insert(n, slice(None))
            f = T[tuple(sl)]
            want += np.outer(f, f)
        np.testing.assert_allclose(Tn @ Tn.T, want, atol=1e-12)


@pytest.mark.parametrize("shape,r", [((30, 20), 5), ((12, 40), 3), ((25, 25), 1)])
def test_eckart_young_order2(shape, r):
    X = _rand(shape, 3)
    res = tucker.hooi(X, (r, r), max_iters=5, tol=1e-14)
    s = np.linalg.svd(X, compute_uv=False)
    fit_ey = 1.0 - np.sqrt(np.sum(s[r:] ** 2)) / np.linalg.norm(X)
    assert abs(res.fit - fit_ey) < 1e-12
    U, _, Vt = np.linalg.svd(X)
    np.testing.assert_allclose(res.factors[0] @ res.factors[0].T, U[:, :r] @ U[:, :r].T, atol=1e-10)
    np.testing.assert_allclose(res.factors[1] @ res.factors[1].T, Vt[:r].T @ Vt[:r], atol=1e-10)
    # HOOI on a matrix is already optimal after the first sweep
    assert abs(res.fit_history[0] - fit_ey) < 1e-12


def test_full_multilinear_rank_is_exact():
    X = _rand((6, 5, 3, 4), 4)
    res = tucker.hooi(X, X.shape, max_iters=3, tol=0.0)
    Xh = tucker.reconstruct(res.core, res.factors)
    assert tucker.relative_error(X, Xh) < 1e-13
    assert abs(res.fit - 1.0) < 1e-7


def test_hosvd_all_orthogonality():
    # De Lathauwer's HOSVD property behind Eq. 3 to Eq. 5: with the full
    # factors, slices of the core along any mode are mutually orthogonal and
    # their norms are the singular values of that unfolding.
    X = _rand((5, 4, 3, 3), 5)
    U = tucker.thosvd(X, X.shape)
    Q = tucker.core_of(X, U)
    for n in range(4):
        Qn = tucker.unfold(Q, n)
        G = Qn @ Qn.T
        s = np.linalg.svd(tucker.unfold(X, n), compute_uv=False)
        np.testing.assert_allclose(np.sqrt(np.diag(G)), s, rtol=1e-10)
        off = G - np.diag(np.diag(G))
        assert np.abs(off).max() < 1e-10 * s[0] ** 2


def test_planted_low_rank_recovered():
    rng = np.random.default_rng(6)
    shape, ranks = (20, 15, 3, 6), (4, 3, 2, 3)
    G = rng.standard_normal(ranks)
    Qs = [_orthonormal(s, r, rng) for s, r in zip(shape, ranks)]
    X = tucker.reconstruct(G, Qs)
    res = tucker.hooi(X, ranks, max_iters=5, tol=0.0)
    assert res.fit > 1.0 - 1e-7
    assert tucker.relative_error(X, tucker.reconstruct(res.core, res.factors)) < 1e-12
    for U, Q in zip(res.factors, Qs):
        np.testing.assert_allclose(U @ U.T, Q @ Q.T, atol=1e-10)


def _noisy_low_rank(seed, shape=(16, 12, 3, 5), ranks=(5, 4, 2, 3), noise=0.05):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(ranks) * 3
    Qs = [_orthonormal(s, r, rng) for s, r in zip(shape, ranks)]
    return tucker.reconstruct(G, Qs) + noise * rng.standard_normal(shape)


def test_orthonormal_factors_and_energy_identity():
    X = _noisy_low_rank(7)
    ranks = (4, 3, 2, 2)
    res = tucker.hooi(X, ranks, max_iters=20, tol=0.0)
    for U, r in zip(res.factors, ranks):
        assert U.shape[1] == r
        assert np.abs(U.T @ U - np.eye(r)).max() < 1e-13
    Xh = tucker.reconstruct(res.core, res.factors)
    lhs = np.sum(X * X) - np.sum(res.core ** 2)
    rhs = np.sum((X - Xh) ** 2)
    assert abs(lhs - rhs) <= 1e-10 * rhs
    assert abs(res.fit - (1 - np.sqrt(rhs) / np.linalg.norm(X))) < 1e-12


def test_fit_non_decreasing_across_sweeps():
    X = _noisy_low_rank(8, noise=0.3)
    res = tucker.hooi(X, (3, 3, 2, 2), max_iters=15, tol=0.0)
    h = np.array(res.fit_history)
    assert np.all(np.diff(h) >= -1e-12)


def test_core_is_least_squares_solution():
    X = _rand((4, 3, 2, 2), 9)
    ranks = (2, 2, 1, 2)
    res = tucker.hooi(X, ranks, max_iters=10, tol=0.0)
    # vec(X) ~ (U4 kron U3 kron U2 kron U1) vec(G) with column-major vec
    K = np.ones((1, 1))
    for U in res.factors:
        K = np.kron(U, K)
    g, *_ = np.linalg.lstsq(K, X.ravel(order="F"), rcond=None)
    np.testing.assert_allclose(res.core.ravel(order="F"), g, atol=1e-12)


def test_local_optimality_under_grassmann_perturbation():
    X = _noisy_low_rank(10, noise=0.2)
    ranks = (4, 3, 2, 2)
    res = tucker.hooi(X, ranks, max_iters=200, tol=1e-15)
    best = np.sum(res.core ** 2)
    rng = np.random.default_rng(12)
    for _ in range(200):
        n = rng.integers(4)
        Us = [U.copy() for U in res.factors]
        D = 1e-3 * rng.standard_normal(Us[n].shape)
        Us[n], _ = np.linalg.qr(Us[n] + D)
        val = np.sum(tucker.core_of(X, Us) ** 2)
        assert val <= best * (1 + 1e-12)


def test_two_by_two_angle_enumeration():
    X = np.array([[3.0, 1.0], [1.0, 2.0]]) @ np.array([[1.0, 0.5], [-0.2, 1.0]])
    res = tucker.hooi(X, (1, 1), max_iters=5, tol=0.0)
    th = np.linspace(0, np.pi, 200001)
    u = np.stack([np.cos(th), np.sin(th)])
    vals = np.sum((X.T @ u) ** 2, axis=0)
    ub = u[:, np.argmax(vals)]
    assert abs(abs(ub @ res.factors[0][:, 0]) - 1.0) < 1e-9
    assert abs(res.core[0, 0] ** 2 - vals.max()) < 1e-8 * vals.max()


def test_sign_convention():
    X = _noisy_low_rank(13)
    res = tucker.hooi(X, (3, 3, 2, 2), max_iters=5, tol=0.0)
    for U in res.factors:
        idx = np.argmax(np.abs(U), axis=0)
        assert np.all(U[idx, np.arange(U.shape[1])] > 0)
    # the core stays consistent with the signed factors
    np.testing.assert_allclose(res.core, tucker.core_of(X, res.factors), atol=1e-12)


def test_stopping_rule_runs_at_least_two_sweeps():
    X = _noisy_low_rank(14)
    res = tucker.hooi(X, (3, 3, 2, 2), max_iters=10, tol=1.0)
    assert res.iters == 2
    res = tucker.hooi(X, (3, 3, 2, 2), max_iters=1, tol=1.0)
    assert res.iters == 1


def test_psnr_definition():
    X = np.linspace(0, 1, 100).reshape(10, 10)
    Xh = X + 0.01
    # peak = max - min = 1, mse = 1e-4  ->  40 dB
    assert abs(tucker.psnr(X, Xh) - 40.0) < 1e-9


def test_element_wise_model_matches_reconstruction():
    rng = np.random.default_rng(15)
    core = rng.standard_normal((3, 2, 2, 3))
    Us = [rng.standard_normal((s, r)) for s, r in zip((5, 4, 3, 4), core.shape)]
    full = tucker.reconstruct(core, Us)
    for idx in [(0, 0, 0, 0), (4, 3, 2, 3), (2, 1, 0, 2)]:
        # brute-force sum of Eq. 2
        want = 0.0
        for q in itertools.product(*[range(r) for r in core.shape]):
            term = core[q]
            for U, t, qq in zip(Us, idx, q):
                term *= U[t, qq]
            want += term
        assert abs(tucker.element(core, Us, idx) - want) < 1e-12
        assert abs(full[idx] - want) < 1e-12


def test_st_hosvd_error_is_the_sum_of_dropped_eigenvalues():
    # The truncations of ST-HOSVD are orthogonal projections applied one
    # after another, so ||T - T_hat||^2 splits exactly into the energy each
    # step drops: the sum over modes of the discarded eigenvalues of the Gram
    # of the tensor truncated so far (an identity, not a bound).
    rng = np.random.default_rng(31)
    T = rng.standard_normal((9, 7, 5, 4))
    ranks = (4, 3, 2, 3)
    Us, dropped = tucker.st_hosvd(T, ranks)
    Xh = tucker.reconstruct(tucker.core_of(T, Us), Us)
    err2 = np.sum((T - Xh) ** 2)
    assert abs(err2 - sum(dropped)) < 1e-10 * np.sum(T ** 2)
    for U in Us:
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-13


def test_st_hosvd_order2_is_truncated_svd():
    # For a matrix, truncating the rows first leaves U1^T T, whose leading
    # right singular vectors are those of T: the result is the Eckart-Young
    # truncated SVD (same fit as numpy's SVD)
    rng = np.random.default_rng(32)
    T = rng.standard_normal((12, 9))
    Us, _ = tucker.st_hosvd(T, (4, 4))
    Xh = tucker.reconstruct(tucker.core_of(T, Us), Us)
    sv = np.linalg.svd(T, compute_uv=False)
    assert abs(np.sum((T - Xh) ** 2) - np.sum(sv[4:] ** 2)) < 1e-10 * np.sum(T ** 2)


def test_st_hosvd_full_rank_is_exact_and_hooi_reaches_the_same_fit():
    rng = np.random.default_rng(33)
    T = rng.standard_normal((6, 5, 3, 2))
    Us, dropped = tucker.st_hosvd(T, T.shape)
    assert max(dropped) < 1e-10
    assert tucker.relative_error(T, tucker.reconstruct(tucker.core_of(T, Us), Us)) < 1e-13
    # started from either initialisation, HOOI converges to the same fit here
    T2 = rng.standard_normal((10, 8, 3, 2))
    ranks = (4, 3, 3, 2)
    a = tucker.hooi(T2, ranks, 200, 1e-14)
    b = tucker.hooi(T2, ranks, 200, 1e-14, init_factors=tucker.st_hosvd(T2, ranks)[0])
    assert abs(a.fit - b.fit) < 1e-9
