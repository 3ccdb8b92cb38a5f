"""Pins of the oracle's QR, R^-1, leverage scores and least squares (CPU).

QR: Q^T Q = I, Q R = B, R upper with R_jj > 0, agreement with a library QR
up to row signs.  Exact leverage scores: sum = rank, range [0, 1], the
[I; 0] special case, a library SVD, Alg. 13.  Sketched scores: the QR route
equals the SVD route of Alg. 15 (||A_i R^-1|| = ||A_i V Sigma^-1||) and
lies in the (1 +- eps)^-2 band of the exact scores when the sketch is an
eps-embedding (Def. 2).  LSQ: LSQR against a library least-squares solve,
and Alg. 12 reaching eta <= 1e-10.
"""
import numpy as np
import pytest

from oracle import gaussian as ga
from oracle import leverage, lsq, qr, rownorms


def test_householder_qr_properties():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((40, 12)) * 10.0 ** rng.uniform(-3, 3, size=12)
    refl, R, signs = qr.householder_qr(B)
    Q = qr.thin_q(refl, signs, 40)
    assert np.allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    assert np.allclose(Q @ R, B, rtol=0, atol=1e-12 * np.abs(B).max())
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    _, Rnp = np.linalg.qr(B)
    assert np.allclose(np.abs(Rnp), np.abs(R), rtol=1e-10, atol=1e-12 * np.abs(R).max())
    y = rng.standard_normal(40)
    assert np.allclose(qr.apply_qt(refl, signs, y), Q.T @ y, atol=1e-12)


def test_upper_triangular_inverse():
    rng = np.random.default_rng(1)
    R = np.triu(rng.standard_normal((20, 20))) + 5 * np.eye(20)
    X = qr.upper_triangular_inverse(R)
    assert np.allclose(X @ R, np.eye(20), atol=1e-13)
    assert np.array_equal(X, np.triu(X))


def test_rank_deficiency_detected():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((30, 6))
    B[:, 4] = B[:, 1] - 2 * B[:, 2]
    with pytest.raises(qr.RankDeficient):
        qr.check_full_rank(qr.qr_r(B))
    qr.check_full_rank(qr.qr_r(rng.standard_normal((30, 6))))


def test_exact_leverage_invariants_and_library_svd():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((200, 7))
    A[0] *= 100
    ell = leverage.leverage_scores_exact_qr(A)
    assert np.isclose(ell.sum(), 7.0, rtol=1e-12)
    assert np.all(ell >= 0) and np.all(ell <= 1 + 1e-12)
    U = np.linalg.svd(A, full_matrices=False)[0]
    assert np.allclose(ell, np.sum(U**2, axis=1), atol=1e-12)
    assert np.allclose(leverage.leverage_scores_exact_gram(A), ell, atol=1e-10)


def test_exact_leverage_identity_block():
    A = np.vstack([np.eye(5), np.zeros((20, 5))])
    ell = leverage.leverage_scores_exact_qr(A)
    assert np.allclose(ell, np.r_[np.ones(5), np.zeros(20)], atol=1e-14)


@pytest.mark.parametrize("k", [0, 40])
def test_sketched_qr_route_equals_svd_route(k):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3000, 8)) * 10.0 ** rng.uniform(-2, 2, size=8)
    B = leverage.sketch_dense(A, 500, k, 11)
    ell, R = leverage.leverage_scores_dense(A, 500, k, 11)
    _, s, Vt = np.linalg.svd(B, full_matrices=False)
    ell_svd = np.sum((A @ (Vt.T / s)) ** 2, axis=1)
    assert np.allclose(ell, ell_svd, rtol=1e-9)
    assert np.allclose(R.T @ R, B.T @ B, rtol=1e-10, atol=1e-10 * np.abs(B.T @ B).max())


def test_sketched_scores_within_embedding_band():
    rng = np.random.default_rng(5)
    n, d, r, k = 20000, 10, 2000, 60
    A = rng.standard_normal((n, d))
    A[:5] *= 100.0
    ell, _ = leverage.leverage_scores_dense(A, r, k, 3)
    exact = leverage.leverage_scores_exact_gram(A)
    # eps of this sketch as a subspace embedding of range(A)
    Q = np.linalg.qr(A)[0]
    sv = np.linalg.svd(leverage.sketch_dense(Q, r, k, 3), compute_uv=False)
    lo, hi = 1.0 / sv.max() ** 2, 1.0 / sv.min() ** 2
    ratio = ell / exact
    assert np.all(ratio >= lo * (1 - 1e-9)) and np.all(ratio <= hi * (1 + 1e-9))
    # the scaled rows are the top-5 scores (config-1 style outliers)
    assert set(np.argsort(-ell)[:5]) == set(range(5))


def test_bf16_mode_changes_scores_little():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((4000, 6))
    e32, _ = leverage.leverage_scores_dense(A, 400, 30, 8, ga.PREC_FP32)
    e16, _ = leverage.leverage_scores_dense(A, 400, 30, 8, ga.PREC_BF16)
    assert np.max(np.abs(e16 / e32 - 1)) < 0.05


def test_lsqr_matches_library_lstsq():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((300, 12))
    b = rng.standard_normal(300)
    y, it = lsq.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 12)
    assert np.allclose(y, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-9, atol=1e-10)
    assert it <= 40


def test_sketch_precondition_lsq_reaches_tolerance():
    rng = np.random.default_rng(8)
    n, d = 5000, 16
    A = rng.standard_normal((n, d)) * 10.0 ** rng.uniform(-3, 3, size=d)
    xs = rng.standard_normal(d)
    b = A @ xs + 1e-6 * rng.standard_normal(n)
    x, info = lsq.lsq_dense(A, b, r=d * d, k=2 * d, seed=1)
    assert info["eta"] <= 1e-10
    x_ls = lsq.least_squares_qr(A, b)
    x_np = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.allclose(x_ls, x_np, rtol=1e-8)
    assert np.linalg.norm(x - x_ls) <= 1e-8 * np.linalg.norm(x_ls)
    eta_ls = lsq.normal_equation_residual(lambda v: A @ v, lambda u: A.T @ u, b, x_ls)
    assert eta_ls < 1e-10


def test_jl_scores_unbiased_and_concentrated():
    """Alg. 15 with Pi: with R fixed, the mean of ||A_i R^-1 Pi||^2 over
    independent Pi is ||A_i R^-1||^2; with large m the scores of
    leverage_scores_jl_dense approach those without Pi (same sketch seed)."""
    A = np.random.default_rng(8).standard_normal((3000, 12)).astype(np.float64)
    A[:4] *= 30.0
    ell, R = leverage.leverage_scores_dense(A, 600, 48, 5)
    Rinv = qr.upper_triangular_inverse(R)
    acc = np.zeros(A.shape[0])
    trials = 400
    for s in range(trials):
        acc += rownorms.rownorms_prod_dense(A, Rinv @ ga.jl_matrix(12, 4, 1000 + s))
    mean = acc / trials
    # ||x Pi||^2 / ||x||^2 ~ chi^2_4 / 4 per trial: relative sd sqrt(2/4) / sqrt(trials)
    assert np.all(np.abs(mean / ell - 1.0) < 5 * np.sqrt(0.5 / trials))
    big, R2 = leverage.leverage_scores_jl_dense(A, 600, 48, 2000, 5)
    assert np.array_equal(R2, R)                                  # same sketch, same R
    assert np.all(np.abs(big / ell - 1.0) < 6 * np.sqrt(2.0 / 2000))
    V, J, I = _csr_bernoulli(4000, 10, 0.3, 6)
    ell_c, _ = leverage.leverage_scores_csr(V, J, I, 4000, 10, 400, 40, 2)
    big_c, _ = leverage.leverage_scores_jl_csr(V, J, I, 4000, 10, 400, 40, 2000, 2)
    nz = ell_c > 0
    assert np.all(big_c[~nz] == 0)
    assert np.all(np.abs(big_c[nz] / ell_c[nz] - 1.0) < 6 * np.sqrt(2.0 / 2000))


def _csr_bernoulli(n, d, p, seed):
    """CSR (V, J, I) with each entry kept with probability p (test input)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, d)) < p
    I = np.concatenate([[0], np.cumsum(mask.sum(axis=1))]).astype(np.int64)
    J = np.nonzero(mask)[1].astype(np.int32)
    V = rng.standard_normal(J.size).astype(np.float32)
    return V, J, I
