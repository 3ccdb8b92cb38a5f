"""Pins of the oracle's column subset selection (Alg. 9) and the leverage
scores built on it (Alg. 14, 16): the pivoted QR's defining properties, cases
whose selection is fixed by construction, and reductions to closed forms."""
import numpy as np

from oracle import css
from oracle import gaussian as ga
from oracle import leverage


def test_pivoted_qr_orthogonal_columns_sorted_by_norm():
    """Orthogonal columns: the remaining norms never change, so the pivots are
    the columns in decreasing norm and |R_jj| are those norms."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 7)))
    scales = np.array([3.0, 0.5, 7.0, 1.0, 2.0, 0.1, 5.0])
    perm, rdiag = css.pivoted_qr(Q * scales)
    assert list(perm) == list(np.argsort(-scales))
    assert np.allclose(rdiag, np.sort(scales)[::-1], rtol=1e-12)


def test_pivoted_qr_properties_on_a_random_matrix():
    """|R_jj| is non-increasing, and each pivot has the largest remaining norm:
    |R_jj| equals the distance of column perm[j] from the span of the earlier
    pivots, and no other remaining column is farther."""
    B = np.random.default_rng(1).standard_normal((30, 12)) * np.logspace(0, 2, 12)
    perm, rdiag = css.pivoted_qr(B)
    assert np.all(np.diff(rdiag) <= 1e-12 * rdiag[0])
    for j in range(12):
        Qj = np.linalg.qr(B[:, perm[:j]])[0] if j else np.zeros((30, 0))
        dist = [np.linalg.norm(B[:, c] - Qj @ (Qj.T @ B[:, c])) for c in perm[j:]]
        assert abs(dist[0] - rdiag[j]) <= 1e-10 * rdiag[0]
        assert dist[0] >= max(dist) * (1 - 1e-12)


def test_pivoted_qr_rank_revealing_on_planted_rank():
    """Columns 0..3 independent, the rest in their span: the first four pivots
    are independent columns and |R_44| vanishes."""
    rng = np.random.default_rng(2)
    basis = rng.standard_normal((50, 4))
    B = np.hstack([basis, basis @ rng.standard_normal((4, 6)) * 0.1])
    perm, rdiag = css.pivoted_qr(B)
    assert np.linalg.matrix_rank(B[:, perm[:4]]) == 4
    assert rdiag[4] <= 1e-12 * rdiag[0]


def test_column_select_picks_dominant_columns_through_the_sketch():
    """A with a few columns of much larger norm, mutually independent: any
    subspace embedding keeps them on top, so Alg. 9 selects exactly them."""
    rng = np.random.default_rng(3)
    n, d = 5000, 16
    A = rng.standard_normal((n, d))
    big = [11, 2, 7]
    A[:, big] *= np.array([1000.0, 300.0, 100.0])
    K = css.column_select_dense(A, 512, 64, 5, ga.PREC_FP32, 3)
    assert list(K) == big


def test_hrn_exact_with_all_columns_is_alg13():
    """k = d: A[:, K] spans the column space of A, so Alg. 14 returns the exact
    leverage scores ||Q_i||^2 (the definition)."""
    A = np.random.default_rng(4).standard_normal((3000, 10)) * np.logspace(-1, 1, 10)
    theta, K = css.hrn_exact_dense(A, 256, 40, 2, ga.PREC_FP32, 10)
    assert sorted(K) == list(range(10))
    exact = leverage.leverage_scores_exact_qr(A)
    assert np.max(np.abs(theta - exact) / exact) <= 1e-10


def test_hrn_approx_with_all_columns_matches_alg15():
    """k = d: Alg. 16 is Alg. 15 (without Pi) up to the column order, which
    leaves ||A_i R^-1||^2 unchanged."""
    A = np.random.default_rng(5).standard_normal((4000, 8)) * np.logspace(0, 2, 8)
    theta, K = css.hrn_approx_dense(A, 400, 32, 9, ga.PREC_FP32, 8)
    ref, _ = leverage.leverage_scores_dense(A, 400, 32, 9, ga.PREC_FP32)
    assert np.max(np.abs(theta - ref) / ref) <= 1e-10


def test_hrn_scores_of_a_subset_sum_to_k():
    """Leverage scores of an n x k full-rank matrix sum to k (trace of the
    projector); the sketched ones to within the sketch's distortion."""
    A = np.random.default_rng(6).standard_normal((6000, 12))
    theta, K = css.hrn_exact_dense(A, 400, 48, 1, ga.PREC_FP32, 5)
    assert len(K) == 5 and abs(theta.sum() - 5.0) <= 1e-9
    theta2, K2 = css.hrn_approx_dense(A, 400, 48, 1, ga.PREC_FP32, 5)
    assert list(K2) == list(K) and 0.5 * 5 <= theta2.sum() <= 2.0 * 5


def test_truncated_scores_on_planted_rank():
    """A of rank 5 (d = 12): the truncation finds rank 5; the scores are those
    of Alg. 15 on A[:, K] (the sketch of A restricted to K is the sketch of
    A[:, K]); and they approximate the exact leverage scores of A, ||U_i||^2
    over its 5 left singular vectors, within the sketch's distortion."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((4000, 5)) @ rng.standard_normal((5, 12))
    A[:3] *= 20.0
    theta, rank, K = css.leverage_scores_truncated_dense(A, 20000, 600, 3, ga.PREC_FP32, 1e-8)
    assert rank == 5
    alg15, _ = leverage.leverage_scores_dense(A[:, K], 20000, 600, 3, ga.PREC_FP32)
    assert np.max(np.abs(theta - alg15) / alg15) <= 1e-9
    U = np.linalg.svd(A, full_matrices=False)[0][:, :5]
    exact = np.sum(U * U, axis=1)
    assert np.all((theta / exact > 0.6) & (theta / exact < 1.6))


def test_truncated_scores_full_rank_is_alg15():
    A = np.random.default_rng(8).standard_normal((3000, 9)) * np.logspace(0, 2, 9)
    theta, rank, K = css.leverage_scores_truncated_dense(A, 300, 36, 4, ga.PREC_FP32, 1e-10)
    ref, _ = leverage.leverage_scores_dense(A, 300, 36, 4, ga.PREC_FP32)
    assert rank == 9 and np.max(np.abs(theta - ref) / ref) <= 1e-10
