"""Leverage scores: sketched (Alg. 15, without and with its Pi) and exact
(oracle; test infrastructure).

Alg. 15 (Sec. 4.3): sketch A (here G*S*A, Alg. 3; k = 0 means S*A alone,
as the m = 0 convention of csrcgs, Sec. 5), factor the sketch, and return
the squared row norms of A times the factor's inverse (Alg. 8):
``leverage_scores_*`` return ||A_i R^-1||^2; ``leverage_scores_jl_*`` apply
Alg. 15's right Gaussian Pi (d x m, scaled by 1/sqrt(m)) and return
||A_i R^-1 Pi||^2.

Exact scores (Alg. 13, and the definition ||Q_i||^2 for A = Q R) pin the
sketched ones.
"""
import numpy as np

from . import countsketch, gaussian, qr, rownorms


def sketch_dense(A, r, k, seed, prec=gaussian.PREC_FP32):
    """G*S*A (k > 0) or S*A (k == 0) for dense A, float64."""
    SA = countsketch.cs_sketch_dense(A, r, seed)
    if k == 0:
        return SA
    return gaussian.gauss_sketch(SA, k, seed, prec)


def sketch_csr(V, J, I, n, d, r, k, seed, prec=gaussian.PREC_FP32):
    SA = countsketch.cs_sketch_csr(V, J, I, n, d, r, seed)
    if k == 0:
        return SA
    return gaussian.gauss_sketch(SA, k, seed, prec)


def sketch_R(B):
    """Sign-normalised R of the sketch, after the full-rank check."""
    R = qr.qr_r(B)
    qr.check_full_rank(R)
    return R


def leverage_scores_dense(A, r, k, seed, prec=gaussian.PREC_FP32):
    """(ell, R): ell_i = ||A_i R^-1||^2 with R from the sketch of A."""
    R = sketch_R(sketch_dense(A, r, k, seed, prec))
    Rinv = qr.upper_triangular_inverse(R)
    return rownorms.rownorms_prod_dense(A, Rinv), R


def leverage_scores_csr(V, J, I, n, d, r, k, seed, prec=gaussian.PREC_FP32):
    R = sketch_R(sketch_csr(V, J, I, n, d, r, k, seed, prec))
    Rinv = qr.upper_triangular_inverse(R)
    return rownorms.rownorms_prod_csr_alg8(V, J, I, n, Rinv), R


def leverage_scores_jl_dense(A, r, k, m, seed, prec=gaussian.PREC_FP32):
    """Alg. 15 with the right JL projection: ell_i ~ ||A_i R^-1 Pi||^2, R from
    the sketch of A (QR in place of the SVD), Pi = jl_matrix(d, m, seed)."""
    A = np.asarray(A, dtype=np.float64)
    R = sketch_R(sketch_dense(A, r, k, seed, prec))
    X = qr.upper_triangular_inverse(R) @ gaussian.jl_matrix(A.shape[1], m, seed)
    return rownorms.rownorms_prod_dense(A, X), R


def leverage_scores_jl_csr(V, J, I, n, d, r, k, m, seed, prec=gaussian.PREC_FP32):
    R = sketch_R(sketch_csr(V, J, I, n, d, r, k, seed, prec))
    X = qr.upper_triangular_inverse(R) @ gaussian.jl_matrix(d, m, seed)
    return rownorms.rownorms_prod_csr_alg8(V, J, I, n, X), R


def leverage_scores_exact_qr(A):
    """ell_i = ||Q_i||^2 for the thin Householder Q of A (full column rank)."""
    A = np.asarray(A, dtype=np.float64)
    refl, R, signs = qr.householder_qr(A)
    Q = qr.thin_q(refl, signs, A.shape[0])
    return np.sum(Q * Q, axis=1)


def leverage_scores_exact_gram(A, rcond=1e-12):
    """Alg. 13: B = A^T A, B = V Sigma^2 V^T, theta_i = ||A_i V Sigma^-1||^2.

    Singular values below rcond * max are truncated (Alg. 13's "truncate if
    needed"); the eigen-decomposition of the symmetric B is the library step.
    """
    A = np.asarray(A, dtype=np.float64)
    B = A.T @ A
    w, V = np.linalg.eigh(B)
    keep = w > rcond * w.max()
    X = V[:, keep] / np.sqrt(w[keep])[None, :]
    return np.sum((A @ X) ** 2, axis=1)
