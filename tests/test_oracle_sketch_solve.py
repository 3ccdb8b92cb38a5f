"""Pins of the oracle's sketch-and-solve (Alg. 11) and Gaussian CSR sketch
(Alg. 4, csrjlt) against what the paper and the mathematics fix: exact
recovery on consistent systems, the paper's own SVD formula, the sketch's
residual distortion, Alg. 4's loop order on tiny inputs, and JL moments."""
import numpy as np
import pytest

import workloads
from oracle import gaussian as ga
from oracle import leverage
from oracle import lsq


def _csr_from_dense(A):
    n, d = A.shape
    I = [0]
    J, V = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        J.extend(nz.tolist())
        V.extend(A[i, nz].tolist())
        I.append(len(J))
    return np.array(V), np.array(J, dtype=np.int64), np.array(I, dtype=np.int64)


def _sparse_matrix(n, d, p, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * (rng.random((n, d)) < p)
    A[np.arange(d) % n, np.arange(d)] += 1.0        # full column rank
    return A


@pytest.mark.parametrize("prec", [ga.PREC_FP32, ga.PREC_BF16])
def test_sketch_solve_consistent_system_is_exact(prec):
    """b = A x*: the sketched system is consistent too, so Alg. 11 returns x*."""
    A = workloads.dense_normal(4000, 12, seed=1).astype(np.float64) * np.logspace(-2, 2, 12)
    xs = np.linspace(-3, 3, 12)
    x = lsq.sketch_solve_dense(A, A @ xs, 400, 48, 7, prec)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_sketch_solve_countsketch_only_consistent():
    A = workloads.dense_normal(3000, 10, seed=2).astype(np.float64)
    xs = np.arange(1.0, 11.0)
    x = lsq.sketch_solve_dense(A, A @ xs, 300, 0, 3)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_sketch_solve_matches_the_svd_formula():
    """Alg. 11 step 3: x = V Sigma^+ U^T b~ on the same sketch."""
    A = workloads.dense_normal(5000, 16, seed=3).astype(np.float64) * np.logspace(0, 3, 16)
    b = workloads.dense_normal(5000, 1, seed=4)[:, 0].astype(np.float64)
    Ab = np.hstack([A, b[:, None]])
    SAb = leverage.sketch_dense(Ab, 512, 64, 9)
    U, sig, Vt = np.linalg.svd(SAb[:, :-1], full_matrices=False)
    x_svd = Vt.T @ ((U.T @ SAb[:, -1]) / sig)
    x = lsq.sketch_solve_dense(A, b, 512, 64, 9)
    kappa = sig[0] / sig[-1]
    assert np.linalg.norm(x - x_svd) <= 1e-13 * kappa * np.linalg.norm(x_svd)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_sketch_solve_residual_within_distortion(seed):
    """With an oblivious subspace embedding of (A b), ||A x^ - b|| is within
    (1 + eps) of the least-squares residual; r = 4 (d + 1)^2 buckets and
    k = 8 (d + 1) Gaussian rows keep eps well under 1/2 at these sizes."""
    n, d = 20000, 8
    rng = np.random.default_rng(100 + seed)
    A = rng.standard_normal((n, d)) * np.logspace(-1, 1, d)
    b = A @ rng.standard_normal(d) + 0.5 * rng.standard_normal(n)
    x_ls = lsq.least_squares_qr(A, b)
    x = lsq.sketch_solve_dense(A, b, 4 * (d + 1) ** 2, 8 * (d + 1), seed)
    r_ls = np.linalg.norm(A @ x_ls - b)
    ratio = np.linalg.norm(A @ x - b) / r_ls
    assert 1.0 - 1e-12 <= ratio <= 1.5


def test_sketch_solve_csr_equals_dense():
    A = _sparse_matrix(2000, 9, 0.3, 5)
    b = np.random.default_rng(6).standard_normal(2000)
    V, J, I = _csr_from_dense(A)
    x_csr = lsq.sketch_solve_csr(V, J, I, 2000, 9, b, 300, 40, 11)
    x_dense = lsq.sketch_solve_dense(A, b, 300, 40, 11)
    assert np.linalg.norm(x_csr - x_dense) <= 1e-11 * np.linalg.norm(x_dense)


@pytest.mark.parametrize("prec", [ga.PREC_FP32, ga.PREC_BF16])
def test_csrjlt_follows_alg4_loops(prec):
    """Alg. 4 on a tiny matrix, loop by loop: for each row k of A, a fresh
    Gaussian column g; for each nonzero h of the row and each i, C[i, J_h] +=
    g_i V_h."""
    n, d, m, seed = 37, 5, 9, 4
    A = _sparse_matrix(n, d, 0.4, 7)
    V, J, I = _csr_from_dense(A)
    G = ga.gaussian_columns(m, 0, n, seed, prec, ga.STREAM_JLT)
    C = np.zeros((m, d))
    for k in range(n):
        g = G[:, k]
        for h in range(I[k], I[k + 1]):
            for i in range(m):
                C[i, J[h]] += g[i] * V[h]
    Co = ga.csrjlt(V, J, I, n, d, m, seed, prec, batch=8)
    assert np.max(np.abs(Co - C)) <= 1e-12 * np.max(np.abs(C))
    if prec == ga.PREC_BF16:
        g32 = G.astype(np.float32)
        assert np.array_equal(ga.float32_to_bf16_rne(g32), G)


def test_csrjlt_jl_moments():
    """E ||G a||^2 = ||a||^2 and Var = 2 ||a||^4 / m for G with N(0, 1/m)
    entries: the squared column norms of C over many columns."""
    n, d, m = 300, 400, 32
    A = np.random.default_rng(8).standard_normal((n, d))
    V, J, I = _csr_from_dense(A)
    C = ga.csrjlt(V, J, I, n, d, m, 12)
    ratio = np.sum(C * C, axis=0) / np.sum(A * A, axis=0)
    assert abs(ratio.mean() - 1.0) <= 4.0 * np.sqrt(2.0 / m / d)
    assert abs(ratio.var() / (2.0 / m) - 1.0) <= 0.35


def test_csrjlt_stream_is_its_own():
    """Stream 3 draws differ from the Gaussian stage's (stream 1) and the
    right projection's (stream 2) for the same seed and indices."""
    a = ga.gaussian_columns(8, 0, 16, 5, ga.PREC_FP32, ga.STREAM_JLT)
    b = ga.gaussian_columns(8, 0, 16, 5, ga.PREC_FP32, ga.STREAM_G)
    c = ga.gaussian_columns(8, 0, 16, 5, ga.PREC_FP32, ga.STREAM_PI)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    assert abs(np.corrcoef(a.ravel(), b.ravel())[0, 1]) < 0.35


def test_least_squares_gram_matches_qr_and_recovers_consistent_systems():
    """Alg. 10 against the Householder least-squares solution (a different
    route) on a well-conditioned problem, and exact on b = A x*."""
    rng = np.random.default_rng(20)
    A = rng.standard_normal((3000, 15)) * np.logspace(0, 1, 15)
    b = rng.standard_normal(3000)
    x_qr = lsq.least_squares_qr(A, b)
    assert np.linalg.norm(lsq.least_squares_gram(A, b) - x_qr) <= 1e-11 * np.linalg.norm(x_qr)
    xs = np.linspace(-2, 2, 15)
    assert np.linalg.norm(lsq.least_squares_gram(A, A @ xs) - xs) <= 1e-11 * np.linalg.norm(xs)
