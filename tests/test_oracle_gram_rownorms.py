"""Pins of the oracle's Gram (Alg. 5 / 7) and row norms (Alg. 8) (CPU only):
brute force per-row outer products, the dense definition, symmetry, the
alpha/beta update, (SA)^T(SA) = A^T A for an injective hash, and the trace
identity sum_i ||A_i B||^2 = trace(B^T (A^T A) B) tying the two together."""
import numpy as np
import pytest

from oracle import countsketch as cs
from oracle import gram, rownorms


def _random_csr(n, d, p, seed, integer=False):
    rng = np.random.default_rng(seed)
    mask = rng.random((n, d)) < p
    mask[3] = False                       # an empty row
    mask[5] = True                        # a full row
    A = np.zeros((n, d))
    vals = rng.integers(-6, 7, size=mask.sum()) if integer else rng.standard_normal(mask.sum())
    A[mask] = vals
    rows, cols = np.nonzero(A)
    I = np.concatenate([[0], np.cumsum(np.sum(A != 0, axis=1))]).astype(np.int64)
    return A, A[rows, cols], cols.astype(np.int32), I


def test_gram_csr_alg5_equals_brute_force_outer_products():
    A, V, J, I = _random_csr(60, 9, 0.3, 1)
    brute = np.zeros((9, 9))
    for i in range(A.shape[0]):                # sum_i a_i a_i^T, one row at a time
        for a in range(9):
            for b in range(9):
                brute[a, b] += A[i, a] * A[i, b]
    assert np.allclose(gram.gram_csr(V, J, I, 9), brute, rtol=1e-14, atol=1e-12)
    assert np.allclose(gram.gram_dense(A), brute, rtol=1e-14, atol=1e-12)


def test_gram_alpha_beta_and_symmetry():
    A, V, J, I = _random_csr(200, 12, 0.2, 2)
    C0 = np.random.default_rng(3).standard_normal((12, 12))
    got = gram.gram_csr(V, J, I, 12, alpha=-0.5, beta=2.0, C=C0)
    assert np.allclose(got, -0.5 * A.T @ A + 2.0 * C0, rtol=1e-13, atol=1e-12)
    G = gram.gram_csr(V, J, I, 12)
    assert np.array_equal(G, G.T)


def test_sketch_gram_equals_gram_for_injective_hash():
    n, d, r = 40, 5, 100000
    A, _, _, _ = _random_csr(n, d, 0.7, 4, integer=True)
    bucket, sign = cs.countsketch_hash(n, r, 17)
    assert len(np.unique(bucket)) == n         # injective on these rows
    SA = cs.countsketch_apply_dense(A, bucket, sign, r)
    assert np.array_equal(gram.gram_dense(SA), gram.gram_dense(A))


@pytest.mark.parametrize("c", [1, 4, 9])
def test_rownorms_dense_csr_alg8_agree(c):
    A, V, J, I = _random_csr(80, 9, 0.35, 5)
    B = np.random.default_rng(6).standard_normal((9, c))
    ref = np.array([np.sum((A[i] @ B) ** 2) for i in range(80)])
    d1 = rownorms.rownorms_prod_dense(A, B)
    d2 = rownorms.rownorms_prod_csr_direct(V, J, I, 80, 9, B)
    d3 = rownorms.rownorms_prod_csr_alg8(V, J, I, 80, B)
    for got in (d1, d2, d3):
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    assert d3[3] == 0.0                        # empty row


def test_rownorms_alpha_beta():
    A, V, J, I = _random_csr(30, 6, 0.5, 7)
    B = np.random.default_rng(8).standard_normal((6, 6))
    x0 = np.arange(30, dtype=np.float64)
    got = rownorms.rownorms_prod_csr_alg8(V, J, I, 30, B, alpha=3.0, beta=-1.0, x=x0)
    assert np.allclose(got, 3.0 * np.sum((A @ B) ** 2, axis=1) - x0, rtol=1e-12, atol=1e-11)


def test_trace_identity_ties_gram_and_rownorms():
    A, V, J, I = _random_csr(300, 10, 0.3, 9)
    B = np.random.default_rng(10).standard_normal((10, 7))
    q = rownorms.rownorms_prod_csr_alg8(V, J, I, 300, B)
    C = gram.gram_csr(V, J, I, 10)
    assert np.isclose(q.sum(), np.trace(B.T @ C @ B), rtol=1e-12)
