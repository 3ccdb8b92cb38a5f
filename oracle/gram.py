"""Gram matrix C <- alpha * A^T A + beta * C (oracle; test infrastructure).

Sec. 3: csrrk(alpha, A, beta, C).  Alg. 5 accumulates, for every row i of
A, the outer product of the row with itself: for every pair (k, j) of
nonzeros of row i, B[J_k, J_j] += V_k * V_j.  Alg. 6 / Alg. 7 add the
alpha, beta update.  The oracle evaluates Alg. 5 directly over all pairs
in float64 (dense A: every entry is a "nonzero", which is A^T A).
"""
import numpy as np


def _row_pairs(I):
    """All (k, j) nonzero-position pairs inside each CSR row (Alg. 5 loops)."""
    I = np.asarray(I, dtype=np.int64)
    cnt = np.diff(I)
    n = len(cnt)
    # pairs per row = cnt^2; enumerate (k, j) = (start + a, start + b)
    npairs = cnt * cnt
    row = np.repeat(np.arange(n, dtype=np.int64), npairs)
    off = np.arange(int(npairs.sum()), dtype=np.int64) - np.repeat(np.cumsum(npairs) - npairs, npairs)
    c = cnt[row]
    a = off // np.maximum(c, 1)
    b = off - a * c
    start = I[:-1][row]
    return start + a, start + b


def gram_csr(V, J, I, d, alpha=1.0, beta=0.0, C=None):
    """alpha * A^T A + beta * C for CSR A = (V, J, I), 0-based (Alg. 5 / 7)."""
    V = np.asarray(V, dtype=np.float64)
    J = np.asarray(J, dtype=np.int64)
    B = np.zeros((d, d), dtype=np.float64)
    k, j = _row_pairs(I)
    np.add.at(B, (J[k], J[j]), V[k] * V[j])
    out = alpha * B
    if beta != 0.0:
        out = out + beta * np.asarray(C, dtype=np.float64)
    return out


def gram_dense(A, alpha=1.0, beta=0.0, C=None):
    """alpha * sum_i a_i a_i^T + beta * C for dense A (the rows' outer products)."""
    A = np.asarray(A, dtype=np.float64)
    out = alpha * (A.T @ A)
    if beta != 0.0:
        out = out + beta * np.asarray(C, dtype=np.float64)
    return out
