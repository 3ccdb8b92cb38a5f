"""Squared row norms x <- alpha * diag(A B B^T A^T) + beta * x.
Oracle; test infrastructure.

Sec. 3.3: csrsqn(alpha, A, B, beta, x) / rmsqn.  The plain definition is
q_i = ||e_i^T A B||^2.  Alg. 8 evaluates the same quantity for a CSR A with
Btilde = B B^T: q_i = sum_{k,j in row i} V_k V_j Btilde[J_j, J_k].  Both are
given here in float64; tests check that they agree.
"""
import numpy as np

from .gram import _row_pairs


def rownorms_prod_dense(A, B, alpha=1.0, beta=0.0, x=None):
    """alpha * ||A_i B||^2 + beta * x_i for dense A (n x d), B (d x c)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    q = np.sum((A @ B) ** 2, axis=1)
    out = alpha * q
    if beta != 0.0:
        out = out + beta * np.asarray(x, dtype=np.float64)
    return out


def rownorms_prod_csr_direct(V, J, I, n, d, B, alpha=1.0, beta=0.0, x=None):
    """alpha * ||A_i B||^2 + beta * x_i for CSR A, through the rows of A B."""
    V = np.asarray(V, dtype=np.float64)
    J = np.asarray(J, dtype=np.int64)
    B = np.asarray(B, dtype=np.float64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(I, dtype=np.int64)))
    AB = np.zeros((n, B.shape[1]), dtype=np.float64)
    np.add.at(AB, rows, V[:, None] * B[J])
    out = alpha * np.sum(AB * AB, axis=1)
    if beta != 0.0:
        out = out + beta * np.asarray(x, dtype=np.float64)
    return out


def rownorms_prod_csr_alg8(V, J, I, n, B, alpha=1.0, beta=0.0, x=None):
    """Alg. 8: Btilde = B B^T, then q_i = sum over nonzero pairs of row i."""
    V = np.asarray(V, dtype=np.float64)
    J = np.asarray(J, dtype=np.int64)
    B = np.asarray(B, dtype=np.float64)
    Bt = B @ B.T
    k, j = _row_pairs(I)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(I, dtype=np.int64)) ** 2)
    q = np.zeros(n, dtype=np.float64)
    np.add.at(q, rows, V[k] * V[j] * Bt[J[j], J[k]])
    out = alpha * q
    if beta != 0.0:
        out = out + beta * np.asarray(x, dtype=np.float64)
    return out
