"""Column subset selection (Alg. 9) and the leverage scores built on it
(Alg. 14, Alg. 16) -- oracle; test infrastructure.

Alg. 9 (Sec. 4.1): B = G S A (CountGauss, m ~ 2d Gaussian rows, r ~ d^2
buckets), a pivoted QR of B gives a permutation P, and the first k columns
of P pick the "top-k" columns of A.  The pivoted QR here is Householder QR
with column pivoting (Businger & Golub, Numer. Math. 7 (1965)): at step j
the remaining column of largest norm (rows j..m-1 of the partly reduced B)
is swapped to position j, ties going to the lowest column index; then the
reflector is applied.  Everything is float64.

Alg. 14 (ls_hrn_exact): the exact leverage scores (Alg. 13) of A[:, K].

"Truncate if needed" (Alg. 15 step 3, Alg. 13 step 2), read as a
rank-revealing truncation: the numerical rank of the sketch is the number
of column-pivoted QR steps with |R_jj| > rcond |R_00|, and the scores are
those of A restricted to the columns those steps pick (they span the
dominant column space): ``leverage_scores_truncated_dense``.
Alg. 16 (ls_hrn_approx): Alg. 15 on A[:, K].  Reading: the sketch of A[:, K]
is the sketch of A restricted to the columns K (column selection commutes
with the left sketch G S), so the B of Alg. 9 is reused; R from the QR of
B[:, K], and the scores ||A[i, K] R^-1||^2 (no right projection).
"""
import numpy as np

from . import leverage, qr, rownorms


def pivoted_qr(B, kmax=None):
    """(perm, rdiag): column order of Householder QR with column pivoting of
    B (m x d) for the first kmax steps (all if None), and |R_jj| of those."""
    W = np.array(B, dtype=np.float64, copy=True)
    m, d = W.shape
    steps = min(m, d) if kmax is None else min(kmax, m, d)
    perm = np.arange(d)
    rdiag = np.zeros(steps)
    for j in range(steps):
        norms = np.sum(W[j:, j:] ** 2, axis=0)
        p = j + int(np.argmax(norms))            # first maximum: lowest index
        if p != j:
            W[:, [j, p]] = W[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        x = W[j:, j]
        nrm = np.linalg.norm(x)
        rdiag[j] = nrm
        if nrm == 0.0:
            continue
        v = x.copy()
        v[0] += np.copysign(nrm, x[0])
        beta = 2.0 / float(v @ v)
        W[j:, j:] -= beta * np.outer(v, v @ W[j:, j:])
    return perm, rdiag


def column_select_dense(A, r, k, seed, prec, c):
    """Alg. 9: the first c pivots of the pivoted QR of the sketch of A."""
    perm, _ = pivoted_qr(leverage.sketch_dense(A, r, k, seed, prec), c)
    return perm[:c].copy()


def column_select_csr(V, J, I, n, d, r, k, seed, prec, c):
    perm, _ = pivoted_qr(leverage.sketch_csr(V, J, I, n, d, r, k, seed, prec), c)
    return perm[:c].copy()


def hrn_exact_dense(A, r, k, seed, prec, c):
    """Alg. 14: (theta, K) -- exact leverage scores (Alg. 13) of A[:, K]."""
    A = np.asarray(A, dtype=np.float64)
    K = column_select_dense(A, r, k, seed, prec, c)
    return leverage.leverage_scores_exact_gram(A[:, K]), K


def hrn_approx_dense(A, r, k, seed, prec, c):
    """Alg. 16: (theta, K) -- ||A[i, K] R^-1||^2 with R from the QR of the
    Alg. 9 sketch restricted to the columns K."""
    A = np.asarray(A, dtype=np.float64)
    B = leverage.sketch_dense(A, r, k, seed, prec)
    perm, _ = pivoted_qr(B, c)
    K = perm[:c].copy()
    R = leverage.sketch_R(B[:, K])
    return rownorms.rownorms_prod_dense(A[:, K], qr.upper_triangular_inverse(R)), K


def numerical_rank(rdiag, rcond):
    """Steps of a column-pivoted QR with |R_jj| > rcond |R_00|."""
    if len(rdiag) == 0 or rdiag[0] == 0.0:
        return 0
    return int(np.sum(rdiag > rcond * rdiag[0]))


def leverage_scores_truncated_dense(A, r, k, seed, prec, rcond):
    """(theta, rank, K): scores on the numerical-rank column subset of the
    sketch (Alg. 15 with its truncation), R from the QR of B[:, K]."""
    A = np.asarray(A, dtype=np.float64)
    B = leverage.sketch_dense(A, r, k, seed, prec)
    perm, rdiag = pivoted_qr(B)
    rank = numerical_rank(rdiag, rcond)
    K = perm[:rank].copy()
    R = qr.qr_r(B[:, K])
    return rownorms.rownorms_prod_dense(A[:, K], qr.upper_triangular_inverse(R)), rank, K
