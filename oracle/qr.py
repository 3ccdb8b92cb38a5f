"""Householder QR of the sketch, R^-1, the full-rank check.
Oracle; test infrastructure.

Alg. 12 and Alg. 15 factor the small sketch (G*S*A or S*A) with an SVD; the
reading used here factors it with a QR, B = Q R, which yields the same
row norms ||A_i R^-1|| = ||A_i V Sigma^-1|| in exact arithmetic (R^-1 and
V Sigma^-1 differ by an orthogonal factor on the right).  The QR is plain
Householder triangularisation (Golub & Van Loan, Matrix Computations, 4th
ed., Sec. 5.2.2): column by column, a reflector P = I - beta v v^T maps the
remaining part of the column onto a multiple of e_1 and is applied to the
trailing columns.  R is sign-normalised (R_jj > 0), which makes it unique
for a full-rank B.  The paper truncates small singular values ("truncate if
needed", Alg. 12 / 15, rcond unspecified); the reading used here requires
full column rank instead and reports rank deficiency when
min R_jj <= 16 * eps64 * d * max R_jj.
"""
import numpy as np

EPS64 = np.finfo(np.float64).eps


class RankDeficient(ValueError):
    pass


def _house(x):
    """Reflector (v, beta) with (I - beta v v^T) x = -copysign(||x||, x_0) e_1."""
    nrm = np.linalg.norm(x)
    if nrm == 0.0:
        return None, 0.0
    v = x.copy()
    v[0] += np.copysign(nrm, x[0])
    return v, 2.0 / float(v @ v)


def householder_qr(B):
    """Householder QR of B (m x n, m >= n).

    Returns (reflectors, R) where reflectors is a list of (v, beta) for
    columns 0..n-1 (v acts on rows j..m-1) and R (n x n) is upper triangular
    with a non-negative diagonal.  The sign normalisation is recorded in
    the returned ``signs`` so that B = Q R with Q = H_0 ... H_{n-1} [I; 0] D.
    """
    W = np.array(B, dtype=np.float64, copy=True)
    m, n = W.shape
    if m < n:
        raise ValueError("householder_qr needs m >= n")
    refl = []
    for j in range(n):
        v, beta = _house(W[j:, j])
        refl.append((v, beta))
        if v is not None:
            W[j:, j:] -= beta * np.outer(v, v @ W[j:, j:])
    R = np.triu(W[:n, :n])
    signs = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    R = signs[:, None] * R
    return refl, R, signs


def qr_r(B):
    """Sign-normalised R of B = Q R (upper triangular, R_jj >= 0)."""
    return householder_qr(B)[1]


def apply_qt(refl, signs, y):
    """Q^T y for the thin Q of :func:`householder_qr` (first n entries)."""
    y = np.array(y, dtype=np.float64, copy=True)
    for j, (v, beta) in enumerate(refl):
        if v is not None:
            y[j:] -= beta * v * (v @ y[j:])
    n = len(refl)
    return signs * y[:n]


def thin_q(refl, signs, m):
    """Explicit thin Q (m x n) of :func:`householder_qr`."""
    n = len(refl)
    Q = np.zeros((m, n), dtype=np.float64)
    Q[:n, :n] = np.eye(n)
    for j in range(n - 1, -1, -1):
        v, beta = refl[j]
        if v is not None:
            Q[j:, :] -= beta * np.outer(v, v @ Q[j:, :])
    return Q * signs[None, :]


def check_full_rank(R):
    """Raise RankDeficient when min R_jj <= 16 eps d max R_jj."""
    dg = np.abs(np.diag(R))
    d = len(dg)
    if d == 0 or not np.all(np.isfinite(R)) or dg.min() <= 16.0 * EPS64 * d * dg.max():
        raise RankDeficient("sketch is numerically rank deficient")


def upper_triangular_inverse(R):
    """R^-1 for upper-triangular R by back substitution, one row at a time."""
    R = np.asarray(R, dtype=np.float64)
    d = R.shape[0]
    X = np.zeros((d, d), dtype=np.float64)
    E = np.eye(d)
    for i in range(d - 1, -1, -1):
        X[i, :] = (E[i, :] - R[i, i + 1:] @ X[i + 1:, :]) / R[i, i]
    return X
