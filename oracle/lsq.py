"""Least squares (oracle; test infrastructure): through the Gram pseudoinverse (Alg. 10), through
sketches: sketch-and-precondition (Alg. 12) with LSQR, and sketch-and-solve
(Alg. 11).

Alg. 12 (Sec. 4.2): sketch A, factor the sketch, take N as the inverse
factor, solve min_y ||A N y - b|| with "a parallel preconditioned iterative
method", and return x = N y.  The reading used here: N = R^-1 from the QR
of the sketch (see ``oracle/qr.py``), the iterative method is LSQR (Paige &
Saunders, ACM TOMS 8(1), 1982, Sec. 4), and the solve is wrapped in
iterative refinement: r_t = b - A x_t, dy = LSQR(A N, r_t), x_{t+1} =
x_t + N dy, until the relative normal-equation residual
eta = ||A^T (b - A x)|| / ||A^T b|| is small.  Everything here is float64.
"""
import numpy as np

from . import leverage, qr


def lsqr(matvec, rmatvec, b, n_cols, atol=1e-14, btol=1e-14, max_iter=1000):
    """LSQR of Paige & Saunders (1982, Sec. 4.1) for min ||M y - b||.

    matvec(v) = M v, rmatvec(u) = M^T u.  Returns (y, iterations).
    Stops when ||M^T r|| <= atol ||M|| ||r|| or ||r|| <= btol ||b||.
    """
    b = np.asarray(b, dtype=np.float64)
    y = np.zeros(n_cols)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return y, 0
    u = b / beta
    v = rmatvec(u)
    alpha = np.linalg.norm(v)
    if alpha == 0.0:
        return y, 0
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = 0.0
    for it in range(1, max_iter + 1):
        # bidiagonalisation step
        u = matvec(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0.0:
            u = u / beta
        anorm2 += alpha * alpha + beta * beta
        v = rmatvec(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0.0:
            v = v / alpha
        # plane rotation eliminating beta
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        # update y and w
        y = y + (phi / rho) * w
        w = v - (theta / rho) * w
        # stopping tests (Paige & Saunders, Sec. 6)
        rnorm = phibar
        arnorm = phibar * alpha * abs(c)
        if arnorm <= atol * np.sqrt(anorm2) * rnorm or rnorm <= btol * np.linalg.norm(b):
            return y, it
    return y, max_iter


def normal_equation_residual(matvec, rmatvec, b, x):
    """eta = ||A^T (b - A x)|| / ||A^T b|| in float64."""
    r = np.asarray(b, dtype=np.float64) - matvec(x)
    return np.linalg.norm(rmatvec(r)) / np.linalg.norm(rmatvec(np.asarray(b, dtype=np.float64)))


def sketch_precondition_lsq(matvec, rmatvec, b, Rinv, tol=1e-10, max_refine=10,
                            max_iter=1000):
    """Alg. 12 with N = Rinv, LSQR inner solves and float64 refinement.

    Returns (x, info) with info = dict(iters, refinements, eta).
    """
    d = Rinv.shape[0]
    x = np.zeros(d)
    iters = 0
    eta = np.inf
    for t in range(max_refine + 1):
        eta = normal_equation_residual(matvec, rmatvec, b, x)
        if eta <= tol:
            return x, dict(iters=iters, refinements=t, eta=eta)
        r = np.asarray(b, dtype=np.float64) - matvec(x)
        dy, it = lsqr(lambda v: matvec(Rinv @ v), lambda u: Rinv.T @ rmatvec(u), r, d,
                      max_iter=max_iter)
        iters += it
        x = x + Rinv @ dy
    return x, dict(iters=iters, refinements=max_refine, eta=eta)


def lsq_dense(A, b, r, k, seed, prec=0, tol=1e-10):
    """Alg. 12 for dense A: R from the sketch, then preconditioned LSQR."""
    A = np.asarray(A, dtype=np.float64)
    R = leverage.sketch_R(leverage.sketch_dense(A, r, k, seed, prec))
    Rinv = qr.upper_triangular_inverse(R)
    return sketch_precondition_lsq(lambda v: A @ v, lambda u: A.T @ u, b, Rinv, tol)


def least_squares_qr(A, b):
    """x_ls = R^-1 Q^T b from the Householder QR of A (reference solution)."""
    refl, R, signs = qr.householder_qr(A)
    qtb = qr.apply_qt(refl, signs, b)
    Rinv = qr.upper_triangular_inverse(R)
    return Rinv @ qtb


def sketch_solve(SAb):
    """Alg. 11 on a sketched augmented matrix SAb = (A~ b~) (rows x (d + 1)):
    x = argmin ||A~ x - b~||, from the Householder QR of A~ (full column
    rank required; the QR stands in for the SVD of Alg. 11 step 2, which gives
    the same minimiser when A~ has full rank)."""
    SAb = np.asarray(SAb, dtype=np.float64)
    At, bt = SAb[:, :-1], SAb[:, -1]
    refl, R, signs = qr.householder_qr(At)
    qr.check_full_rank(R)
    return qr.upper_triangular_inverse(R) @ qr.apply_qt(refl, signs, bt)


def sketch_solve_dense(A, b, r, k, seed, prec=0):
    """Alg. 11 for dense A: (A~ b~) = G S (A b) (k = 0: S (A b)), then solve."""
    A = np.asarray(A, dtype=np.float64)
    Ab = np.hstack([A, np.asarray(b, dtype=np.float64)[:, None]])
    return sketch_solve(leverage.sketch_dense(Ab, r, k, seed, prec))


def sketch_solve_csr(V, J, I, n, d, b, r, k, seed, prec=0):
    """Alg. 11 for CSR A: the augmented column b joins every row (CSR of (A b))."""
    V = np.asarray(V, dtype=np.float64)
    J = np.asarray(J)
    I = np.asarray(I)
    b = np.asarray(b, dtype=np.float64)
    cnt = np.diff(I) + 1
    I2 = np.concatenate([[0], np.cumsum(cnt)])
    V2 = np.empty(I2[-1])
    J2 = np.empty(I2[-1], dtype=np.int64)
    for i in range(n):
        a, e = I[i], I[i + 1]
        V2[I2[i]:I2[i + 1] - 1] = V[a:e]
        J2[I2[i]:I2[i + 1] - 1] = J[a:e]
        V2[I2[i + 1] - 1] = b[i]
        J2[I2[i + 1] - 1] = d
    return sketch_solve(leverage.sketch_csr(V2, J2, I2, n, d + 1, r, k, seed, prec))


def least_squares_gram(A, b, rcond=1e-12):
    """Alg. 10: B = A^T A, B = V Sigma V^T (eigen-decomposition of the
    symmetric B, the library step), c = A^T b, x = V Sigma^+ V^T c, with
    eigenvalues below rcond * max truncated."""
    A = np.asarray(A, dtype=np.float64)
    w, V = np.linalg.eigh(A.T @ A)
    keep = w > rcond * w.max()
    c = A.T @ np.asarray(b, dtype=np.float64)
    return V[:, keep] @ ((V[:, keep].T @ c) / w[keep])
