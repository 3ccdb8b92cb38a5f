"""GPU parity of sketch-and-solve (Alg. 11, lsk_sketch_solve) and the
Gaussian CSR sketch (Alg. 4, lsk_csrjlt) against the oracle, on the same
seeded inputs and draws."""
import numpy as np
import pytest
import torch

import workloads
from oracle import gaussian as oga
from oracle import leverage as olev
from oracle import lsq as olsq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsk():
    from paper_2203_02798_gb300 import build
    build.build()
    import paper_2203_02798_gb300 as p
    return p


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def dense_csr(V, J, I, n, d):
    A = np.zeros((n, d))
    for i in range(n):
        A[i, J[I[i]:I[i + 1]]] += V[I[i]:I[i + 1]]
    return A


# ------------------------------------------------------------ sketch-and-solve
@pytest.mark.parametrize("prec,k", [("fp32", 128), ("bf16", 128), ("fp32", 0)])
def test_sketch_solve_dense(lsk, prec, k):
    n, d, r, seed = 60_000, 32, 2048, 5
    A = workloads.dense_normal(n, d, seed=1) * np.logspace(-1, 1, d).astype(np.float32)
    rng = np.random.default_rng(2)
    b = A.astype(np.float64) @ rng.standard_normal(d) + 0.3 * rng.standard_normal(n)
    x = host(lsk.sketch_solve(dev(A), dev(b), r, k, seed, prec))
    lsk.context().sync()
    op = oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32
    A64 = A.astype(np.float64)
    xo = olsq.sketch_solve_dense(A64, b, r, k, seed, op)
    # the GPU's x solves the oracle's sketched problem as well as the oracle's x
    SAb = olev.sketch_dense(np.hstack([A64, b[:, None]]), r, k, seed, op)
    res = lambda v: np.linalg.norm(SAb[:, :-1] @ v - SAb[:, -1])
    assert res(x) <= (1 + 1e-6) * res(xo)
    # the sketch differs from the oracle's by its FP32 (BF16x3: ~2^-17) rounding,
    # amplified by cond(A~) ~ 1e2 here
    assert np.linalg.norm(x - xo) <= (1e-3 if prec == "bf16" else 1e-4) * np.linalg.norm(xo)
    # and, as a sketch-and-solve solution, is near the least-squares residual
    x_ls = olsq.least_squares_qr(A64, b)
    assert np.linalg.norm(A64 @ x - b) <= 1.5 * np.linalg.norm(A64 @ x_ls - b)


def test_sketch_solve_consistent_system(lsk):
    n, d = 40_000, 20
    A = workloads.dense_normal(n, d, seed=3) * np.logspace(-2, 2, d).astype(np.float32)
    xs = np.linspace(-1, 2, d)
    b = A.astype(np.float64) @ xs
    x = host(lsk.sketch_solve(dev(A), dev(b), 1500, 80, 7, "fp32"))
    lsk.context().sync()
    # b~ is exact in FP64, A~ carries the FP32 rounding of the sketch sums, so
    # the sketched system is consistent only to that rounding, times cond(A)
    kappa = np.linalg.cond(A.astype(np.float64))
    assert np.linalg.norm(x - xs) <= 10 * 2.0**-24 * kappa * np.linalg.norm(xs)


def test_sketch_solve_csr(lsk):
    n, d, p = 100_000, 64, 0.05
    V, J, I = workloads.csr_bernoulli(n, d, p, seed=4)
    A64 = dense_csr(V.astype(np.float64), J, I, n, d)
    rng = np.random.default_rng(5)
    b = A64 @ rng.standard_normal(d) + 0.1 * rng.standard_normal(n)
    x = host(lsk.sketch_solve(lsk.csr_from_numpy(V, J, I, d), dev(b), 4096, 256, 3, "fp32"))
    lsk.context().sync()
    xo = olsq.sketch_solve_csr(V, J, I, n, d, b, 4096, 256, 3)
    assert np.linalg.norm(x - xo) <= 1e-4 * np.linalg.norm(xo)


def test_sketch_solve_rank_deficient_reported(lsk):
    A = workloads.dense_normal(5000, 8, seed=6)
    A[:, 3] = A[:, 2]
    b = np.ones(5000)
    lsk.sketch_solve(dev(A), dev(b), 256, 32, 1)
    with pytest.raises(lsk.LskError, match="RANK_DEFICIENT"):
        lsk.context().sync()


# ------------------------------------------------------------------ csrjlt
def rel_fro(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,d,p,m,prec", [(30_000, 100, 0.05, 64, "fp32"), (30_000, 100, 0.05, 64, "bf16"),
                                          (9_999, 300, 0.02, 37, "fp32"), (4_001, 7, 0.5, 129, "fp32"),
                                          (1_000, 700, 0.01, 40, "fp32")])
def test_csrjlt(lsk, n, d, p, m, prec):
    V, J, I = workloads.csr_bernoulli(n, d, p, seed=d)
    op = oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32
    C = host(lsk.csrjlt(lsk.csr_from_numpy(V, J, I, d), m, 11, prec)).astype(np.float64)
    lsk.context().sync()
    Co = oga.csrjlt(V, J, I, n, d, m, 11, op)
    assert rel_fro(C, Co) <= 1e-5
    # elementwise: FP32 products and sums of the column's nonzeros
    A = dense_csr(V.astype(np.float64), J, I, n, d)
    absG = np.abs(oga.gaussian_columns(m, 0, n, 11, op, oga.STREAM_JLT))
    bound = 2.0**-22 * (absG @ np.abs(A)) * (np.sum(A != 0, axis=0)[None, :] + 8) ** 0.5 + 1e-30
    assert np.all(np.abs(C - Co) <= 8 * bound)


def test_csrjlt_empty_rows_and_dense_rejected(lsk):
    n, d = 5000, 16
    V, J, I = workloads.csr_bernoulli(n, d, 0.0, seed=1)       # every row empty
    C = host(lsk.csrjlt(lsk.csr_from_numpy(V, J, I, d), 8, 1))
    lsk.context().sync()
    assert np.all(C == 0)
    with pytest.raises(lsk.LskError, match="UNSUPPORTED"):
        lsk.csrjlt(dev(workloads.dense_normal(100, 4, seed=1)), 8, 1)


# ------------------------------------------- Alg. 13 and Alg. 10 (Gram route)
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_leverage_scores_exact_dense(lsk, prec):
    n, d = 50_000, 48
    A = workloads.dense_normal(n, d, seed=8) * np.logspace(0, 1.5, d).astype(np.float32)
    A[:7] *= 40.0                                                # a few high-leverage rows
    theta = host(lsk.leverage_scores_exact(dev(A), prec)).astype(np.float64)
    lsk.context().sync()
    ref = olev.leverage_scores_exact_gram(A.astype(np.float64))
    assert np.max(np.abs(theta - ref) / ref) <= 1e-3
    assert abs(theta.sum() - d) <= 1e-3 * d


def test_leverage_scores_exact_csr(lsk):
    n, d = 80_000, 30
    V, J, I = workloads.csr_bernoulli(n, d, 0.1, seed=9)
    theta = host(lsk.leverage_scores_exact(lsk.csr_from_numpy(V, J, I, d))).astype(np.float64)
    lsk.context().sync()
    ref = olev.leverage_scores_exact_gram(dense_csr(V.astype(np.float64), J, I, n, d))
    nz = ref > 0
    assert np.all(theta[~nz] == 0)
    assert np.max(np.abs(theta[nz] - ref[nz]) / ref[nz]) <= 1e-3


@pytest.mark.parametrize("kind", ["dense", "csr"])
def test_least_squares_gram(lsk, kind):
    n, d = 60_000, 40
    rng = np.random.default_rng(11)
    if kind == "dense":
        A = workloads.dense_normal(n, d, seed=12) * np.logspace(0, 1.5, d).astype(np.float32)
        A64 = A.astype(np.float64)
        Ad = dev(A)
    else:
        V, J, I = workloads.csr_bernoulli(n, d, 0.2, seed=12)
        A64 = dense_csr(V.astype(np.float64), J, I, n, d)
        Ad = lsk.csr_from_numpy(V, J, I, d)
    b = A64 @ rng.standard_normal(d) + 0.2 * rng.standard_normal(n)
    x = host(lsk.least_squares_gram(Ad, dev(b), refine=2))
    lsk.context().sync()
    x_ls = olsq.least_squares_qr(A64, b)
    assert np.linalg.norm(x - x_ls) <= 1e-9 * np.linalg.norm(x_ls)
    xo = olsq.least_squares_gram(A64, b)
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
