"""GPU parity of column subset selection (Alg. 9) and the leverage scores on
the selected columns (Alg. 14, Alg. 16) against the oracle, same seeds."""
import numpy as np
import pytest
import torch

import workloads
from oracle import css as ocss
from oracle import gaussian as oga
from oracle import leverage as olev

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


def scaled(n, d, seed, lo=0.0, hi=2.0):
    return workloads.dense_normal(n, d, seed=seed) * np.logspace(lo, hi, d).astype(np.float32)


def test_column_select_dominant_columns(lsk):
    A = workloads.dense_normal(20_000, 32, seed=1)
    big = [29, 3, 17, 8]
    A[:, big] *= np.array([1000.0, 300.0, 100.0, 30.0], dtype=np.float32)
    cols = host(lsk.column_select(dev(A), 2048, 128, 5, 4))
    lsk.context().sync()
    assert list(cols) == big


@pytest.mark.parametrize("prec,k", [("fp32", 128), ("bf16", 128), ("fp32", 0)])
def test_column_select_matches_oracle(lsk, prec, k):
    """Well-separated column norms: the pivot sequence is unique, so the
    GPU's Gram-pivoted order equals the oracle's pivoted Householder order."""
    n, d, r, c = 30_000, 48, 2304, 24
    A = scaled(n, d, 2, 0.0, 3.0)
    op = oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32
    cols = host(lsk.column_select(dev(A), r, k, 7, c, prec))
    lsk.context().sync()
    ref = ocss.column_select_dense(A.astype(np.float64), r, k, 7, op, c)
    assert list(cols) == list(ref)


def test_column_select_csr(lsk):
    n, d = 100_000, 40
    V, J, I = workloads.csr_bernoulli(n, d, 0.05, seed=3)
    scale = np.logspace(0, 3, d)
    V = (V * scale[J]).astype(np.float32)
    cols = host(lsk.column_select(lsk.csr_from_numpy(V, J, I, d), 1600, 96, 2, 12))
    lsk.context().sync()
    ref = ocss.column_select_csr(V, J, I, n, d, 1600, 96, 2, oga.PREC_FP32, 12)
    assert list(cols) == list(ref)


@pytest.mark.parametrize("exact", [True, False])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_leverage_scores_hrn(lsk, exact, prec):
    n, d, r, k, c = 40_000, 64, 4096, 128, 20
    A = scaled(n, d, 4, 0.0, 2.0)
    op = oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32
    theta, cols = lsk.leverage_scores_hrn(dev(A), r, k, 3, c, exact=exact, prec=prec)
    lsk.context().sync()
    theta = host(theta).astype(np.float64)
    fn = ocss.hrn_exact_dense if exact else ocss.hrn_approx_dense
    ref, K = fn(A.astype(np.float64), r, k, 3, op, c)
    assert list(host(cols)) == list(K)
    assert np.max(np.abs(theta - ref) / ref) <= 1e-3
    if exact:
        assert abs(theta.sum() - c) <= 1e-3 * c                 # trace of the projector


def test_hrn_approx_with_all_columns_is_leverage(lsk):
    """c = d: Alg. 16 is Alg. 15 (the column order does not change A R^-1's row norms)."""
    A = scaled(30_000, 32, 5)
    theta, _ = lsk.leverage_scores_hrn(dev(A), 1024, 64, 9, 32, exact=False)
    ell = lsk.leverage_scores(dev(A), 1024, 64, 9)
    lsk.context().sync()
    theta, ell = host(theta).astype(np.float64), host(ell).astype(np.float64)
    assert np.max(np.abs(theta - ell) / ell) <= 1e-4


def test_column_select_planted_rank(lsk):
    """Rank 6 of d = 16: six independent pivots, then the deferred rank error."""
    rng = np.random.default_rng(6)
    basis = rng.standard_normal((10_000, 6))
    A = np.hstack([basis, basis @ rng.standard_normal((6, 10))]).astype(np.float32)
    cols = lsk.column_select(dev(A), 1024, 64, 1, 10)
    with pytest.raises(lsk.LskError, match="RANK_DEFICIENT"):
        lsk.context().sync()
    cols = host(cols)
    assert np.linalg.matrix_rank(A[:, cols[:6]].astype(np.float64)) == 6
    assert sorted(set(cols)) == sorted(cols)                    # a selection, no repeats


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_leverage_scores_truncated(lsk, prec):
    """Planted rank 7 of d = 24: the numerical rank is found and the scores
    equal the oracle's truncated Alg. 15 on the same sketch."""
    rng = np.random.default_rng(13)
    A = (rng.standard_normal((30_000, 7)) @ rng.standard_normal((7, 24))).astype(np.float32)
    A[:5] *= 30.0
    op = oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32
    theta, rank = lsk.leverage_scores_truncated(dev(A), 2048, 96, 4, rcond=1e-5, prec=prec)
    lsk.context().sync()
    ref, rank_o, K = ocss.leverage_scores_truncated_dense(A.astype(np.float64), 2048, 96, 4, op, 1e-5)
    assert rank == rank_o == 7
    theta = host(theta).astype(np.float64)
    assert np.max(np.abs(theta - ref) / ref) <= 1e-3


def test_leverage_scores_truncated_full_rank(lsk):
    A = scaled(20_000, 16, 14)
    theta, rank = lsk.leverage_scores_truncated(dev(A), 1024, 64, 2, rcond=1e-7)
    ell = lsk.leverage_scores(dev(A), 1024, 64, 2)
    lsk.context().sync()
    assert rank == 16
    theta, ell = host(theta).astype(np.float64), host(ell).astype(np.float64)
    assert np.max(np.abs(theta - ell) / ell) <= 1e-4


def test_new_entry_points_reject_bad_arguments(lsk):
    """Argument errors are reported before any launch and leave the context usable."""
    A = dev(workloads.dense_normal(2000, 8, seed=1))
    b = torch.zeros(2000, dtype=torch.float64, device="cuda")
    with pytest.raises(lsk.LskError, match="INVALID"):
        lsk.column_select(A, 256, 32, 1, 0)                      # c = 0
    with pytest.raises(lsk.LskError, match="INVALID"):
        lsk.column_select(A, 256, 32, 1, 9)                      # c > d
    with pytest.raises(lsk.LskError, match="INVALID"):
        lsk.leverage_scores_truncated(A, 256, 32, 1, rcond=1.5)
    with pytest.raises(lsk.LskError, match="INVALID"):
        lsk.least_squares_gram(A, b, refine=11)
    with pytest.raises(lsk.LskError, match="INVALID"):
        lsk.sketch_solve(A, b, 4, 0, 1)                          # r < d
    theta = lsk.leverage_scores_exact(A)
    lsk.context().sync()
    assert abs(host(theta).astype(np.float64).sum() - 8) <= 1e-3 * 8


def test_new_entry_points_on_empty_and_single_column(lsk):
    # d = 1: a single column selects itself; its exact scores are a_i^2 / ||a||^2
    a = workloads.dense_normal(3000, 1, seed=2)
    cols = host(lsk.column_select(dev(a), 64, 8, 1, 1))
    theta = host(lsk.leverage_scores_exact(dev(a))).astype(np.float64)
    lsk.context().sync()
    assert list(cols) == [0]
    ref = a[:, 0].astype(np.float64) ** 2 / np.sum(a.astype(np.float64) ** 2)
    assert np.max(np.abs(theta - ref) / ref) <= 1e-5
    # CSR with n = 0 rows: the Gaussian sketch is all zeros
    V = np.zeros(0, dtype=np.float32); J = np.zeros(0, dtype=np.int32); I = np.zeros(1, dtype=np.int64)
    C = host(lsk.csrjlt(lsk.csr_from_numpy(V, J, I, 5), 16, 1))
    lsk.context().sync()
    assert C.shape == (16, 5) and np.all(C == 0)
