"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times.  The oracle forms the whole FP64 sketch and R
(Householder QR of the sketch) and then computes exact scores for a sample of
rows, one by one; properties that hold at any size are checked on all rows.

  CSR 1,000,000 x 200, p = 0.01, r = 40,000, k = 400, FP32
  dense 4,000,000 x 256 (column scales 10^U(-3,3)), r = 65,536,
            k = 512, BF16 stages -- the bench's step; also the "next" rows
            on it: Alg. 15 with Pi, sketch-and-solve, column selection and
            the Alg. 16 scores
  the 512-problem batch (graph-captured, grouped stages), three
            problems checked against the oracle, every problem's scores in
            [0, 1.5] with sum within the sketch's distortion band
  one large served least-squares problem against the Householder
            least-squares solution
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import countsketch as ocs
from oracle import css as ocss
from oracle import gaussian as oga
from oracle import leverage as olev
from oracle import lsq as olsq
from oracle import qr as oqr

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def lsk():
    from paper_2203_02798_gb300 import build
    build.build()
    import paper_2203_02798_gb300 as p
    return p


def sampled_scores(rows_dense, R):
    """ell_i = ||a_i R^-1||^2 for the given dense rows (FP64 definition)."""
    Rinv = oqr.upper_triangular_inverse(R)
    Y = np.asarray(rows_dense, dtype=np.float64) @ Rinv
    return np.sum(Y * Y, axis=1)


def sample_rows(n, step, rng_seed=0):
    rng = np.random.default_rng(rng_seed)
    return np.unique(np.concatenate([np.arange(0, n, step), rng.integers(0, n, 2000), [n - 1]]))


@pytest.fixture(scope="module")
def dense_4m():
    """The 4,000,000 x 256 A (column scales 10^U(-3,3)) and the
    oracle's FP64 sketches of it (CountSketch r = 65,536, BF16 G with
    k = 512), formed once for the tests of this module."""
    n, d, r, k, seed = 4_000_000, 256, 65_536, 512, 2
    A = np.empty((n, d), dtype=np.float32)
    workloads.dense_colscaled(n=n, d=d, seed=2, out=A)
    SA = ocs.cs_sketch_dense(A, r, seed)                       # FP64, all 4M rows
    GSA = oga.gauss_sketch(SA, k, seed, oga.PREC_BF16)
    return dict(A=A, n=n, d=d, r=r, k=k, seed=seed, SA=SA, GSA=GSA, R=olev.sketch_R(GSA))


def test_dense_4M_x_256_bf16(lsk, dense_4m):
    c3 = dense_4m
    A, n, d = c3["A"], c3["n"], c3["d"]
    Ad = torch.from_numpy(A).cuda()
    ell, R = lsk.leverage_scores(Ad, c3["r"], c3["k"], c3["seed"], "bf16", return_R=True)
    lsk.context().sync()
    ell = ell.cpu().numpy().astype(np.float64)
    Rg = R.cpu().numpy()
    del Ad
    torch.cuda.empty_cache()
    Ro = c3["R"]
    rows = sample_rows(n, 997)
    ref = sampled_scores(A[rows], Ro)
    assert np.max(np.abs(ell[rows] - ref) / ref) <= 1e-3
    colnorm = np.linalg.norm(Ro, axis=0)
    assert np.all(np.abs(Rg - Ro) <= 1e-4 * colnorm[None, :])
    assert np.all(ell >= 0) and np.all(np.isfinite(ell))
    # sum of the estimates = ||A R^-1||_F^2 = sum of sigma_j^2 of A R^-1: d up to the
    # sketch's distortion (k = 2d Gaussian after CountSketch)
    assert 0.2 * d <= ell.sum() <= 5.0 * d


def test_dense_4M_x_256_tf32(lsk, dense_4m):
    """Config 3 as it names its arithmetic: the BF16 Gaussian stage and the
    fused TF32 row-norm kernel (the bench's headline step), against the
    oracle's scores on sampled rows."""
    c3 = dense_4m
    A, n, d = c3["A"], c3["n"], c3["d"]
    Ad = torch.from_numpy(A).cuda()
    ctx = lsk.context()
    ctx.profile(True)
    ctx.profile_reset()
    ell = lsk.leverage_scores(Ad, c3["r"], c3["k"], c3["seed"], "tf32")
    ctx.sync()
    names = set(ctx.profile_totals())
    ctx.profile(False)
    ell = ell.cpu().numpy().astype(np.float64)
    del Ad
    torch.cuda.empty_cache()
    assert "rownorm_dense_tf32" in names
    rows = sample_rows(n, 997, 3)
    ref = sampled_scores(A[rows], c3["R"])
    assert np.max(np.abs(ell[rows] - ref) / ref) <= 1e-3
    assert np.all(ell >= 0) and np.all(np.isfinite(ell))


def test_dense_4M_x_256_count_gauss(lsk, dense_4m):
    """The fused CountSketch + Gaussian stage (S A kept on chip) at the bench's
    size against the oracle's FP64 G (S A) on the same seeds."""
    c3 = dense_4m
    Ad = torch.from_numpy(c3["A"]).cuda()
    got = lsk.count_gauss(Ad, c3["r"], c3["k"], c3["seed"]).cpu().numpy().astype(np.float64)
    del Ad
    torch.cuda.empty_cache()
    ref = c3["GSA"]
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)


def test_dense_4M_x_256_jl_sketch_solve_and_column_selection(lsk, dense_4m):
    """The "next" rows at the bench's size: Alg. 15 with Pi (m = 64), sketch-
    and-solve (Alg. 11) and column selection with the Alg. 16 scores (c = 64),
    each against the oracle on the same FP64 sketch."""
    c3 = dense_4m
    A, n, d, r, k, seed = c3["A"], c3["n"], c3["d"], c3["r"], c3["k"], c3["seed"]
    Ro = c3["R"]
    Ad = torch.from_numpy(A).cuda()
    rows = sample_rows(n, 1999, 7)
    # Alg. 15 with the right projection
    ell = lsk.leverage_scores_jl(Ad, r, k, 64, seed, "bf16").cpu().numpy().astype(np.float64)
    X = oqr.upper_triangular_inverse(Ro) @ oga.jl_matrix(d, 64, seed)
    ref = np.sum((A[rows].astype(np.float64) @ X) ** 2, axis=1)
    assert np.max(np.abs(ell[rows] - ref) / ref) <= 1e-3
    # sketch-and-solve: b through the same S and G
    rng = np.random.default_rng(31)
    xs = rng.standard_normal(d) / np.linalg.norm(Ro, axis=0)
    b = np.empty(n)
    for i0 in range(0, n, 1 << 18):
        b[i0:i0 + (1 << 18)] = A[i0:i0 + (1 << 18)].astype(np.float64) @ xs
    b += rng.standard_normal(n) * 0.1 * np.std(b)
    x = lsk.sketch_solve(Ad, torch.from_numpy(b).cuda(), r, k, seed, "bf16").cpu().numpy()
    Sb = ocs.cs_sketch_dense(b[:, None], r, seed)
    bt = oga.gauss_sketch(Sb, k, seed, oga.PREC_BF16)[:, 0]
    xo = olsq.sketch_solve(np.hstack([c3["GSA"], bt[:, None]]))
    res = lambda v: np.linalg.norm(c3["GSA"] @ v - bt)
    assert res(x) <= (1 + 1e-6) * res(xo)
    # column selection and the Alg. 16 scores on the selected columns
    theta, cols = lsk.leverage_scores_hrn(Ad, r, k, seed, 64, exact=False, prec="bf16")
    lsk.context().sync()
    cols = cols.cpu().numpy()
    perm, rdiag = ocss.pivoted_qr(c3["GSA"], 64)
    assert len(set(cols)) == 64
    mism = [j for j in range(64) if cols[j] != perm[j]]
    if mism:
        # the two sketches differ by rounding, so the order is unique only up to
        # near-ties: at the first difference both columns must be (nearly)
        # farthest from the span of the common prefix
        j = mism[0]
        Q = np.linalg.qr(c3["GSA"][:, perm[:j]])[0]
        dist = lambda col: np.linalg.norm(c3["GSA"][:, col] - Q @ (Q.T @ c3["GSA"][:, col]))
        assert abs(dist(cols[j]) - dist(perm[j])) <= 1e-5 * dist(perm[j])
    Rk = olev.sketch_R(c3["GSA"][:, cols])
    Y = A[rows][:, cols].astype(np.float64) @ oqr.upper_triangular_inverse(Rk)
    ref = np.sum(Y * Y, axis=1)
    theta = theta.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(theta[rows] - ref) / ref) <= 1e-3
    del Ad
    torch.cuda.empty_cache()


def test_csr_1M_x_200_fp32(lsk):
    n, d, r, k, seed = 1_000_000, 200, 40_000, 400, 1
    V, J, I = workloads.csr_bernoulli(n, d, 0.01, seed=1)
    ell = lsk.leverage_scores(lsk.csr_from_numpy(V, J, I, d), r, k, seed, "fp32")
    lsk.context().sync()
    ell = ell.cpu().numpy().astype(np.float64)
    SA = ocs.cs_sketch_csr(V, J, I, n, d, r, seed)
    Ro = olev.sketch_R(oga.gauss_sketch(SA, k, seed, oga.PREC_FP32))
    rows = sample_rows(n, 499, 1)
    dense = np.zeros((rows.size, d))
    for t, i in enumerate(rows):
        dense[t, J[I[i]:I[i + 1]]] = V[I[i]:I[i + 1]]
    ref = sampled_scores(dense, Ro)
    nz = ref > 0
    assert np.all(ell[rows][~nz] == 0)                         # empty rows score zero
    assert np.max(np.abs(ell[rows][nz] - ref[nz]) / ref[nz]) <= 1e-3
    empty = np.diff(I) == 0
    assert np.all(ell[empty] == 0)
    assert 0.2 * d <= ell.sum() <= 5.0 * d


def test_batch_512_problems(lsk):
    specs = workloads.batch_specs(512, seed=3)
    probs = []
    for sp in specs:
        if sp["kind"] == "dense":
            A = workloads.batch_problem_torch(sp)
        else:
            V, J, I = workloads.batch_problem_torch(sp)
            A = lsk.CSR(V, J, I, sp["n"], sp["d"])
        probs.append((A, sp["r"], sp["k"], sp["sketch_seed"]))
    outs = lsk.batch_leverage_scores(probs, prec="bf16", graph=True, autotune=True)
    lsk.context().sync()
    for (A, r, k, s), ell, sp in zip(probs, outs, specs):
        e = ell.cpu().numpy()
        assert np.all(np.isfinite(e)) and np.all(e >= 0) and np.all(e <= 1.5), sp
        assert 0.2 * sp["d"] <= e.sum() <= 5.0 * sp["d"], sp
    # against the oracle: the largest dense d = 256 problem, the largest CSR
    # d = 256 problem and the smallest CSR d = 32 problem
    dense256 = max((i for i, sp in enumerate(specs) if sp["kind"] == "dense" and sp["d"] == 256),
                   key=lambda i: specs[i]["n"])
    csr256 = max((i for i, sp in enumerate(specs) if sp["kind"] == "csr" and sp["d"] == 256),
                 key=lambda i: specs[i]["n"])
    csr32 = min((i for i, sp in enumerate(specs) if sp["kind"] == "csr" and sp["d"] == 32),
                key=lambda i: specs[i]["n"])
    for i in (dense256, csr256, csr32):
        sp = specs[i]
        A, r, k, s = probs[i]
        ell = outs[i].cpu().numpy().astype(np.float64)
        n, d = sp["n"], sp["d"]
        if sp["kind"] == "dense":
            Ah = A.cpu().numpy()
            SA = ocs.cs_sketch_dense(Ah, r, s)
        else:
            V, J, I = (A.V.cpu().numpy(), A.J.cpu().numpy(), A.I.cpu().numpy())
            SA = ocs.cs_sketch_csr(V, J, I, n, d, r, s)
        Ro = olev.sketch_R(oga.gauss_sketch(SA, k, s, oga.PREC_BF16))
        rows = sample_rows(n, max(1, n // 3000), i)
        if sp["kind"] == "dense":
            dense = Ah[rows]
        else:
            dense = np.zeros((rows.size, d))
            for t, j in enumerate(rows):
                dense[t, J[I[j]:I[j + 1]]] = V[I[j]:I[j + 1]]
        ref = sampled_scores(dense, Ro)
        nz = ref > 0
        assert np.all(ell[rows][~nz] == 0)
        assert np.max(np.abs(ell[rows][nz] - ref[nz]) / ref[nz]) <= 1e-3, sp


def test_large_served_least_squares(lsk):
    specs = workloads.batch_specs(512, seed=3)
    i = max((i for i, sp in enumerate(specs) if sp["kind"] == "dense" and sp["d"] == 256),
            key=lambda i: specs[i]["n"])
    sp = specs[i]
    A = workloads.batch_problem_torch(sp)
    xs, b = workloads.lsq_rhs_torch(lambda x: (A.double() @ x), sp["n"], sp["d"], seed=10_000 + i)
    x, info = lsk.sketch_precondition_lsq(A, b, r=sp["r"], k=sp["k"], seed=sp["sketch_seed"])
    lsk.context().sync()
    assert info["status"] == 0 and info["eta"] <= 1e-10
    Ah = A.cpu().numpy().astype(np.float64)
    bh = b.cpu().numpy()
    xh = x.cpu().numpy()
    eta = olsq.normal_equation_residual(lambda v: Ah @ v, lambda v: Ah.T @ v, bh, xh)
    assert eta <= 1e-10                                        # recomputed on the host in FP64
    x_ls = olsq.least_squares_qr(Ah, bh)
    assert np.linalg.norm(xh - x_ls) <= 1e-8 * np.linalg.norm(x_ls)
