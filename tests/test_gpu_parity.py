"""GPU parity: every C-ABI call against the FP64 oracle, element by element.

Sizes span several tiles / warps / buckets and a ragged tail.  Tolerances:
  - hash and signs: bit-exact;
  - integer-valued inputs (every FP32 partial sum exact): bit-exact;
  - FP32 paths: the stated bound of 1e-5 relative Frobenius error on SA
    and A^T A, plus element-wise bounds from the summation length;
  - leverage scores: max relative error <= 1e-3 against the oracle's estimate
    on the same seeds;
  - least squares: eta = ||A^T(b - Ax)|| / ||A^T b|| <= 1e-10, computed by the
    oracle in FP64 on the GPU's x.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import countsketch as ocs
from oracle import gaussian as oga
from oracle import gram as ogr
from oracle import leverage as olev
from oracle import lsq as olsq
from oracle import qr as oqr
from oracle import rownorms as orn

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def csr_dev(lsk, V, J, I, d):
    return lsk.csr_from_numpy(V, J, I, d)


# ---------------------------------------------------------------- hash / G --
@pytest.mark.parametrize("n,r,seed", [(100_003, 2500, 0), (70_001, 1, 5), (5000, 2**31 - 1, 2**63 + 17),
                                      (1, 7, 3), (0, 3, 1)])
def test_hash_bit_exact(lsk, n, r, seed):
    b, s = lsk.debug_hash(n, r, seed)
    ob, os_ = ocs.countsketch_hash(n, r, seed)
    assert np.array_equal(host(b).astype(np.int64), ob)
    assert np.array_equal(host(s).astype(np.int8), os_)


@pytest.mark.parametrize("k,r,seed", [(100, 2500, 0), (13, 777, 2**40 + 3)])
def test_gaussian_fp32_matches(lsk, k, r, seed):
    G = host(lsk.debug_gauss(k, r, seed, "fp32")).astype(np.float64)
    Go = oga.gaussian_matrix(k, r, seed, oga.PREC_FP32)
    # the same float32-exact uniforms on both sides: only the float32
    # evaluation of log / sqrt / sincospi and the scaling differ (a few ulp)
    assert np.all(np.abs(G - Go) <= 16 * U32 * np.abs(Go) + 4 * U32 / np.sqrt(k))


def test_gaussian_bf16_rounding_agrees(lsk):
    k, r, seed = 64, 20000, 9
    G = host(lsk.debug_gauss(k, r, seed, "bf16")).astype(np.float64)
    Go = oga.gaussian_matrix(k, r, seed, oga.PREC_BF16)
    diff = G != Go
    # both sides round the float32 value; only few-ulp float32 evaluation
    # differences that straddle a bfloat16 rounding midpoint disagree, by one
    # bf16 ulp (expected rate ~ ulps * 2^-16)
    assert diff.mean() < 2e-4
    if diff.any():
        assert np.all(np.abs(G[diff] - Go[diff]) <= 2.0**-7 * np.abs(Go[diff]) * 1.01)


# ---------------------------------------------------------------- S * A ----
@pytest.mark.parametrize("n,d,r", [(20_011, 50, 2500), (9_000, 256, 700), (4_099, 130, 5000),
                                   (3_000, 3, 1), (1_000, 1, 7), (2_500, 64, 40_000),
                                   (300_000, 4, 81_925), (200_003, 4, 1_000_003)])
def test_cs_sketch_dense_integer_bit_exact(lsk, n, d, r):
    """Exact on integer data; the last two cases span 41 and 489 tiles of
    the bucket-offset scan, so its look-back reads more than one window of 32
    tiles (r not a multiple of the 2,048-counter tile, r > n)."""
    A = workloads.integer_dense(n, d, seed=n + d)
    SA = host(lsk.cs_sketch(dev(A), r, seed=11))
    ref = ocs.cs_sketch_dense(A, r, 11)
    assert np.array_equal(SA.astype(np.float64), ref)


@pytest.mark.parametrize("n,d,r,seed", [(20_000, 50, 2500, 0), (60_000, 256, 1024, 3),
                                        (7_777, 200, 333, 2**50)])
def test_cs_sketch_dense_float(lsk, n, d, r, seed):
    A = workloads.dense_normal(n, d, seed=seed + 1)
    SA = host(lsk.cs_sketch(dev(A), r, seed)).astype(np.float64)
    bucket, sign = ocs.countsketch_hash(n, r, seed)
    ref = ocs.countsketch_apply_dense(A, bucket, sign, r)
    absref = ocs.countsketch_apply_dense(np.abs(A), bucket, np.ones_like(sign), r)
    m = np.bincount(bucket, minlength=r).max()
    assert rel_fro(SA, ref) <= 1e-5
    assert np.all(np.abs(SA - ref) <= 2 * m * U32 * absref + 1e-30)


def test_cs_sketch_dense_strided_and_empty(lsk):
    A = workloads.dense_normal(3000, 40, seed=4)
    big = torch.zeros((3000, 48), dtype=torch.float32, device="cuda")
    big[:, :40] = dev(A)
    SA = host(lsk.cs_sketch(big[:, :40], 97, 5)).astype(np.float64)
    assert rel_fro(SA, ocs.cs_sketch_dense(A, 97, 5)) <= 1e-6
    empty = torch.zeros((0, 16), dtype=torch.float32, device="cuda")
    SA0 = lsk.cs_sketch(empty, 10, 1)
    assert torch.count_nonzero(SA0).item() == 0


@pytest.mark.parametrize("n,d,p,r", [(50_000, 200, 0.01, 4000), (20_000, 64, 0.2, 300), (1000, 33, 0.0, 17)])
def test_cs_sketch_csr_integer_bit_exact(lsk, n, d, p, r):
    V, J, I = workloads.integer_csr(n, d, p, seed=n)
    SA = host(lsk.cs_sketch(csr_dev(lsk, V, J, I, d), r, 7))
    ref = ocs.cs_sketch_csr(V, J, I, n, d, r, 7)
    assert np.array_equal(SA.astype(np.float64), ref)


def test_cs_sketch_csr_float(lsk):
    n, d, r = 200_000, 200, 8000
    V, J, I = workloads.csr_bernoulli(n, d, 0.01, seed=1)
    SA = host(lsk.cs_sketch(csr_dev(lsk, V, J, I, d), r, 1)).astype(np.float64)
    ref = ocs.cs_sketch_csr(V, J, I, n, d, r, 1)
    assert rel_fro(SA, ref) <= 1e-6


def test_cs_sketch_bad_csr_reported(lsk):
    n, d = 500, 16
    V, J, I = workloads.integer_csr(n, d, 0.3, seed=3)
    J = J.copy()
    J[len(J) // 2] = d          # out of range: skipped by the kernel, flagged
    ctx = lsk.context()
    lsk.cs_sketch(csr_dev(lsk, V, J, I, d), 10, 1)
    with pytest.raises(lsk.LskError) as ei:
        ctx.sync()
    assert ei.value.name == "BAD_CSR"
    ctx.sync()                   # the flag is cleared


# ---------------------------------------------------------------- G * SA ---
# fp32 with r >= 8192 runs on the tensor cores (three bf16 terms of G and SA)
@pytest.mark.parametrize("r,d,k,prec", [(2500, 50, 100, "fp32"), (40_000, 200, 400, "fp32"),
                                        (8192, 256, 512, "fp32"), (20_011, 64, 100, "fp32"), (9000, 130, 257, "fp32"),
                                        (3000, 256, 512, "bf16"), (777, 3, 5, "fp32"), (1000, 129, 70, "bf16"),
                                        (65_536, 256, 512, "bf16"), (40_000, 200, 400, "bf16"), (31, 7, 3, "bf16"),
                                        (2500, 50, 100, "bf16")])
def test_gauss_sketch(lsk, r, d, k, prec):
    SA = workloads.dense_normal(r, d, seed=r + d)
    got = host(lsk.gauss_sketch(dev(SA), k, 21, prec)).astype(np.float64)
    ref = oga.gauss_sketch(SA.astype(np.float64), k, 21, oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32)
    # FP32: 1e-5.  BF16: G is exact in bf16 on both sides except the rare
    # rounding disagreements above (each one bf16 ulp of one entry)
    assert rel_fro(got, ref) <= (1e-5 if prec == "fp32" else 1e-4)
    G = oga.gaussian_matrix(k, r, 21, oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32)
    bound = np.abs(G) @ np.abs(SA.astype(np.float64))
    slack = (2.0**-7 if prec == "bf16" else 0.0) * bound   # rare bf16 rounding disagreements of G
    assert np.all(np.abs(got - ref) <= 2 * (r + 16) * U32 * bound + slack + 1e-30)


# ---------------------------------------------------------------- A^T A ----
@pytest.mark.parametrize("n,d", [(20_000, 50), (33_000, 256), (1000, 3), (5000, 130)])
def test_gram_dense(lsk, n, d):
    A = workloads.dense_normal(n, d, seed=d)
    C = host(lsk.gram(dev(A))).astype(np.float64)
    ref = ogr.gram_dense(A)
    assert rel_fro(C, ref) <= 1e-5
    assert np.array_equal(C, C.T)


def test_gauss_fp32_runs_on_the_tensor_cores(lsk):
    """The FP32 Gaussian stage of a long sketch takes the three-term tensor-core
    kernel (checked by its profile name), and its result is as close to the
    FP64 product as the SIMT FP32 kernel's is on a short sketch."""
    r, d, k = 16_384, 200, 400
    SA = workloads.dense_normal(r, d, seed=4) * (10.0 ** np.linspace(-3, 3, d)).astype(np.float32)
    ctx = lsk.context()
    ctx.profile(True)
    ctx.profile_reset()
    got = host(lsk.gauss_sketch(dev(SA), k, 5, "fp32")).astype(np.float64)
    ctx.sync()
    names = set(ctx.profile_totals())
    ctx.profile(False)
    assert "gauss_tc_fp32" in names and "gauss_simt" not in names
    # against the oracle: the FP32 tolerance (G's float32 evaluation differs
    # from the oracle's by a few ulp, as on the SIMT path)
    G = oga.gaussian_matrix(k, r, 5, oga.PREC_FP32)
    assert rel_fro(got, G @ SA.astype(np.float64)) <= 1e-5
    # the tensor-core arithmetic alone: against the FP64 product of the
    # device's own G -- products of three-term splits (below 2^-22 |G||SA|
    # each) and FP32 sums; the tensor pipe's FP32 accumulation rounds toward
    # zero, ~2^-25 of the running sum per accumulation (96 a slice here), so
    # the entries come out ~2e-6 small in magnitude: bounded by 4e-6 relative
    Gd = host(lsk.debug_gauss(k, r, 5, "fp32")).astype(np.float64)
    ref = Gd @ SA.astype(np.float64)
    bound = np.abs(Gd) @ np.abs(SA.astype(np.float64))
    assert np.all(np.abs(got - ref) <= (2 * (r + 16) * U32 + 2.0**-21) * bound)
    assert rel_fro(got, ref) <= 4e-6


def test_gram_dense_integer_exact_and_alpha_beta(lsk):
    A = workloads.integer_dense(4000, 70, seed=2, lo=-3, hi=3)
    C = host(lsk.gram(dev(A))).astype(np.float64)
    assert np.array_equal(C, ogr.gram_dense(A))
    C0 = workloads.dense_normal(70, 70, seed=3)
    Ct = dev(C0.copy())
    lsk.gram(dev(A), alpha=0.5, beta=-2.0, C=Ct)
    ref = ogr.gram_dense(A, 0.5, -2.0, C0)
    assert rel_fro(host(Ct).astype(np.float64), ref) <= 1e-6


@pytest.mark.parametrize("n,d", [(100_003, 256), (5_000, 50), (2_049, 130), (1, 7), (4_096, 128)])
def test_gram_dense_bf16_tensor_cores(lsk, n, d):
    """BF16x3 Gram on tcgen05: two M tiles (d > 128), ragged d and slices,
    one row.  Bound per entry: the split leaves at most 2^-16 |a_i a_j| per
    product, and at most 3 * 1024 products are added in FP32 per slice."""
    A = workloads.dense_normal(n, d, seed=d + 7) * (10.0 ** np.linspace(-1, 1, d)).astype(np.float32)
    C = host(lsk.gram(dev(A), prec="bf16")).astype(np.float64)
    lsk.context().sync()
    A64 = A.astype(np.float64)
    ref = ogr.gram_dense(A64)
    absg = np.abs(A64).T @ np.abs(A64)
    assert np.all(np.abs(C - ref) <= (2.0**-16 + 3 * 1024 * U32) * absg + 1e-30)
    assert rel_fro(C, ref) <= 1e-5
    assert np.array_equal(C, C.T)


def test_gram_bf16_alpha_beta_and_empty(lsk):
    A = workloads.dense_normal(3000, 96, seed=4)
    C0 = workloads.dense_normal(96, 96, seed=5)
    Ct = dev(C0.copy())
    lsk.gram(dev(A), alpha=0.25, beta=3.0, C=Ct, prec="bf16")
    lsk.context().sync()
    ref = ogr.gram_dense(A.astype(np.float64), 0.25, 3.0, C0.astype(np.float64))
    assert rel_fro(host(Ct).astype(np.float64), ref) <= 1e-5
    import torch
    E = torch.zeros((0, 16), dtype=torch.float32, device="cuda")
    Ce = dev(C0[:16, :16].copy())
    lsk.gram(E, alpha=1.0, beta=2.0, C=Ce, prec="bf16")       # no rows: C <- beta C
    lsk.context().sync()
    assert np.allclose(host(Ce), 2.0 * C0[:16, :16], rtol=1e-6, atol=0)


@pytest.mark.parametrize("n,d,p", [(200_000, 200, 0.01), (30_000, 256, 0.05), (4000, 20, 0.5)])
def test_gram_csr(lsk, n, d, p):
    V, J, I = workloads.csr_bernoulli(n, d, p, seed=d)
    C = host(lsk.gram(csr_dev(lsk, V, J, I, d))).astype(np.float64)
    ref = ogr.gram_csr(V, J, I, d)
    assert rel_fro(C, ref) <= 1e-5


# ----------------------------------------------------- row norms of A * B ---
RN_CASES = [(20_011, 50, 50, True), (10_000, 256, 256, True), (3_333, 130, 17, False), (500, 1, 1, False),
            (70_000, 64, 64, True), (1_000, 256, 160, False), (2_000, 256, 256, False), (129, 200, 200, True)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("n,d,c,tri", RN_CASES)
def test_rownorms_dense(lsk, n, d, c, tri, prec):
    A = workloads.dense_normal(n, d, seed=c) * (10.0 ** np.linspace(-2, 2, d)).astype(np.float32)
    B = workloads.dense_normal(d, c, seed=d + 1)
    if tri:
        B = np.triu(B)
    x = host(lsk.rownorms_prod(dev(A), dev(B), upper_triangular=tri, prec=prec)).astype(np.float64)
    lsk.context().sync()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = orn.rownorms_prod_dense(A64, B64)
    y = A64 @ B64
    absy = np.abs(A64) @ np.abs(B64)
    if prec == "fp32":
        E = (d + 2) * U32 * absy                       # FP32 dot products of length d
    else:
        # split-bf16 operands (~2^-17 each, dropped lo*lo ~2^-18) + FP32 sums of 3d terms
        E = (2.0**-15 + 3 * (d + 2) * U32) * absy
    bound = np.sum(2 * np.abs(y) * E + E * E, axis=1) + 2 * U32 * ref * c
    assert np.all(np.abs(x - ref) <= bound)
    assert np.max(np.abs(x - ref) / ref) <= (1e-5 if prec == "fp32" else 1e-3)


@pytest.mark.parametrize("n,d,c,tri", [RN_CASES[0], RN_CASES[1], RN_CASES[5], RN_CASES[7]])
def test_rownorms_dense_bf16_single_cta_form(lsk, monkeypatch, n, d, c, tri):
    """Both tensor-core forms on the same inputs: the single-CTA kernel
    (forced) and the default choice (the CTA-pair kernel where B is large,
    e.g. d = c = 256).  Both split and sum identically, so they agree to the
    FP32 accumulation order."""
    A = workloads.dense_normal(n, d, seed=c) * (10.0 ** np.linspace(-2, 2, d)).astype(np.float32)
    B = workloads.dense_normal(d, c, seed=d + 1)
    if tri:
        B = np.triu(B)
    pair = host(lsk.rownorms_prod(dev(A), dev(B), upper_triangular=tri, prec="bf16")).astype(np.float64)
    monkeypatch.setenv("LSK_ROWNORM_SINGLE_CTA", "1")
    single = host(lsk.rownorms_prod(dev(A), dev(B), upper_triangular=tri, prec="bf16")).astype(np.float64)
    lsk.context().sync()
    ref = orn.rownorms_prod_dense(A.astype(np.float64), B.astype(np.float64))
    assert np.max(np.abs(single - ref) / ref) <= 1e-3
    assert np.max(np.abs(single - pair) / ref) <= 1e-5


@pytest.mark.parametrize("n,d,c,tri,ld", [(10_000, 256, 256, True, 256), (2_000, 256, 256, False, 256),
                                            (1_000, 256, 160, False, 256), (5_003, 200, 200, True, 200),
                                            (300, 232, 232, True, 236), (70_001, 256, 256, True, 260)])
def test_rownorms_dense_bf16_tma_form(lsk, monkeypatch, n, d, c, tri, ld):
    """The CTA-pair kernel in its two feeds: register-staged loads (default)
    and the TMA stage ring with in-place hi / lo split (LSK_ROWNORM_TMA=1).
    Both split and multiply identically, so the scores agree bit for bit;
    ragged row tails, K-chunks past d (zero-filled by the copy) and row
    strides above d included."""
    W = workloads.dense_normal(n, ld, seed=c) * (10.0 ** np.linspace(-2, 2, ld)).astype(np.float32)
    B = workloads.dense_normal(d, c, seed=d + 1)
    if tri:
        B = np.triu(B)
    Ad = dev(W)[:, :d]
    regs = host(lsk.rownorms_prod(Ad, dev(B), upper_triangular=tri, prec="bf16")).astype(np.float64)
    monkeypatch.setenv("LSK_ROWNORM_TMA", "1")
    tma = host(lsk.rownorms_prod(Ad, dev(B), upper_triangular=tri, prec="bf16")).astype(np.float64)
    lsk.context().sync()
    A64 = W[:, :d].astype(np.float64)
    ref = orn.rownorms_prod_dense(A64, B.astype(np.float64))
    assert np.max(np.abs(tma - ref) / ref) <= 1e-3
    assert np.array_equal(tma, regs)


TF32_CASES = [(10_000, 256, 256, True, 256), (2_000, 256, 256, False, 256), (1_000, 256, 160, False, 256),
              (5_003, 200, 200, True, 200), (300, 232, 232, True, 236), (70_001, 256, 256, True, 260),
              (20_011, 52, 52, True, 52), (4_096, 32, 32, True, 32), (777, 96, 40, False, 100)]


@pytest.mark.parametrize("n,d,c,tri,ld", TF32_CASES)
def test_rownorms_dense_tf32(lsk, n, d, c, tri, ld):
    """The one-product TF32 kernel (checked by its profile name): A and B each
    rounded to the nearest TF32 (11 significant bits, relative error <= 2^-11
    an entry), products exact in FP32, FP32 sums of d products and of the c
    squares.  Ragged row tails, K-chunks past d (zero-filled by the copy),
    row strides above d and general B included.  Rounding to nearest leaves
    no systematic bias (dropping the low mantissa bits instead shrinks the
    scores by ~1.4e-3 here)."""
    W = workloads.dense_normal(n, ld, seed=c) * (10.0 ** np.linspace(-2, 2, ld)).astype(np.float32)
    B = workloads.dense_normal(d, c, seed=d + 1)
    if tri:
        B = np.triu(B)
    ctx = lsk.context()
    ctx.profile(True)
    ctx.profile_reset()
    x = host(lsk.rownorms_prod(dev(W)[:, :d], dev(B), upper_triangular=tri, prec="tf32")).astype(np.float64)
    ctx.sync()
    names = set(ctx.profile_totals())
    ctx.profile(False)
    assert "rownorm_dense_tf32" in names
    A64, B64 = W[:, :d].astype(np.float64), B.astype(np.float64)
    ref = orn.rownorms_prod_dense(A64, B64)
    y = A64 @ B64
    absy = np.abs(A64) @ np.abs(B64)
    E = (2.0**-10 + 2.0**-21 + 2.05 * (d + 2) * U32) * absy
    bound = np.sum(2 * np.abs(y) * E + E * E, axis=1) + 2 * U32 * ref * c
    assert np.all(np.abs(x - ref) <= bound)
    # no systematic bias: the summed scores within 6e-4 (B's own rounding, fixed
    # for all rows, leaves up to ~2.5e-4 at d = 32; truncation gives >= 1.2e-3)
    assert abs(x.sum() - ref.sum()) <= 6e-4 * ref.sum()


def test_rownorms_tf32_rounds_to_nearest(lsk):
    """Entries 1 + 3 2^-12 (13 low bits 0x1800) with B = I: the nearest TF32
    is 1 + 2^-10, the truncated one 1; the scores are 32 (1 + 2^-10)^2."""
    for sign in (1.0, -1.0):
        A = np.full((512, 32), sign * (1.0 + 3.0 * 2.0**-12), dtype=np.float32)
        x = host(lsk.rownorms_prod(dev(A), dev(np.eye(32, dtype=np.float32)), upper_triangular=True,
                                   prec="tf32")).astype(np.float64)
        want = 32.0 * (1.0 + 2.0**-10) ** 2
        assert np.all(np.abs(x - want) <= 1e-6 * want)


def test_rownorms_alpha_beta(lsk):
    A = workloads.dense_normal(1000, 20, seed=1)
    B = workloads.dense_normal(20, 7, seed=2)
    x0 = workloads.dense_normal(1000, 1, seed=3)[:, 0]
    xt = dev(x0.copy())
    lsk.rownorms_prod(dev(A), dev(B), alpha=2.0, beta=-0.5, x=xt)
    ref = orn.rownorms_prod_dense(A, B, 2.0, -0.5, x0)
    assert np.max(np.abs(host(xt) - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,d,p,c", [(100_000, 200, 0.01, 200), (20_000, 256, 0.05, 256), (3000, 40, 0.3, 9)])
def test_rownorms_csr(lsk, n, d, p, c):
    V, J, I = workloads.csr_bernoulli(n, d, p, seed=c)
    B = workloads.dense_normal(d, c, seed=5)
    x = host(lsk.rownorms_prod(csr_dev(lsk, V, J, I, d), dev(B))).astype(np.float64)
    ref = orn.rownorms_prod_csr_alg8(V, J, I, n, B)
    nz = ref > 0
    assert np.all(x[~nz] == 0)
    assert np.max(np.abs(x[nz] - ref[nz]) / ref[nz]) <= 1e-5


# ---------------------------------------------------------------- R, R^-1 --
@pytest.mark.parametrize("k,d", [(100, 50), (512, 256), (40, 37), (300, 1)])
def test_sketch_qr(lsk, k, d):
    B = workloads.dense_normal(k, d, seed=k) * (10.0 ** np.linspace(-3, 3, d)).astype(np.float32)
    R, Ri = lsk.sketch_qr(dev(B))
    R, Ri = host(R), host(Ri)
    Ro = oqr.qr_r(B.astype(np.float64))
    colnorm = np.linalg.norm(B.astype(np.float64), axis=0)
    assert np.all(np.abs(R - Ro) <= 1e-9 * colnorm[None, :])
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    Rio = oqr.upper_triangular_inverse(Ro)
    assert np.all(np.abs(Ri - Rio) <= 1e-8 * np.abs(Rio).max(axis=0)[None, :] + 1e-300)


def test_sketch_qr_rank_deficient(lsk):
    B = workloads.dense_normal(64, 8, seed=1)
    B[:, 5] = B[:, 2]
    ctx = lsk.context()
    lsk.sketch_qr(dev(B))
    with pytest.raises(lsk.LskError) as ei:
        ctx.sync()
    assert ei.value.name == "RANK_DEFICIENT"


# ---------------------------------------------------------- leverage scores -
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_leverage_dense_outliers_20000x50(lsk, prec):
    A = workloads.dense_outliers().astype(np.float32)          # the FP32 path casts once
    ell, R = lsk.leverage_scores(dev(A), 2500, 100, 0, prec, return_R=True)
    lsk.context().sync()
    ell = host(ell).astype(np.float64)
    ref, Ro = olev.leverage_scores_dense(A.astype(np.float64), 2500, 100, 0,
                                         oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32)
    assert np.max(np.abs(ell - ref) / ref) <= 1e-3
    assert set(np.argsort(-ell)[:5]) == set(range(5))
    colnorm = np.linalg.norm(Ro, axis=0)
    assert np.all(np.abs(host(R) - Ro) <= 1e-4 * colnorm[None, :])


def test_leverage_dense_tf32(lsk):
    """Config 3's mixed recipe at a smaller size: the BF16 Gaussian stage and
    the TF32 row norms (checked by profile name), against the oracle's
    estimates on the same seeds (G rounded to bfloat16 as in the BF16 mode)."""
    n, d, r, k = 200_000, 64, 8192, 256
    A = workloads.dense_normal(n, d, seed=11) * (10.0 ** np.linspace(-3, 3, d)).astype(np.float32)
    ctx = lsk.context()
    ctx.profile(True)
    ctx.profile_reset()
    ell, R = lsk.leverage_scores(dev(A), r, k, 5, "tf32", return_R=True)
    ctx.sync()
    names = set(ctx.profile_totals())
    ctx.profile(False)
    assert "rownorm_dense_tf32" in names and "rownorm_dense_tc" not in names
    ell = host(ell).astype(np.float64)
    ref, Ro = olev.leverage_scores_dense(A.astype(np.float64), r, k, 5, oga.PREC_BF16)
    assert np.max(np.abs(ell - ref) / ref) <= 1e-3
    colnorm = np.linalg.norm(Ro, axis=0)
    assert np.all(np.abs(host(R) - Ro) <= 1e-4 * colnorm[None, :])


def test_leverage_countsketch_only_k0(lsk):
    A = workloads.dense_normal(30_000, 20, seed=7)
    ell = lsk.leverage_scores(dev(A), 2000, 0, 3)
    lsk.context().sync()
    ell = host(ell).astype(np.float64)
    ref, _ = olev.leverage_scores_dense(A.astype(np.float64), 2000, 0, 3)
    assert np.max(np.abs(ell - ref) / ref) <= 1e-3


def test_leverage_csr(lsk):
    n, d = 200_000, 100
    V, J, I = workloads.csr_bernoulli(n, d, 0.02, seed=2)
    ell = lsk.leverage_scores(csr_dev(lsk, V, J, I, d), 10_000, 200, 1, "fp32")
    lsk.context().sync()
    ell = host(ell).astype(np.float64)
    ref, _ = olev.leverage_scores_csr(V, J, I, n, d, 10_000, 200, 1)
    nz = ref > 0
    assert np.all(ell[~nz] == 0)          # empty rows score zero
    assert np.max(np.abs(ell[nz] - ref[nz]) / ref[nz]) <= 1e-3


# ------------------------------------------ Alg. 15 with the right JL Pi -
@pytest.mark.parametrize("prec,m", [("fp32", 64), ("bf16", 64), ("bf16", 200), ("fp32", 1), ("bf16", 300)])
def test_leverage_jl_dense(lsk, prec, m):
    """||A_i R^-1 Pi||^2 against the oracle on the same seeds: the tensor-core
    row norms for m <= 256 (a ragged m = 200 tile), the SIMT path for m = 300
    and FP32, and the single-column m = 1."""
    A = workloads.dense_outliers().astype(np.float32)
    op = oga.PREC_BF16 if prec == "bf16" else oga.PREC_FP32
    ell, R = lsk.leverage_scores_jl(dev(A), 2500, 100, m, 4, prec, return_R=True)
    lsk.context().sync()
    ell = host(ell).astype(np.float64)
    ref, Ro = olev.leverage_scores_jl_dense(A.astype(np.float64), 2500, 100, m, 4, op)
    if m >= 16:
        assert np.max(np.abs(ell - ref) / ref) <= 1e-3
    else:
        # few columns: a score (A_i x)^2 can cancel to ~0, so the error is
        # measured against its expectation ||A_i R^-1||^2 (same sketch and R)
        expect, _ = olev.leverage_scores_dense(A.astype(np.float64), 2500, 100, 4, op)
        assert np.max(np.abs(ell - ref) / expect) <= 1e-3
    colnorm = np.linalg.norm(Ro, axis=0)
    assert np.all(np.abs(host(R) - Ro) <= 1e-4 * colnorm[None, :])


def test_leverage_jl_csr(lsk):
    n, d, m = 200_000, 100, 48
    V, J, I = workloads.csr_bernoulli(n, d, 0.02, seed=2)
    ell = lsk.leverage_scores_jl(csr_dev(lsk, V, J, I, d), 10_000, 200, m, 1, "fp32")
    lsk.context().sync()
    ell = host(ell).astype(np.float64)
    ref, _ = olev.leverage_scores_jl_csr(V, J, I, n, d, 10_000, 200, m, 1)
    nz = ref > 0
    assert np.all(ell[~nz] == 0)
    assert np.max(np.abs(ell[nz] - ref[nz]) / ref[nz]) <= 1e-3


def test_leverage_jl_edges(lsk):
    A = workloads.dense_normal(3000, 16, seed=5)
    with pytest.raises(RuntimeError):
        lsk.leverage_scores_jl(dev(A), 500, 64, 0, 1)
    with pytest.raises(RuntimeError):
        lsk.leverage_scores_jl(dev(A), 500, 64, 4097, 1)
    # an empty A has rank 0 < d: no scores, and the deferred rank-deficiency status
    e = torch.zeros((0, 16), dtype=torch.float32, device="cuda")
    assert lsk.leverage_scores_jl(e, 500, 64, 8, 1).numel() == 0
    with pytest.raises(lsk.LskError, match="RANK_DEFICIENT"):
        lsk.context().sync()
    # a larger m concentrates the estimate on ||A_i R^-1||^2 (relative spread sqrt(2/m))
    full = host(lsk.leverage_scores(dev(A), 500, 64, 1)).astype(np.float64)
    jl = host(lsk.leverage_scores_jl(dev(A), 500, 64, 4096, 1)).astype(np.float64)
    lsk.context().sync()
    assert np.max(np.abs(jl / full - 1)) <= 8 * np.sqrt(2 / 4096)


# ------------------------------------------------------------ least squares -
@pytest.mark.parametrize("kind", ["dense", "csr"])
def test_sketch_precondition_lsq(lsk, kind):
    n, d = 50_000, 32
    if kind == "dense":
        A = workloads.dense_normal(n, d, seed=9) * (10.0 ** np.linspace(-2, 2, d)).astype(np.float32)
        A64 = A.astype(np.float64)
        mv, rmv = (lambda v: A64 @ v), (lambda u: A64.T @ u)
        Ad = dev(A)
    else:
        V, J, I = workloads.csr_bernoulli(n, d, 0.2, seed=9)
        rows = np.repeat(np.arange(n), np.diff(I))
        def mv(v):
            return np.bincount(rows, weights=V.astype(np.float64) * v[J], minlength=n)
        def rmv(u):
            return np.bincount(J, weights=V.astype(np.float64) * u[rows], minlength=d)
        Ad = csr_dev(lsk, V, J, I, d)
    xs, b = workloads.lsq_rhs(n, d, mv, seed=4)
    x, info = lsk.sketch_precondition_lsq(Ad, dev(b), r=d * d, k=2 * d, seed=5)
    x = host(x)
    eta = olsq.normal_equation_residual(mv, rmv, b, x)
    assert eta <= 1e-10, (eta, info)
    assert info["status"] == 0 and info["eta"] <= 1e-10
    assert np.linalg.norm(x - xs) <= 1e-3 * np.linalg.norm(xs)


# ------------------------------------------------------- failure detection -
def test_bounded_wait_gives_up_and_context_stays_usable(lsk):
    """A device wait on a barrier that nothing arrives on ends after its limit
    with the TIMEOUT status (no trap, no hang); the same context then runs a
    leverage-score call normally."""
    import time
    ctx = lsk.context()
    t0 = time.perf_counter()
    lsk.debug_wait_timeout(20_000, ctx=ctx)          # 20 ms
    with pytest.raises(lsk.LskError) as ei:
        ctx.sync()
    assert ei.value.name == "TIMEOUT"
    assert time.perf_counter() - t0 < 5.0
    A = workloads.dense_normal(4000, 16, seed=5)
    ell = lsk.leverage_scores(dev(A), 256, 32, 1, "bf16")
    ctx.sync()
    ref, _ = olev.leverage_scores_dense(A.astype(np.float64), 256, 32, 1, oga.PREC_BF16)
    assert np.max(np.abs(host(ell) - ref) / ref) <= 1e-3


@pytest.mark.parametrize("kind", ["dense", "csr"])
def test_sketch_precondition_lsq_large_residual(lsk, kind):
    """b with no component to speak of in range(A) (pure noise): the residual
    is large and nearly orthogonal to range(A); eta still reaches 1e-10 and x
    matches the Householder least-squares solution."""
    n, d = 200_000, 48
    rng = np.random.default_rng(21)
    if kind == "dense":
        A = workloads.dense_normal(n, d, seed=22) * (10.0 ** np.linspace(0, 2, d)).astype(np.float32)
        A64 = A.astype(np.float64)
        Ad = dev(A)
    else:
        V, J, I = workloads.csr_bernoulli(n, d, 0.1, seed=22)
        rows = np.repeat(np.arange(n), np.diff(I))
        A64 = np.zeros((n, d))
        A64[rows, J] = V
        Ad = csr_dev(lsk, V, J, I, d)
    b = rng.standard_normal(n)
    x, info = lsk.sketch_precondition_lsq(Ad, dev(b), r=d * d, k=2 * d, seed=3)
    lsk.context().sync()
    assert info["status"] == 0 and info["eta"] <= 1e-10
    x_ls = olsq.least_squares_qr(A64, b)
    x = host(x)
    assert np.linalg.norm(x - x_ls) <= 1e-8 * np.linalg.norm(x_ls)


@pytest.mark.parametrize("n,d", [(50_000, 256), (7_000, 36)])
def test_gram_default_runs_on_the_tensor_cores(lsk, n, d):
    """lsk_gram on dense A with d <= 256 takes the BF16x3 tensor-core kernel
    (within the 1e-5 relative bound); CSR A keeps the FP32 path."""
    A = workloads.dense_normal(n, d, seed=d + 1) * (10.0 ** np.linspace(-2, 2, d)).astype(np.float32)
    ctx = lsk.context()
    ctx.sync()
    ctx.profile(True)
    ctx.profile_reset()
    try:
        C = host(lsk.gram(dev(A), prec=None)).astype(np.float64)
        ctx.sync()
        names = set(ctx.profile_totals())
    finally:
        ctx.profile(False)
    assert "gram_tc" in names and "gram_dense" not in names
    assert rel_fro(C, ogr.gram_dense(A.astype(np.float64))) <= 1e-5
    V, J, I = workloads.csr_bernoulli(20_000, 40, 0.05, seed=2)
    Cc = host(lsk.gram(csr_dev(lsk, V, J, I, 40), prec=None)).astype(np.float64)
    assert rel_fro(Cc, ogr.gram_csr(V, J, I, 40)) <= 1e-6
