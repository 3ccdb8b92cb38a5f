"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the bench and the oracle's callers.  It
holds none of the method's arithmetic (no hashing, sketching, factoring or
norms): only numpy random draws with fixed seeds, in the shapes, value
distributions and sparsity patterns of the five workloads below.  The paper
(Sec. 6, Table 2) uses synthetic tall dense and 5%-sparse matrices and ships
none of them; these stand in for them.

  dense_outliers   20,000 x 50 float64, iid N(0,1), rows 0..4 scaled x100
  csr_bernoulli    1,000,000 x 200 CSR float32, each entry kept with p=0.01,
                   values N(0,1), sorted column indices, int64 rowptr
  dense_colscaled  4,000,000 x 256 float32, N(0,1) times 10^u_j, u_j ~ U(-3,3)
  batch_specs      512 problems: n = floor(10^U(4,6)), d in {32,64,128,256},
                   first half dense N(0,1), second half CSR, density
                   U(0.005, 0.05); r = d^2, k = 2d
  lsq_rhs          x* ~ N(0,1), b = A x* + 1e-6 N(0,1) (float64)
  poisson_arrivals exponential inter-arrival gaps at a given rate
"""
import numpy as np


def _rng(seed, stream=0):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def dense_outliers(n=20_000, d=50, n_outliers=5, scale=100.0, seed=0):
    """Dense float64 A with iid N(0,1) entries and rows 0..n_outliers-1 scaled."""
    A = _rng(seed).standard_normal((n, d))
    A[:n_outliers] *= scale
    return A


def csr_bernoulli(n=1_000_000, d=200, p=0.01, seed=1, chunk=65536):
    """CSR (V float32, J int32, I int64): entry (i, j) kept with probability p."""
    rng = _rng(seed)
    Vs, Js, counts = [], [], []
    for i0 in range(0, n, chunk):
        m = min(chunk, n - i0)
        mask = rng.random((m, d), dtype=np.float32) < p
        rows, cols = np.nonzero(mask)
        counts.append(np.bincount(rows, minlength=m))
        Js.append(cols.astype(np.int32))
        Vs.append(rng.standard_normal(len(cols), dtype=np.float32))
    I = np.zeros(n + 1, dtype=np.int64)
    I[1:] = np.cumsum(np.concatenate(counts)) if counts else 0
    V = np.concatenate(Vs) if Vs else np.zeros(0, np.float32)
    J = np.concatenate(Js) if Js else np.zeros(0, np.int32)
    return V, J, I


def column_scales(d, seed=2, lo=-3.0, hi=3.0):
    return 10.0 ** _rng(seed, 1).uniform(lo, hi, size=d)


def dense_colscaled(n=4_000_000, d=256, seed=2, out=None, chunk=1 << 18):
    """float32 A[i, j] = z_ij * 10^u_j, z ~ N(0,1), u_j ~ U(-3, 3).

    ``out`` may be a preallocated float32 (n, d) array (e.g. pinned memory).
    """
    scale = column_scales(d, seed).astype(np.float32)
    rng = _rng(seed)
    A = np.empty((n, d), dtype=np.float32) if out is None else out
    for i0 in range(0, n, chunk):
        m = min(chunk, n - i0)
        z = rng.standard_normal((m, d), dtype=np.float32)
        np.multiply(z, scale[None, :], out=A[i0:i0 + m])
    return A


def dense_normal(n, d, seed, dtype=np.float32):
    return _rng(seed).standard_normal((n, d), dtype=dtype)


def integer_dense(n, d, seed, lo=-8, hi=8, dtype=np.float32):
    """Small-integer-valued dense A (every float32 partial sum exact)."""
    return _rng(seed).integers(lo, hi + 1, size=(n, d)).astype(dtype)


def integer_csr(n, d, p, seed, lo=-8, hi=8):
    V, J, I = csr_bernoulli(n, d, p, seed)
    V = _rng(seed, 7).integers(lo, hi + 1, size=len(V)).astype(np.float32)
    V[V == 0] = 1.0
    return V, J, I


def batch_specs(count=512, seed=3):
    """Per-problem (n, d, kind, density, r, k, data_seed, sketch_seed)."""
    rng = _rng(seed)
    n = np.floor(10.0 ** rng.uniform(4.0, 6.0, size=count)).astype(np.int64)
    d = rng.choice(np.array([32, 64, 128, 256]), size=count)
    density = rng.uniform(0.005, 0.05, size=count)
    specs = []
    for p in range(count):
        kind = "dense" if p < count // 2 else "csr"
        dp = int(d[p])
        specs.append(dict(index=p, n=int(n[p]), d=dp, kind=kind,
                          density=float(density[p]) if kind == "csr" else 1.0,
                          r=dp * dp, k=2 * dp, data_seed=seed * 100003 + p,
                          sketch_seed=seed * (1 << 32) + p))
    return specs


def batch_problem(spec):
    """Materialise one problem of :func:`batch_specs` (dense array or CSR)."""
    if spec["kind"] == "dense":
        return dense_normal(spec["n"], spec["d"], spec["data_seed"])
    return csr_bernoulli(spec["n"], spec["d"], spec["density"], spec["data_seed"])


def lsq_rhs(n, d, matvec64, seed, noise=1e-6):
    """(x*, b): x* ~ N(0,1)^d, b = A x* + noise * N(0,1)^n in float64.

    ``matvec64(x)`` must return A x in float64 for the caller's A.
    """
    rng = _rng(seed, 11)
    xs = rng.standard_normal(d)
    b = matvec64(xs) + noise * rng.standard_normal(n)
    return xs, b


def poisson_arrivals(rate=200.0, count=2000, seed=4):
    """Arrival times (s) of a Poisson process with the given mean rate."""
    gaps = _rng(seed, 13).exponential(1.0 / rate, size=count)
    return np.cumsum(gaps)


def batch_problem_torch(spec, device="cuda"):
    """One problem of :func:`batch_specs` drawn on the device (seeded torch
    generator; same shapes and distributions as :func:`batch_problem`, not the
    same numbers).  Dense: float32 tensor; CSR: (V, J, I) tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(spec["data_seed"]))
    n, d = spec["n"], spec["d"]
    if spec["kind"] == "dense":
        return torch.randn((n, d), generator=g, device=device, dtype=torch.float32)
    mask = torch.rand((n, d), generator=g, device=device) < spec["density"]
    rows, cols = torch.nonzero(mask, as_tuple=True)     # row-major: columns ascending per row
    del mask
    counts = torch.bincount(rows, minlength=n)
    I = torch.zeros(n + 1, dtype=torch.int64, device=device)
    I[1:] = torch.cumsum(counts, 0)
    V = torch.randn(rows.numel(), generator=g, device=device, dtype=torch.float32)
    return V, cols.to(torch.int32), I


def lsq_rhs_torch(A_mv, n, d, seed, noise=1e-6, device="cuda"):
    """(x*, b) on the device: x* ~ N(0,1)^d, b = A x* + noise N(0,1)^n (float64)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    xs = torch.randn(d, generator=g, device=device, dtype=torch.float64)
    b = A_mv(xs) + noise * torch.randn(n, generator=g, device=device, dtype=torch.float64)
    return xs, b
