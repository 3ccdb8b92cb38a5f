"""lsk_cs_sketch_noalloc: the CountSketch entry point for callers that cannot
let a library allocate device memory (their pool allocator owns HBM, or they
cannot afford cudaMalloc's synchronisation).  It runs the CountSketch kernels
with scratch in a fixed device array instead of a context workspace.

Checked through the C ABI against the context entry point lsk_cs_sketch,
within the same tolerances as the CountSketch parity tests, on calls in a
row with different sizes (the shared scratch keeps the previous call's
contents), and its size limits are rejected before anything is launched.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from oracle import countsketch as ocs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lsk():
    from paper_2203_02798_gb300 import build
    build.build()
    import paper_2203_02798_gb300 as p
    lib = p.load_library()
    fn = lib.lsk_cs_sketch_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(p._Mat), ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    return p


def noalloc(lsk, A, r, seed):
    m, n, d = lsk._mat(A)
    out = torch.full((r, d), float("nan"), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lsk.load_library().lsk_cs_sketch_noalloc(ctypes.byref(m), r, seed, ctypes.c_void_p(out.data_ptr()),
                                                  stream)
    torch.cuda.synchronize()
    return rc, out


def dense(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def within_tolerance(got, ref, absref, m):
    nb = np.linalg.norm(ref)
    assert np.linalg.norm(got - ref) <= 1e-5 * nb
    assert np.all(np.abs(got - ref) <= 2 * m * U32 * absref + 1e-30)


def test_noalloc_matches_context_entry_point_on_consecutive_calls(lsk):
    # call 1: dense, large r; call 2: CSR, smaller r; call 3: dense again
    n1, d1, r1, s1 = 300_000, 256, 65_536, 5
    A1 = workloads.dense_normal(n1, d1, seed=1)
    rc, got1 = noalloc(lsk, dense(A1), r1, s1)
    assert rc == 0
    ref1 = lsk.cs_sketch(dense(A1), r1, s1)
    lsk.context().sync()
    b1, g1 = ocs.countsketch_hash(n1, r1, s1)
    absref1 = ocs.countsketch_apply_dense(np.abs(A1), b1, np.ones_like(g1), r1)
    within_tolerance(got1.cpu().numpy().astype(np.float64), ref1.cpu().numpy().astype(np.float64), absref1,
                     np.bincount(b1, minlength=r1).max())

    n2, d2, r2, s2 = 200_000, 200, 8_000, 6
    V, J, I = workloads.csr_bernoulli(n2, d2, 0.01, seed=2)
    A2 = lsk.csr_from_numpy(V, J, I, d2)
    rc, got2 = noalloc(lsk, A2, r2, s2)
    assert rc == 0
    ref2 = lsk.cs_sketch(A2, r2, s2)
    lsk.context().sync()
    b2, g2 = ocs.countsketch_hash(n2, r2, s2)
    absref2 = ocs.countsketch_apply_csr(np.abs(V), J, I, n2, d2, b2, np.ones_like(g2), r2)
    m2 = np.bincount(b2, minlength=r2).max()
    within_tolerance(got2.cpu().numpy().astype(np.float64), ref2.cpu().numpy().astype(np.float64), absref2, m2)

    A3 = workloads.integer_dense(50_000, 64, seed=3)      # integer data: both exact, bit-identical
    rc, got3 = noalloc(lsk, dense(A3), 4096, 7)
    assert rc == 0
    ref3 = lsk.cs_sketch(dense(A3), 4096, 7)
    lsk.context().sync()
    assert torch.equal(got3, ref3)


def test_noalloc_second_call_leaves_free_memory_unchanged(lsk):
    """The first call on a device places the scratch array there (lazy module
    loading); every later call must take no device memory at all."""
    A = dense(workloads.dense_normal(100_000, 128, seed=4))
    rc, _ = noalloc(lsk, A, 16_384, 3)                 # warm-up: set-up happens here
    assert rc == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out = torch.empty((16_384, 128), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()               # after torch's own allocation for the output
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    m, _, _ = lsk._mat(A)
    for seed in (4, 5):
        rc = lsk.load_library().lsk_cs_sketch_noalloc(ctypes.byref(m), 16_384, seed,
                                                      ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1, (free0, free1, free2)


def test_noalloc_rejects_sizes_beyond_its_capacity(lsk):
    lib = lsk.load_library()
    too_many_rows = torch.zeros((lsk_max_rows(lib) + 1, 1), dtype=torch.float32, device="cuda")
    rc, out = noalloc(lsk, too_many_rows, 8, 1)
    assert rc == -3                                    # LSK_ERR_UNSUPPORTED
    assert torch.isnan(out).all()                      # nothing was launched
    small = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    m, _, _ = lsk._mat(small)
    rc = lib.lsk_cs_sketch_noalloc(ctypes.byref(m), (1 << 18) + 1, 1, ctypes.c_void_p(small.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -3


def lsk_max_rows(lib):
    return 1 << 20     # LSK_NOALLOC_MAX_ROWS in include/lsk.h
