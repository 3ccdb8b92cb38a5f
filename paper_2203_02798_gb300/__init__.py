"""Python binding of liblsk.so -- GB300 sketching for tall-and-skinny matrices.

Thin ctypes marshalling over the C ABI in ``include/lsk.h`` (same names,
without the ``lsk_`` prefix).  Every step of every call runs in the CUDA
kernels of liblsk.so; PyTorch only provides device memory and the stream.
There is no CPU fallback: if the library or a CUDA device is missing, the
calls raise.

Matrices are either a 2-D ``torch.float32`` CUDA tensor (dense, row-major,
unit column stride) or a :class:`CSR` of CUDA tensors (V float32, J int32,
I int64, 0-based, sorted/unique column indices per row).

The operations follow Sobczyk & Gallopoulos, "pylspack" (arXiv 2203.02798):
``cs_sketch`` = S*A (Def. 3, Alg. 2); ``gauss_sketch`` = G*(S*A) (Alg. 3);
``gram`` = alpha A^T A + beta C (Alg. 5/7, csrrk); ``rownorms_prod`` =
alpha diag(A B B^T A^T) + beta x (Alg. 8, csrsqn/rmsqn); ``leverage_scores``
(Alg. 15 without Pi); ``sketch_precondition_lsq`` (Alg. 12).
"""
import ctypes
import os
from collections import namedtuple

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblsk.so")

# prec: "fp32" FP32 accuracy; "bf16" tensor cores (bf16 G, split-bf16
# operands); "tf32" the bf16 mode with the row-norm GEMM A B as one TF32
# product (A rounded to the nearest TF32 by the copy engine)
PREC_FP32, PREC_TF32, PREC_BF16 = 0, 1, 2
_PRECS = {"fp32": PREC_FP32, "tf32": PREC_TF32, "bf16": PREC_BF16}

ERRORS = {
    -1: "INVALID_ARG", -2: "BAD_CSR", -3: "UNSUPPORTED", -4: "RANK_DEFICIENT",
    -5: "NOT_CONVERGED", -6: "OOM", -7: "TIMEOUT", -8: "CUDA",
}

CSR = namedtuple("CSR", ["V", "J", "I", "n", "d"])


class LskError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class _Mat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64),
                ("d", ctypes.c_int64), ("ld", ctypes.c_int64), ("values", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("nnz", ctypes.c_int64)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("A", _Mat), ("r", ctypes.c_int64), ("k", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("ell", ctypes.c_void_p)]


BATCH_GRAPH = 0x100
BATCH_AUTOTUNE = 0x200
BATCH_PER_PROBLEM = 0x400


class LsqOpts(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int64), ("k", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("prec", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("max_refine", ctypes.c_int32),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double)]


class LsqInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("refinements", ctypes.c_int32), ("eta", ctypes.c_double),
                ("status", ctypes.c_int32)]


_lib = None
_P, _I32, _I64, _U64, _D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                            ctypes.c_double)
_SIGS = {
    "lsk_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _P]),
    "lsk_destroy": (ctypes.c_int, [_P]),
    "lsk_set_stream": (ctypes.c_int, [_P, _P]),
    "lsk_sync": (ctypes.c_int, [_P]),
    "lsk_error_string": (ctypes.c_char_p, [_P]),
    "lsk_workspace_bytes": (ctypes.c_size_t, [_P]),
    "lsk_reserve": (ctypes.c_int, [_P, ctypes.c_size_t]),
    "lsk_cs_sketch": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _U64, _P]),
    "lsk_gauss_sketch": (ctypes.c_int, [_P, _P, _I64, _I64, _I64, _U64, _I32, _P]),
    "lsk_count_gauss": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _U64, _P]),
    "lsk_set_fused_sketch": (ctypes.c_int, [ctypes.c_int]),
    "lsk_gram": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _D, _D, _P]),
    "lsk_gram_prec": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _D, _D, _I32, _P]),
    "lsk_rownorms_prod": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _P, _I64, _D, _D, _I32, _I32, _P]),
    "lsk_sketch_qr": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P]),
    "lsk_leverage_scores": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _U64, _I32, _P, _P]),
    "lsk_leverage_scores_jl": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _I64, _U64, _I32, _P, _P]),
    "lsk_sketch_rows": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _U64, _I32, _I64, _I32, _P]),
    "lsk_leverage_scores_from_sketch": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _P, _I64, _I32, _P, _P]),
    "lsk_sketch_solve": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _P, _I64, _I64, _U64, _I32, _P]),
    "lsk_csrjlt": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _U64, _I32, _P]),
    "lsk_column_select": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _U64, _I32, _I64, _P]),
    "lsk_leverage_scores_exact": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I32, _P, _P]),
    "lsk_leverage_scores_truncated": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _U64, _I32,
                                                     ctypes.c_double, _P, ctypes.POINTER(ctypes.c_int64)]),
    "lsk_least_squares_gram": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _P, _I32, _P]),
    "lsk_leverage_scores_hrn": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _I64, _I64, _U64, _I32, _I64, _I32, _P, _P]),
    "lsk_lsq_default_opts": (None, [ctypes.POINTER(LsqOpts), _I64]),
    "lsk_sketch_precondition_lsq": (ctypes.c_int, [_P, ctypes.POINTER(_Mat), _P, _P,
                                                   ctypes.POINTER(LsqOpts), ctypes.POINTER(LsqInfo)]),
    "lsk_debug_hash": (ctypes.c_int, [_P, _I64, _I64, _U64, _P, _P]),
    "lsk_debug_gauss": (ctypes.c_int, [_P, _I64, _I64, _U64, _I32, _P]),
    "lsk_debug_wait_timeout": (ctypes.c_int, [_P, _I64]),
    "lsk_batch_leverage_scores": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_BatchItem), _I32, _I32]),
    "lsk_batch_streams": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_BatchItem), _I32]),
    "lsk_batch_schedule": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_BatchItem), _I32, _P]),
    "lsk_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "lsk_profile_reset": (ctypes.c_int, [_P]),
    "lsk_profile_count": (ctypes.c_int, [_P]),
    "lsk_profile_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
}


def load_library(path=LIB_PATH):
    """Load liblsk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2203_02798_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _prec(p):
    return _PRECS[p] if isinstance(p, str) else int(p)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("liblsk works on CUDA tensors (use .cuda())")


class Context:
    """An lsk_ctx bound to one CUDA device; launches on torch's current stream."""

    def __init__(self, device=None):
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("liblsk needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.lsk_create(ctypes.byref(h), self.device.index,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise LskError(rc, "lsk_create failed")
        self.h = h
        self._lib = lib

    def close(self):
        if getattr(self, "h", None):
            self._lib.lsk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        self._lib.lsk_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))
        rc = getattr(self._lib, name)(self.h, *args)
        if rc != 0:
            raise LskError(rc, self._lib.lsk_error_string(self.h).decode())
        return rc

    def sync(self):
        """Synchronise the stream and raise any deferred device error."""
        self._call("lsk_sync")

    def reserve(self, nbytes):
        self._call("lsk_reserve", ctypes.c_size_t(int(nbytes)))

    def workspace_bytes(self):
        return int(self._lib.lsk_workspace_bytes(self.h))

    def profile(self, on=True):
        """Turn per-kernel CUDA-event timing on or off (lsk_profile_enable)."""
        self._lib.lsk_profile_enable(self.h, int(bool(on)))

    def profile_reset(self):
        self._lib.lsk_profile_reset(self.h)

    def profile_totals(self):
        """{kernel name: (launches, total ms)} recorded since the last reset."""
        out = {}
        buf = ctypes.create_string_buffer(128)
        for i in range(self._lib.lsk_profile_count(self.h)):
            n, ms = ctypes.c_longlong(), ctypes.c_double()
            self._lib.lsk_profile_get(self.h, i, buf, 128, ctypes.byref(n), ctypes.byref(ms))
            out[buf.value.decode()] = (int(n.value), float(ms.value))
        return out


_ctx = {}


def context(device=None):
    """The per-device default :class:`Context`."""
    idx = torch.cuda.current_device() if device is None else int(device)
    if idx not in _ctx:
        _ctx[idx] = Context(idx)
    return _ctx[idx]


def _mat(A):
    m = _Mat()
    if isinstance(A, CSR):
        _check_cuda(A.V, A.J, A.I)
        assert A.V.dtype == torch.float32 and A.J.dtype == torch.int32 and A.I.dtype == torch.int64
        m.kind, m.dtype, m.n, m.d, m.ld = 1, 0, int(A.n), int(A.d), 0
        m.values, m.rowptr, m.colidx, m.nnz = A.V.data_ptr(), A.I.data_ptr(), A.J.data_ptr(), A.V.numel()
        return m, int(A.n), int(A.d)
    _check_cuda(A)
    if A.dtype != torch.float32 or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("dense A must be a 2-D float32 tensor with unit column stride")
    m.kind, m.dtype, m.n, m.d, m.ld = 0, 0, A.shape[0], A.shape[1], max(A.stride(0), A.shape[1])
    m.values, m.rowptr, m.colidx, m.nnz = A.data_ptr(), None, None, 0
    return m, A.shape[0], A.shape[1]


def _dev(A):
    return A.V.device if isinstance(A, CSR) else A.device


def cs_sketch(A, r, seed, out=None, ctx=None):
    """lsk_cs_sketch: S*A (r x d, float32)."""
    m, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    SA = out if out is not None else torch.empty((r, d), dtype=torch.float32, device=_dev(A))
    ctx._call("lsk_cs_sketch", ctypes.byref(m), int(r), int(seed), _ptr(SA))
    return SA


def gauss_sketch(SA, k, seed, prec="fp32", out=None, ctx=None):
    """lsk_gauss_sketch: G*SA (k x d, float32), G scaled by 1/sqrt(k)."""
    _check_cuda(SA)
    r, d = SA.shape
    ctx = ctx or context(SA.device.index)
    GSA = out if out is not None else torch.empty((k, d), dtype=torch.float32, device=SA.device)
    ctx._call("lsk_gauss_sketch", _ptr(SA.contiguous()), int(r), int(d), int(k), int(seed), _prec(prec),
              _ptr(GSA))
    return GSA


def count_gauss(A, r, k, seed, out=None, ctx=None):
    """lsk_count_gauss: G*(S*A) (k x d, float32) in one pass over A, S*A kept
    on chip (the BF16 mode of gauss_sketch)."""
    m, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    GSA = out if out is not None else torch.empty((k, d), dtype=torch.float32, device=_dev(A))
    ctx._call("lsk_count_gauss", ctypes.byref(m), int(r), int(k), int(seed), _ptr(GSA))
    return GSA


def set_fused_sketch(mode):
    """lsk_set_fused_sketch: how the BF16 sketch of the leverage-score,
    least-squares and batch calls is formed -- 0 the two stages, 1 the fused
    kernel where the shape favours it (the default), 2 the fused kernel
    wherever it applies (True is 2, False is 0); process-wide.  Returns the
    previous mode."""
    if isinstance(mode, bool):
        mode = 2 if mode else 0
    return int(load_library().lsk_set_fused_sketch(int(mode)))


def gram(A, alpha=1.0, beta=0.0, C=None, prec="fp32", ctx=None):
    """alpha A^T A + beta C (d x d float32, C updated in place if given).
    prec: "fp32" (lsk_gram_prec FP32: CUDA-core FP32), "bf16" or "tf32"
    (lsk_gram_prec BF16: tensor-core products of a bf16 split), None
    (lsk_gram: the tensor cores for dense d <= 256, else FP32)."""
    m, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    if C is None:
        C = torch.empty((d, d), dtype=torch.float32, device=_dev(A))
        beta = 0.0
    if prec is None:
        ctx._call("lsk_gram", ctypes.byref(m), float(alpha), float(beta), _ptr(C))
    else:
        ctx._call("lsk_gram_prec", ctypes.byref(m), float(alpha), float(beta), _prec(prec), _ptr(C))
    return C


def rownorms_prod(A, B, alpha=1.0, beta=0.0, x=None, upper_triangular=False, prec="fp32", ctx=None):
    """lsk_rownorms_prod: alpha ||A_i B||^2 + beta x_i (n float32).  prec:
    "fp32" CUDA cores; "bf16" BF16x3 on the tensor cores; "tf32" one TF32
    product on the tensor cores (dense A with 32 <= d <= 256, rows 16-byte
    aligned, n >= 256; other shapes take the BF16x3 or FP32 form)."""
    m, n, d = _mat(A)
    _check_cuda(B)
    B = B.contiguous()
    ctx = ctx or context(_dev(A).index)
    if x is None:
        x = torch.empty(n, dtype=torch.float32, device=_dev(A))
        beta = 0.0
    ctx._call("lsk_rownorms_prod", ctypes.byref(m), _ptr(B), int(B.shape[1]), float(alpha), float(beta),
              int(bool(upper_triangular)), _prec(prec), _ptr(x))
    return x


def sketch_qr(B, ctx=None):
    """lsk_sketch_qr: (R, R^-1) of the sketch B (float64, d x d)."""
    _check_cuda(B)
    k, d = B.shape
    ctx = ctx or context(B.device.index)
    R = torch.empty((d, d), dtype=torch.float64, device=B.device)
    Ri = torch.empty((d, d), dtype=torch.float64, device=B.device)
    ctx._call("lsk_sketch_qr", _ptr(B.contiguous()), int(k), int(d), _ptr(R), _ptr(Ri))
    return R, Ri


def leverage_scores(A, r, k, seed, prec="fp32", out=None, return_R=False, ctx=None):
    """lsk_leverage_scores: ell_i = ||A_i R^-1||^2 (n float32); optionally R."""
    m, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    ell = out if out is not None else torch.empty(n, dtype=torch.float32, device=_dev(A))
    R = torch.empty((d, d), dtype=torch.float64, device=_dev(A)) if return_R else None
    ctx._call("lsk_leverage_scores", ctypes.byref(m), int(r), int(k), int(seed), _prec(prec), _ptr(ell),
              _ptr(R))
    return (ell, R) if return_R else ell


def sketch_rows(A, r, k, seed, prec="fp32", row0=0, out=None, accumulate=False, ctx=None):
    """lsk_sketch_rows: the partial sketch of a block of rows whose first row
    is row row0 of the whole matrix -- S_g A (r x d) for k == 0, else
    G S_g A (k x d), float32, written to out or (accumulate) added to it.
    Summed over the blocks of a row partition it is the sketch of the whole
    matrix."""
    m, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    rows = int(k) if k > 0 else int(r)
    if accumulate and out is None:
        raise ValueError("accumulate needs out")
    out = out if out is not None else torch.empty((rows, d), dtype=torch.float32, device=_dev(A))
    ctx._call("lsk_sketch_rows", ctypes.byref(m), int(r), int(k), int(seed), _prec(prec), int(row0),
              int(bool(accumulate)), _ptr(out))
    return out


def leverage_scores_host(A_host, r, k, seed, prec="bf16", out_host=None, chunk_rows=1 << 19, A_dev=None,
                         ctx=None):
    """Leverage scores of a dense matrix in pinned host memory, end to end:
    the host-to-device copy of row block c + 1 runs (on a side stream) while
    the CountSketch of block c runs (lsk_sketch_rows, accumulating S A); then
    the Gaussian stage, R and the row norms of the whole matrix on the device,
    and the scores copied back to out_host (pinned, n floats).  Same result
    as leverage_scores on the device copy with the two-stage sketch.  A_dev:
    the device buffer to copy into (allocated if None).  Returns out_host."""
    n, d = A_host.shape
    if not A_host.is_pinned():
        raise ValueError("A_host must be in pinned memory")
    ctx = ctx or context()
    dev = ctx.device   # the context's stream is the device's current stream (as in every call here)
    A = A_dev if A_dev is not None else torch.empty((n, d), dtype=torch.float32, device=dev)
    main = torch.cuda.current_stream(dev)
    copy = _copy_stream(dev)
    SA = torch.empty((r, d), dtype=torch.float32, device=dev)
    blocks = [(c0, min(n, c0 + chunk_rows)) for c0 in range(0, n, chunk_rows)] or [(0, 0)]
    copy.wait_stream(main)
    events = []
    with torch.cuda.stream(copy):
        for c0, c1 in blocks:
            A[c0:c1].copy_(A_host[c0:c1], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(copy)
            events.append(ev)
    for (c0, c1), ev in zip(blocks, events):
        main.wait_event(ev)
        sketch_rows(A[c0:c1], r, 0, seed, prec, row0=c0, out=SA, accumulate=c0 > 0, ctx=ctx)
    sk = SA if k == 0 else gauss_sketch(SA, k, seed, prec, ctx=ctx)
    ell = leverage_scores_from_sketch(A, sk, prec, ctx=ctx)
    if out_host is None:
        out_host = torch.empty(n, dtype=torch.float32, pin_memory=True)
    out_host.copy_(ell, non_blocking=True)
    A.record_stream(copy)
    return out_host


_COPY_STREAMS = {}


def _copy_stream(dev):
    if dev.index not in _COPY_STREAMS:
        _COPY_STREAMS[dev.index] = torch.cuda.Stream(device=dev)
    return _COPY_STREAMS[dev.index]


def leverage_scores_from_sketch(A, sketch, prec="fp32", out=None, return_R=False, ctx=None):
    """lsk_leverage_scores_from_sketch: R of the given sketch (rows x d
    float32), then ell_i = ||A_i R^-1||^2 for the rows of A (n float32);
    optionally R."""
    m, n, d = _mat(A)
    _check_cuda(sketch)
    sketch = sketch.contiguous()
    ctx = ctx or context(_dev(A).index)
    ell = out if out is not None else torch.empty(n, dtype=torch.float32, device=_dev(A))
    R = torch.empty((d, d), dtype=torch.float64, device=_dev(A)) if return_R else None
    ctx._call("lsk_leverage_scores_from_sketch", ctypes.byref(m), _ptr(sketch), int(sketch.shape[0]), _prec(prec),
              _ptr(ell), _ptr(R))
    return (ell, R) if return_R else ell


def leverage_scores_jl(A, r, k, m, seed, prec="fp32", out=None, return_R=False, ctx=None):
    """lsk_leverage_scores_jl: ell_i = ||A_i R^-1 Pi||^2 with the d x m JL
    projection Pi of Alg. 15 (n float32); optionally R."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    ell = out if out is not None else torch.empty(n, dtype=torch.float32, device=_dev(A))
    R = torch.empty((d, d), dtype=torch.float64, device=_dev(A)) if return_R else None
    ctx._call("lsk_leverage_scores_jl", ctypes.byref(mat), int(r), int(k), int(m), int(seed), _prec(prec),
              _ptr(ell), _ptr(R))
    return (ell, R) if return_R else ell


def leverage_scores_exact(A, prec="fp32", out=None, return_R=False, ctx=None):
    """lsk_leverage_scores_exact (Alg. 13): ||A_i R^-1||^2 with R from A^T A."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    theta = out if out is not None else torch.empty(n, dtype=torch.float32, device=_dev(A))
    R = torch.empty((d, d), dtype=torch.float64, device=_dev(A)) if return_R else None
    ctx._call("lsk_leverage_scores_exact", ctypes.byref(mat), _prec(prec), _ptr(theta), _ptr(R))
    return (theta, R) if return_R else theta


def least_squares_gram(A, b, refine=2, out=None, ctx=None):
    """lsk_least_squares_gram (Alg. 10): x from R of A^T A, refined in FP64."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    if b.dtype != torch.float64 or not b.is_contiguous() or b.device != _dev(A):
        raise ValueError("b must be a contiguous float64 tensor on A's device")
    x = out if out is not None else torch.empty(d, dtype=torch.float64, device=_dev(A))
    ctx._call("lsk_least_squares_gram", ctypes.byref(mat), _ptr(b), int(refine), _ptr(x))
    return x


def leverage_scores_truncated(A, r, k, seed, rcond=1e-6, prec="fp32", out=None, ctx=None):
    """lsk_leverage_scores_truncated: Alg. 15 truncated to the sketch's
    numerical rank -> (theta, rank)."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    theta = out if out is not None else torch.empty(n, dtype=torch.float32, device=_dev(A))
    rank = ctypes.c_int64(0)
    ctx._call("lsk_leverage_scores_truncated", ctypes.byref(mat), int(r), int(k), int(seed), _prec(prec),
              float(rcond), _ptr(theta), ctypes.byref(rank))
    return theta, int(rank.value)


def column_select(A, r, k, seed, c, prec="fp32", ctx=None):
    """lsk_column_select (Alg. 9): the c selected columns of A (int32, pivot order)."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    cols = torch.empty(int(c), dtype=torch.int32, device=_dev(A))
    ctx._call("lsk_column_select", ctypes.byref(mat), int(r), int(k), int(seed), _prec(prec), int(c), _ptr(cols))
    return cols


def leverage_scores_hrn(A, r, k, seed, c, exact=True, prec="fp32", out=None, ctx=None):
    """lsk_leverage_scores_hrn: Alg. 14 (exact=True) or Alg. 16 scores on the
    c columns Alg. 9 selects -> (theta, cols)."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    theta = out if out is not None else torch.empty(n, dtype=torch.float32, device=_dev(A))
    cols = torch.empty(int(c), dtype=torch.int32, device=_dev(A))
    ctx._call("lsk_leverage_scores_hrn", ctypes.byref(mat), int(r), int(k), int(seed), _prec(prec), int(c),
              1 if exact else 0, _ptr(theta), _ptr(cols))
    return theta, cols


def csrjlt(A, m, seed, prec="fp32", out=None, ctx=None):
    """lsk_csrjlt (Alg. 4): C = G A for a CSR A (m x d float32)."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    C = out if out is not None else torch.empty((m, d), dtype=torch.float32, device=_dev(A))
    ctx._call("lsk_csrjlt", ctypes.byref(mat), int(m), int(seed), _prec(prec), _ptr(C))
    return C


def sketch_solve(A, b, r, k, seed, prec="fp32", out=None, ctx=None):
    """lsk_sketch_solve (Alg. 11): x = argmin ||G S (A x - b)|| (d float64)."""
    mat, n, d = _mat(A)
    ctx = ctx or context(_dev(A).index)
    if b.dtype != torch.float64 or not b.is_contiguous() or b.device != _dev(A):
        raise ValueError("b must be a contiguous float64 tensor on A's device")
    x = out if out is not None else torch.empty(d, dtype=torch.float64, device=_dev(A))
    ctx._call("lsk_sketch_solve", ctypes.byref(mat), _ptr(b), int(r), int(k), int(seed), _prec(prec), _ptr(x))
    return x


def batch_leverage_scores(problems, prec="bf16", graph=False, autotune=False, streams=0, outs=None,
                          ctx=None, per_problem=False):
    """lsk_batch_leverage_scores: problems = [(A, r, k, seed), ...] -> [ell, ...].

    A is a dense CUDA tensor or a CSR; all problems run in one call: their
    sketches and row norms on concurrent internal streams, the Gaussian stage
    and R^-1 of the BF16 problems with d <= 256 as grouped launches
    (per_problem=True: no grouped stages).  graph=True: captured into a
    cached CUDA graph; autotune=True: the stream count is timed and chosen."""
    n = len(problems)
    items = (_BatchItem * max(n, 1))()
    if outs is None:
        outs = []
        for (A, r, k, seed) in problems:
            m, rows, d = _mat(A)
            outs.append(torch.empty(rows, dtype=torch.float32, device=_dev(A)))
    dev = _dev(problems[0][0]) if n else torch.device("cuda", torch.cuda.current_device())
    for i, ((A, r, k, seed), ell) in enumerate(zip(problems, outs)):
        m, rows, d = _mat(A)
        items[i].A = m
        items[i].r, items[i].k, items[i].seed = int(r), int(k), int(seed)
        items[i].ell = ell.data_ptr()
    ctx = ctx or context(dev.index)
    flags = ((int(streams) & 0xFF) | (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0)
             | (BATCH_PER_PROBLEM if per_problem else 0))
    ctx._call("lsk_batch_leverage_scores", n, items, _prec(prec), flags)
    return outs


def batch_streams(problems, prec="bf16", ctx=None):
    """Stream count the autotuner chose for this batch signature (0 if none)."""
    items = (_BatchItem * max(len(problems), 1))()
    for i, (A, r, k, seed) in enumerate(problems):
        items[i].A = _mat(A)[0]
        items[i].r, items[i].k, items[i].seed = int(r), int(k), int(seed)
    ctx = ctx or context()
    return int(ctx._lib.lsk_batch_streams(ctx.h, len(problems), items, _prec(prec)))


def batch_schedule(problems, prec="bf16", ctx=None):
    """lsk_batch_schedule: (known, {"streams", "waves", "slice", "tiles"}) of
    this batch signature."""
    items = (_BatchItem * max(len(problems), 1))()
    for i, (A, r, k, seed) in enumerate(problems):
        items[i].A = _mat(A)[0]
        items[i].r, items[i].k, items[i].seed = int(r), int(k), int(seed)
    ctx = ctx or context()
    out = (ctypes.c_int32 * 4)()
    known = int(ctx._lib.lsk_batch_schedule(ctx.h, len(problems), items, _prec(prec), out))
    return bool(known), {"streams": out[0], "waves": out[1], "slice": out[2], "tiles": out[3]}


def lsq_default_opts(d):
    o = LsqOpts()
    load_library().lsk_lsq_default_opts(ctypes.byref(o), int(d))
    return o


def sketch_precondition_lsq(A, b, opts=None, ctx=None, **kw):
    """lsk_sketch_precondition_lsq: x (d float64) and an info dict."""
    m, n, d = _mat(A)
    _check_cuda(b)
    ctx = ctx or context(_dev(A).index)
    o = opts if opts is not None else lsq_default_opts(d)
    for key, val in kw.items():
        setattr(o, key, _prec(val) if key == "prec" else val)
    x = torch.empty(d, dtype=torch.float64, device=_dev(A))
    info = LsqInfo()
    ctx._call("lsk_sketch_precondition_lsq", ctypes.byref(m), _ptr(b.contiguous()), _ptr(x),
              ctypes.byref(o), ctypes.byref(info))
    return x, dict(iters=info.iters, refinements=info.refinements, eta=info.eta, status=info.status)


def debug_hash(n, r, seed, device=None, ctx=None):
    """lsk_debug_hash: (bucket int32[n], sign int8[n]) of the CountSketch."""
    ctx = ctx or context(device)
    b = torch.empty(n, dtype=torch.int32, device=ctx.device)
    s = torch.empty(n, dtype=torch.int8, device=ctx.device)
    ctx._call("lsk_debug_hash", int(n), int(r), int(seed), _ptr(b), _ptr(s))
    return b, s


def debug_wait_timeout(limit_us, device=None, ctx=None):
    """lsk_debug_wait_timeout: a bounded device wait that must give up; the
    next ctx.sync() raises LskError TIMEOUT."""
    ctx = ctx or context(device)
    ctx._call("lsk_debug_wait_timeout", int(limit_us))


def debug_gauss(k, r, seed, prec="fp32", device=None, ctx=None):
    """lsk_debug_gauss: G (k x r float32) as used by gauss_sketch."""
    ctx = ctx or context(device)
    G = torch.empty((k, r), dtype=torch.float32, device=ctx.device)
    ctx._call("lsk_debug_gauss", int(k), int(r), int(seed), _prec(prec), _ptr(G))
    return G


def csr_from_numpy(V, J, I, d, device="cuda"):
    """Copy numpy CSR arrays to the device as a :class:`CSR`."""
    import numpy as np
    return CSR(torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).to(device),
               torch.from_numpy(np.ascontiguousarray(J, dtype=np.int32)).to(device),
               torch.from_numpy(np.ascontiguousarray(I, dtype=np.int64)).to(device),
               len(I) - 1, int(d))
