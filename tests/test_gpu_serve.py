"""Served sketch-and-precondition least squares on the GPU: every request of
a mixed trace reaches eta <= 1e-10 (checked by the FP64 oracle on the host),
requests overlap on the device, and a request's solution is the same alone
and in the mix (within the tolerance the solve guarantees)."""
import numpy as np
import pytest
import torch

import workloads
from oracle import lsq as olsq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server():
    from paper_2203_02798_gb300 import build
    build.build()
    from paper_2203_02798_gb300.serve import Server
    s = Server(slots=4)
    yield s
    s.close()


def make_request(lsk, i, rng):
    d = int(rng.choice([16, 32, 64]))
    n = int(10 ** rng.uniform(4.0, 4.7))
    if i % 2 == 0:
        A = workloads.dense_normal(n, d, seed=500 + i)
        A64 = A.astype(np.float64)
        mv, rmv = (lambda v, A64=A64: A64 @ v), (lambda u, A64=A64: A64.T @ u)
        Ad = torch.from_numpy(A).cuda()
    else:
        V, J, I = workloads.csr_bernoulli(n, d, 0.2, seed=500 + i)
        rows = np.repeat(np.arange(n), np.diff(I))
        Vd = V.astype(np.float64)
        def mv(v, rows=rows, Vd=Vd, J=J, n=n):
            return np.bincount(rows, weights=Vd * v[J], minlength=n)
        def rmv(u, rows=rows, Vd=Vd, J=J, d=d):
            return np.bincount(J, weights=Vd * u[rows], minlength=d)
        Ad = lsk.csr_from_numpy(V, J, I, d)
    xs, b = workloads.lsq_rhs(n, d, mv, seed=900 + i)
    return dict(A=Ad, b=torch.from_numpy(b).cuda(), mv=mv, rmv=rmv, b_host=b, n=n, d=d,
                opts=dict(r=d * d, k=2 * d, seed=31 + i))


def test_served_trace_converges_and_overlaps(server):
    import paper_2203_02798_gb300 as lsk
    from paper_2203_02798_gb300.serve import Request, latency_summary
    rng = np.random.default_rng(3)
    payloads = [make_request(lsk, i, rng) for i in range(12)]
    reqs = [Request(i, 0.002 * i, server.footprint(p["n"], p["d"]), p) for i, p in enumerate(payloads)]
    done, rejected = server.run(reqs)
    assert not rejected and len(done) == 12
    assert all(c.error is None for c in done), [c.error for c in done if c.error]
    for c in done:
        p = payloads[c.rid]
        x, info = c.result
        eta = olsq.normal_equation_residual(p["mv"], p["rmv"], p["b_host"], x)
        assert eta <= 1e-10 and info["eta"] <= 1e-10, (c.rid, eta, info)
    by_id = {c.rid: c for c in done}
    assert any(by_id[i + 1].start < by_id[i].finish for i in range(11))   # overlapped
    s = latency_summary(done)
    assert s["count"] == 12 and s["p99_ms"] >= s["p50_ms"]

    # the same request alone gives the same solution
    from paper_2203_02798_gb300.serve import run_trace
    p0 = payloads[4]
    alone, _ = run_trace([Request(4, 0.0, 1, p0)], lambda slot, req: server.solve(slot, p0["A"], p0["b"], **p0["opts"]),
                         slots=1, hbm_budget=10)
    x_alone = alone[0].result[0]
    x_mix = by_id[4].result[0]
    assert np.linalg.norm(x_alone - x_mix) <= 1e-8 * np.linalg.norm(x_alone)


def test_concurrent_contexts_launch_different_sizes():
    """Eight host threads, each with its own context and stream, run leverage
    scores of problems whose d (and so the kernels' shared-memory needs)
    differ, 24 times each: every call succeeds and equals the same problem
    computed alone.  (The kernels' dynamic shared-memory limits are process-
    wide; per-launch values raced between such threads.)"""
    import threading
    import paper_2203_02798_gb300 as lsk
    dims = [48, 96, 160, 256, 64, 200, 128, 32]
    probs = []
    for t, d in enumerate(dims):
        A = torch.from_numpy(workloads.dense_normal(3000 + 97 * t, d, seed=70 + t)).cuda()
        probs.append((A, max(4 * d, 1024), 2 * d, 11 + t))
    ref = []
    for A, r, k, s in probs:
        ref.append(lsk.leverage_scores(A, r, k, s, "bf16"))
        lsk.context().sync()
    errors, bad = [], []

    def worker(t):
        try:
            A, r, k, s = probs[t]
            stream = torch.cuda.Stream()
            ctx = lsk.Context(0)
            with torch.cuda.stream(stream):
                for _ in range(24):
                    ell = lsk.leverage_scores(A, r, k, s, "bf16", ctx=ctx)
                    ctx.sync()
                    if torch.max(torch.abs(ell - ref[t]) / ref[t]).item() > 1e-4:
                        bad.append(t)
            ctx.close()
        except Exception as e:   # collected and asserted below
            errors.append(f"{t}: {e}")

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(len(dims))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert errors == [] and bad == []
