"""Continuous-batching server for sketch-and-precondition least squares.

A request is one least-squares problem min ||A x - b|| (A dense or CSR,
resident on the device; b on the device) solved with
``lsk_sketch_precondition_lsq`` (Alg. 12: sketch, R of the sketch, CG on the
normal equations of A R^-1 within FP64 refinement).  The server keeps ``slots`` worker threads,
each with its own CUDA stream and library context (its own workspace), so
admitted requests run concurrently on the GPU.  Requests are admitted in
arrival order as soon as a slot is free and their device footprint fits
the HBM budget; a request that arrives while others run starts as soon as
those conditions hold (continuous batching, not a queue in front of a
single executor).  Every request's sketch, R and iterate stay on the device
for its whole solve.

Scheduling and admission are plain host logic (``Scheduler``), tested on
the CPU with fake jobs; ``Server`` binds them to the GPU library.
"""
import collections
import dataclasses
import heapq
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds, trace time
    footprint: int            # device bytes the solve needs (workspace + vectors)
    payload: object = None    # whatever the executor needs (A, b, options)


@dataclasses.dataclass
class Completion:
    rid: int
    arrival: float
    start: float
    finish: float
    result: object = None
    error: str = None

    @property
    def latency(self):
        return self.finish - self.arrival


class Scheduler:
    """Admission by free slots and an HBM budget, FIFO by arrival.

    ``admit(now)`` returns the requests that may start now; ``release`` returns
    a finished request's slot and bytes.  A request larger than the whole
    budget is rejected (it could never be admitted).
    """

    def __init__(self, slots, hbm_budget):
        self.slots = int(slots)
        self.budget = int(hbm_budget)
        self.free_slots = int(slots)
        self.used = 0
        self.waiting = collections.deque()
        self.rejected = []

    def arrive(self, req):
        if req.footprint > self.budget:
            self.rejected.append(req)
            return False
        self.waiting.append(req)
        return True

    def admit(self):
        started = []
        while self.waiting and self.free_slots > 0 and self.used + self.waiting[0].footprint <= self.budget:
            req = self.waiting.popleft()
            self.free_slots -= 1
            self.used += req.footprint
            started.append(req)
        return started

    def release(self, req):
        self.free_slots += 1
        self.used -= req.footprint
        assert self.free_slots <= self.slots and self.used >= 0


def run_trace(requests, execute, slots, hbm_budget, time_scale=1.0, clock=time.perf_counter):
    """Replay ``requests`` (sorted by arrival) against ``execute(slot, req)``.

    ``execute`` runs on one of ``slots`` worker threads and returns the
    request's result.  Arrivals are released at their trace times (scaled by
    ``time_scale``); admission follows :class:`Scheduler`.  Returns the
    completions in finish order and the rejected requests.
    """
    sched = Scheduler(slots, hbm_budget)
    lock = threading.Condition()
    done = []
    free_slot_ids = list(range(slots))
    t0 = clock()
    pending = list(requests)
    pending.reverse()
    active = [0]

    def worker(slot, req, start):
        res, err = None, None
        try:
            res = execute(slot, req)
        except Exception as e:  # reported, not raised: the trace continues
            err = f"{type(e).__name__}: {e}"
        fin = clock() - t0
        with lock:
            done.append(Completion(req.rid, req.arrival * time_scale, start, fin, res, err))
            sched.release(req)
            free_slot_ids.append(slot)
            active[0] -= 1
            lock.notify_all()

    with lock:
        while pending or sched.waiting or active[0]:
            now = clock() - t0
            while pending and pending[-1].arrival * time_scale <= now:
                sched.arrive(pending.pop())
            for req in sched.admit():
                slot = free_slot_ids.pop()
                active[0] += 1
                threading.Thread(target=worker, args=(slot, req, clock() - t0), daemon=True).start()
            if pending:
                wait = pending[-1].arrival * time_scale - (clock() - t0)
                lock.wait(timeout=max(0.0, min(wait, 0.05)))
            elif sched.waiting or active[0]:
                lock.wait(timeout=0.05)
    done.sort(key=lambda c: c.finish)
    return done, sched.rejected


def latency_summary(completions, slots=None):
    """Latency percentiles, split into the wait for admission (arrival to
    start: queueing behind busy slots or the HBM budget) and the service time
    (start to finish: the solve, sharing the GPU with the other slots)."""
    ok = [c for c in completions if c.error is None]
    lat = np.array([c.latency for c in ok])
    if lat.size == 0:
        return {"count": 0}
    queue = np.array([c.start - c.arrival for c in ok])
    service = np.array([c.finish - c.start for c in ok])
    span = max(c.finish for c in completions) - min(c.arrival for c in completions)
    pct = lambda a, q: float(np.percentile(a, q) * 1e3)
    out = {"count": int(lat.size), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
           "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3), "span_s": float(span),
           "throughput_rps": float(lat.size / span) if span > 0 else None,
           "errors": sum(1 for c in completions if c.error is not None),
           "queue_p50_ms": pct(queue, 50), "queue_p99_ms": pct(queue, 99),
           "service_p50_ms": pct(service, 50), "service_p99_ms": pct(service, 99)}
    if slots and span > 0:
        out["slot_busy_frac"] = float(service.sum() / (span * slots))   # mean fraction of the slots in use
    return out


class Server:
    """GPU executor: one library context and CUDA stream per slot."""

    def __init__(self, slots=8, device=0):
        import torch

        import paper_2203_02798_gb300 as lsk
        self.lsk = lsk
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.slots = slots
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.ctxs = [lsk.Context(device) for _ in range(slots)]

    @staticmethod
    def footprint(n, d, nnz=None, r=None, k=None):
        """Device bytes one solve holds beyond its inputs: sketch, factors, vectors."""
        r = r if r is not None else max(d * d, 4 * d)
        k = k if k is not None else 2 * d
        return int(4 * r * d + 4 * k * d + 40 * d * d + 12 * n + 8 * n + (1 << 20))

    def solve(self, slot, A, b, **opts):
        """One request on ``slot``'s stream; returns (x on the host, info)."""
        torch = self.torch
        with torch.cuda.stream(self.streams[slot]):
            x, info = self.lsk.sketch_precondition_lsq(A, b, ctx=self.ctxs[slot], **opts)
            xh = x.cpu()
        return xh.numpy(), info

    def run(self, requests, hbm_budget=150 * 10**9, time_scale=1.0):
        """Replay a trace whose payloads are dicts with A, b and options."""
        def execute(slot, req):
            p = req.payload
            return self.solve(slot, p["A"], p["b"], **p.get("opts", {}))
        return run_trace(requests, execute, self.slots, hbm_budget, time_scale)

    def close(self):
        for c in self.ctxs:
            c.close()
