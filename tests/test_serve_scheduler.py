"""Host logic of the continuous-batching server (CPU only, fake jobs):
FIFO admission by free slots and HBM budget, rejection of requests larger
than the budget, concurrency never above the slot count, the budget never
exceeded, and requests arriving while others run start before those finish."""
import threading
import time

from paper_2203_02798_gb300.serve import Request, Scheduler, latency_summary, run_trace


def test_scheduler_fifo_slots_and_budget():
    s = Scheduler(slots=2, hbm_budget=100)
    for i, f in enumerate([40, 40, 30, 10]):
        assert s.arrive(Request(i, 0.0, f))
    started = s.admit()
    assert [r.rid for r in started] == [0, 1]          # two slots
    assert s.admit() == []
    s.release(started[0])
    nxt = s.admit()
    assert [r.rid for r in nxt] == [2]                 # 40 + 30 <= 100
    s.release(started[1])
    assert [r.rid for r in s.admit()] == [3]
    assert not s.arrive(Request(9, 0.0, 101))          # never fits: rejected
    assert [r.rid for r in s.rejected] == [9]


def test_scheduler_budget_blocks_head_of_line():
    s = Scheduler(slots=4, hbm_budget=100)
    s.arrive(Request(0, 0.0, 90))
    s.arrive(Request(1, 0.0, 20))
    s.arrive(Request(2, 0.0, 5))
    assert [r.rid for r in s.admit()] == [0]           # FIFO: 1 waits for the budget
    assert s.used == 90


def test_run_trace_overlap_and_limits():
    state = {"active": 0, "max_active": 0, "used": 0, "max_used": 0}
    lock = threading.Lock()
    foot = {i: 10 + (i % 3) * 15 for i in range(24)}

    def execute(slot, req):
        with lock:
            state["active"] += 1
            state["used"] += req.footprint
            state["max_active"] = max(state["max_active"], state["active"])
            state["max_used"] = max(state["max_used"], state["used"])
        time.sleep(0.02 + 0.01 * (req.rid % 4))
        with lock:
            state["active"] -= 1
            state["used"] -= req.footprint
        return req.rid * 2

    reqs = [Request(i, 0.004 * i, foot[i]) for i in range(24)]
    done, rejected = run_trace(reqs, execute, slots=3, hbm_budget=70)
    assert not rejected and len(done) == 24
    assert state["max_active"] <= 3 and state["max_used"] <= 70
    assert sorted(c.result for c in done) == [2 * i for i in range(24)]
    # continuous batching: some request started while an earlier one was running
    by_id = {c.rid: c for c in done}
    assert any(by_id[i + 1].start < by_id[i].finish for i in range(23))
    summ = latency_summary(done, slots=3)
    assert summ["count"] == 24 and summ["p99_ms"] >= summ["p50_ms"] > 0
    # latency = admission wait + service, request by request
    for c in done:
        assert c.start >= c.arrival - 1e-9 and c.finish >= c.start
    assert summ["queue_p99_ms"] >= summ["queue_p50_ms"] >= 0
    assert summ["service_p99_ms"] >= summ["service_p50_ms"] > 0
    assert summ["max_ms"] <= 1e3 * max(c.start - c.arrival for c in done) + 1e3 * max(c.finish - c.start for c in done) + 1e-6
    assert 0 < summ["slot_busy_frac"] <= 1.0


def test_run_trace_reports_errors():
    def execute(slot, req):
        if req.rid == 1:
            raise RuntimeError("boom")
        return 0

    done, _ = run_trace([Request(i, 0.0, 1) for i in range(3)], execute, slots=2, hbm_budget=10)
    errs = [c for c in done if c.error]
    assert len(errs) == 1 and "boom" in errs[0].error
