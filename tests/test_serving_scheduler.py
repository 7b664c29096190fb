"""Continuous batching admission (ContinuousServer.run) on the CPU.

The server's slots are given fake library contexts, streams and events: a level
request "runs" for a simulated service time after it is launched, and its event
completes when that time has passed.  What is checked is the scheduling policy
alone: requests are launched in arrival order, never before they arrive, each
exactly once; the workspace bytes of the requests running at any launch plus the
launched one stay within the HBM budget; a request larger than the budget is
rejected instead of waiting forever; the arena's first-fit allocator hands out
disjoint ranges and coalesces what comes back; the device-clock overlap summary
counts time with two or more requests running."""
import time

import pytest

pytest.importorskip("torch")
from paper_2606_09291_gb300.serving import ContinuousServer, FirstFit, device_overlap, poisson_mix_requests  # noqa: E402


class FakeStream:
    def __init__(self):
        self.busy_until = 0.0


class FakeEvent:
    def __init__(self):
        self.t = None

    def record(self, stream):
        # start events are recorded before the launch (stream idle), end events after it
        self.t = max(time.perf_counter(), stream.busy_until)

    def query(self):
        return time.perf_counter() >= self.t

    def elapsed_time(self, end):
        return 1e3 * (end.t - self.t)


class FakeCtx:
    def __init__(self, log, service_s, footprint, budget_check):
        self.log, self.service_s, self.fp, self.check = log, service_s, footprint, budget_check

    def mlsgd_workspace_bytes(self, level, n):
        return self.fp(level, n)

    def mlsgd_set_workspace(self, ptr, nbytes):
        self.ws = (ptr, nbytes)

    def mlsgd_stats_reset(self, st, stream=None):
        pass

    def mlsgd_level_gradient(self, eid, level, first, n, z, st, stream=None):
        now = time.perf_counter()
        self.check(now, self.fp(level, n))
        stream.busy_until = now + self.service_s(level, n)
        self.log.append(dict(t=now, eid=eid, level=level, n=n, until=stream.busy_until))


def make_server(n_slots, n_levels, budget, service_s, footprint):
    log = []
    srv = object.__new__(ContinuousServer)
    srv.cfg = dict(n_levels=n_levels)
    srv.budget = 10 ** 12 if budget is None else budget
    srv.alloc = FirstFit(srv.budget, granule=1)
    srv.base = 0
    srv._new_event = FakeEvent
    srv._ref_stream = FakeStream

    def check(now, fp):  # requests still running at this launch, by their simulated end
        running = sum(footprint(r["level"], r["n"]) for r in log if r["until"] > now)
        assert running + fp <= srv.budget

    srv.slots = [dict(ctx=FakeCtx(log, service_s, footprint, check), stream=FakeStream(),
                      stats=[object() for _ in range(n_levels)], req=None, ev=None, t0=None) for _ in range(n_slots)]
    return srv, log


def _check_run(reqs, out, log):
    assert len(out) == len(reqs) == len(log)
    # launched in arrival order, each exactly once
    assert [(r["eid"], r["level"], r["n"]) for r in log] == [(e, l, n) for (_, e, l, n) in reqs]
    for (a, e, l, n), o in zip(reqs, out):
        assert o is not None and (o["estimate"], o["level"], o["n"]) == (e, l, n)
        assert o["start"] >= a - 1e-9 and o["done"] >= o["start"]
        assert o["service_ms"] >= 0.0


@pytest.mark.parametrize("budget", [None, 6000.0, 4000.0])
def test_fifo_admission_within_budget(budget):
    mix = (4, 2, 1)
    footprint = lambda level, n: 1000.0 * (level + 1)          # noqa: E731  (level 2 alone: 3000)
    service = lambda level, n: 0.002 * (level + 1)             # noqa: E731
    srv, log = make_server(3, len(mix), budget, service, footprint)
    reqs = poisson_mix_requests(mix, 6, rate_per_s=400.0, seed=1)
    out = srv.run(reqs, z=None)
    _check_run(reqs, out, log)


def test_slots_bound_concurrency():
    footprint = lambda level, n: 1.0                           # noqa: E731
    service = lambda level, n: 0.003                           # noqa: E731
    srv, log = make_server(2, 1, None, service, footprint)
    reqs = [(0.0, e, 0, 1) for e in range(6)]                  # all arrive at once
    out = srv.run(reqs, z=None)
    _check_run(reqs, out, log)
    for r in log:  # never more than two requests running together
        assert sum(1 for q in log if q["t"] <= r["t"] < q["until"]) <= 2


def test_budget_serialises_large_requests():
    footprint = lambda level, n: 10.0 * n                      # noqa: E731
    service = lambda level, n: 0.003                           # noqa: E731
    srv, log = make_server(4, 1, 15.0, service, footprint)
    reqs = [(0.0, e, 0, 1) for e in range(5)]                  # 10 bytes each, budget 15: one at a time
    out = srv.run(reqs, z=None)
    _check_run(reqs, out, log)
    for a, b in zip(log, log[1:]):
        assert b["t"] >= a["until"]


def test_request_over_budget_is_rejected():
    srv, log = make_server(2, 1, 5.0, lambda level, n: 0.001, lambda level, n: 10.0)
    with pytest.raises(ValueError):
        srv.run([(0.0, 0, 0, 1)], z=None)
    assert log == []


def test_first_fit_arena():
    a = FirstFit(4096)
    x, y, z = a.alloc(100), a.alloc(1000), a.alloc(256)
    assert (x, y, z) == (0, 256, 1280)  # 256-byte granules
    assert a.alloc(4096) is None
    a.release(y, 1000)
    assert a.alloc(700) == 256          # first fit reuses the hole
    a.release(x, 100)
    a.release(z, 256)
    a.release(256, 700)
    assert a.free == [(0, 4096)]        # coalesced back to one range


def test_device_overlap_summary():
    recs = [dict(dev_start_ms=0.0, dev_end_ms=4.0), dict(dev_start_ms=1.0, dev_end_ms=3.0),
            dict(dev_start_ms=6.0, dev_end_ms=7.0)]
    o = device_overlap(recs)
    assert o["busy_ms"] == 5.0 and o["overlapped_ms"] == 2.0 and o["max_concurrent"] == 2
