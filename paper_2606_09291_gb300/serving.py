"""Serving loop for multilevel gradient estimates (the MLMC mix of levels).

One request is one multilevel gradient estimate: for every level l a batch of
M_l fresh samples (sample identity (seed, request, level, index)) processed by
mlsgd_level_gradient into that level's statistics record (Algorithm 1,
GradientEstimate).  The levels of a request are independent until the combine
step, so the server gives every level its own library context (its own scratch)
and its own CUDA stream: the small, latency-bound levels run concurrently with
the large ones instead of after them.  Results do not depend on this overlap
(every kernel is deterministic and levels share no buffers), which the GPU
tests check bit for bit.

Two servers.  MixServer runs one estimate at a time with its levels overlapped;
its latency under load follows from the measured service times of a FIFO queue
(completion_i = max(arrival_i, completion_{i-1}) + service_i).  ContinuousServer
batches continuously: level requests of many estimates are admitted, as slots and
HBM free up, while others run, and are timed in real time from arrival to
completion.  Throughput is sample-gradients of the mix per second.

    python -m paper_2606_09291_gb300.serving --preset c4 --requests 40
"""
import argparse
import json
import statistics
import sys

import numpy as np
import torch

from . import inputs, mlsgd


def mix_config(preset, precision="mixed"):
    p = dict(inputs.PRESETS[preset])
    mix = tuple(p.pop("mix", (1024, 256, 64, 16, 4, 1)))
    p.pop("counts", None)
    p.pop("thetas", None)
    p.update(precision=precision, rtol=1e-8, max_iter=50, ir_steps=3, field_tc=1,
             max_batch=max(mix))
    return p, mix


class MixServer:
    """Per-level contexts and streams for concurrent level batches."""

    def __init__(self, cfg, mix, concurrent=True):
        self.cfg, self.mix, self.concurrent = dict(cfg), tuple(mix), concurrent
        L = len(self.mix)
        self.ctx = [mlsgd.Context(**self.cfg) for _ in range(L)]
        self.streams = [torch.cuda.Stream() for _ in range(L)] if concurrent else [torch.cuda.current_stream()] * L
        self.stats = [self.ctx[l].new_stats(l) for l in range(L)]
        self.main = torch.cuda.current_stream()

    def close(self):
        for c in self.ctx:
            c.close()

    def submit(self, request, z):
        """Enqueue one multilevel estimate; returns (start, end) events on the main stream."""
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.main)
        done = []
        for l, m in enumerate(self.mix):
            s = self.streams[l]
            s.wait_event(e0)
            self.ctx[l].mlsgd_stats_reset(self.stats[l], stream=s)
            self.ctx[l].mlsgd_level_gradient(request, l, 0, m, z, self.stats[l], stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
            done.append(ev)
        for ev in done:
            self.main.wait_event(ev)
        e1.record(self.main)
        return e0, e1

    def serve(self, requests, z, first_request=0):
        """Service time (ms) of each request, run back to back."""
        times = []
        for r in range(requests):
            e0, e1 = self.submit(first_request + r, z)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times


class FirstFit:
    """First-fit allocator of byte ranges in [0, size) in granules of `granule`
    bytes (256: the library's workspace alignment), the HBM arena of the
    continuous-batching server."""

    def __init__(self, size, granule=256):
        self.size, self.granule = int(size), int(granule)
        self.free = [(0, self.size)]  # sorted, coalesced (offset, length)

    def round(self, n):
        g = self.granule
        return (int(n) + g - 1) // g * g

    def alloc(self, n):
        n = self.round(n)
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                self.free[i:i + 1] = [(off + n, ln - n)] if ln > n else []
                return off
        return None

    def release(self, off, n):
        n = self.round(n)
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


def device_overlap(records):
    """From device timestamps (dev_start_ms, dev_end_ms per request): the time some
    request ran, the time at least two ran together, and the most that ran at once."""
    ev = sorted([(r["dev_start_ms"], 1) for r in records] + [(r["dev_end_ms"], -1) for r in records])
    busy = multi = 0.0
    depth = peak = 0
    last = None
    for t, d in ev:
        if last is not None:
            if depth >= 1:
                busy += t - last
            if depth >= 2:
                multi += t - last
        depth += d
        peak = max(peak, depth)
        last = t
    return dict(busy_ms=busy, overlapped_ms=multi, overlap_fraction=multi / busy if busy > 0 else 0.0,
                max_concurrent=peak)


class ContinuousServer:
    """Continuous batching of per-level sample-solve requests.

    A request is (estimate id, level, sample count): one level batch of one
    multilevel estimate, computed by mlsgd_level_gradient into its own level record
    (sample identity (seed, estimate id, level, index), so a request's result does
    not depend on what else runs).  The server owns n_slots slots, each a library
    context with its own CUDA stream, and one HBM arena of `budget` bytes: a request
    runs in a range of the arena that it holds from launch to completion (handed to
    its slot's context with mlsgd_set_workspace, so the library allocates no
    scratch while serving).  Requests wait in arrival order; the head of the queue
    is admitted as soon as a slot is free and the arena has room for its workspace
    bytes (mlsgd_workspace_bytes), so work arriving while the GPU is busy starts
    without waiting for the running requests to end and overlaps them on the
    device.  The budget defaults to the smaller of half the device memory free at
    construction and n_slots times the largest request's workspace.  Each request's
    start and end are also recorded as device events, so overlap is measured on the
    GPU's own clock."""

    def __init__(self, cfg, n_slots, largest_requests, hbm_budget=None):
        self.cfg = dict(cfg)
        self.slots = []
        L = self.cfg["n_levels"]
        Nc = self.cfg["n0"] << self.cfg.get("ctrl_level", L - 1)
        zwarm = torch.zeros(Nc ** 3, dtype=torch.float64, device="cuda")
        probe = mlsgd.Context(**self.cfg)
        largest = max(probe.mlsgd_workspace_bytes(l, n) for l, n in largest_requests)
        probe.close()
        if hbm_budget is None:
            hbm_budget = min(int(0.5 * torch.cuda.mem_get_info()[0]), n_slots * FirstFit(0).round(largest))
        self.arena = torch.empty(int(hbm_budget), dtype=torch.uint8, device="cuda")
        self.base = self.arena.data_ptr()
        self.set_budget(hbm_budget)
        for _ in range(n_slots):
            ctx = mlsgd.Context(**self.cfg)
            stream = torch.cuda.Stream()
            stats = [ctx.new_stats(l) for l in range(L)]
            for (level, n) in largest_requests:  # build the per-grid tables (arena start as scratch)
                fp = ctx.mlsgd_workspace_bytes(level, n)
                if fp <= self.budget:
                    ctx.mlsgd_set_workspace(self.base, fp)
                    ctx.mlsgd_level_gradient(0, level, 0, n, zwarm, stats[level], stream=stream)
                    stream.synchronize()
            self.slots.append(dict(ctx=ctx, stream=stream, stats=stats, req=None, ev=None, t0=None))
        torch.cuda.synchronize()

    def set_budget(self, nbytes):
        """Admit by at most nbytes of the arena from now on (at most the arena's size)."""
        self.budget = min(int(nbytes), self.arena.numel())
        self.alloc = FirstFit(self.budget)

    @staticmethod
    def _new_event():
        return torch.cuda.Event(enable_timing=True)

    @staticmethod
    def _ref_stream():
        return torch.cuda.current_stream()

    def close(self):
        for s in self.slots:
            s["ctx"].mlsgd_set_workspace(0, 0)
            s["ctx"].close()

    def footprint(self, level, n):
        return self.slots[0]["ctx"].mlsgd_workspace_bytes(level, n)

    def run(self, requests, z, keep=False):
        """requests: list of (arrival_s, estimate_id, level, n), sorted by arrival.
        Returns one dict per request (arrival, start, done, latency_ms, service_ms,
        dev_start_ms / dev_end_ms on the device clock from the start of the run) and,
        with keep, copies of the level records (field, scalars).  self.deferred counts
        the polls in which the queue head waited for arena room while a slot was free.
        A request whose workspace alone exceeds the budget could never be admitted:
        ValueError."""
        import collections
        import time
        for (a, eid, level, n) in requests:
            if self.alloc.round(self.footprint(level, n)) > self.budget:
                raise ValueError("request (estimate %d, level %d, %d samples) needs %d workspace bytes, over the "
                                 "budget of %d" % (eid, level, n, self.footprint(level, n), self.budget))
        pending = collections.deque(range(len(requests)))
        queue = collections.deque()
        out = [None] * len(requests)
        self.deferred = 0
        ref = self._new_event()
        ref.record(self._ref_stream())
        t_start = time.perf_counter()
        while pending or queue or any(s["req"] is not None for s in self.slots):
            now = time.perf_counter() - t_start
            while pending and requests[pending[0]][0] <= now:
                queue.append(pending.popleft())
            for s in self.slots:  # completions
                if s["req"] is not None and s["ev"].query():
                    i = s["req"]
                    a, eid, level, n = requests[i]
                    rec = dict(arrival=a, start=s["t0"], done=now, latency_ms=1e3 * (now - a),
                               service_ms=s["e0"].elapsed_time(s["ev"]), level=level, n=n, estimate=eid,
                               dev_start_ms=ref.elapsed_time(s["e0"]), dev_end_ms=ref.elapsed_time(s["ev"]))
                    if keep:
                        st = s["stats"][level]
                        rec["field"], rec["scalars"] = st.field.clone(), st.scalars.clone()
                    out[i] = rec
                    self.alloc.release(s["off"], self.footprint(level, n))
                    s["req"] = None
            for s in self.slots:  # admissions, in arrival order
                if not queue:
                    break
                if s["req"] is not None:
                    continue
                i = queue[0]
                a, eid, level, n = requests[i]
                fp = self.footprint(level, n)
                off = self.alloc.alloc(fp)
                if off is None:
                    self.deferred += 1
                    break
                queue.popleft()
                st = s["stats"][level]
                s["ctx"].mlsgd_set_workspace(self.base + off, self.alloc.round(fp))
                s["e0"] = self._new_event()
                s["e0"].record(s["stream"])
                s["ctx"].mlsgd_stats_reset(st, stream=s["stream"])
                s["ctx"].mlsgd_level_gradient(eid, level, 0, n, z, st, stream=s["stream"])
                s["ev"] = self._new_event()
                s["ev"].record(s["stream"])
                s["req"], s["t0"], s["off"] = i, now, off
            if not queue or all(s["req"] is not None for s in self.slots):
                time.sleep(1e-4)
        return out


def poisson_mix_requests(mix, n_estimates, rate_per_s, seed=0, first_estimate=0):
    """Estimates arrive as a Poisson process; each brings one request per level."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    for e in range(n_estimates):
        t += rng.exponential(1.0 / rate_per_s) if rate_per_s > 0 else 0.0
        for l, m in enumerate(mix):
            reqs.append((t, first_estimate + e, l, m))
    return reqs


def fifo_latency(service_ms, rate_per_s, seed=0):
    """Latencies (ms) of requests with exponential inter-arrival times served FIFO."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1000.0 / rate_per_s, size=len(service_ms))
    t_arr, t_free, lat = 0.0, 0.0, []
    for g, s in zip(gaps, service_ms):
        t_arr += g
        start = max(t_arr, t_free)
        t_free = start + s
        lat.append(t_free - t_arr)
    return lat


def pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(np.ceil(q * len(v))) - 1)]


def level_throughput(cfg, level, n, reps=3, z=None):
    """Sample-gradients/s of one level batch of n samples alone (one stream)."""
    ctx = mlsgd.Context(**dict(cfg, max_batch=n))
    st = ctx.new_stats(level)
    ctx.mlsgd_level_gradient(0, level, 0, n, z, st)  # warm-up (sizes the scratch)
    torch.cuda.synchronize()
    best = float("inf")
    for r in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.mlsgd_stats_reset(st)
        e0.record()
        ctx.mlsgd_level_gradient(1 + r, level, 0, n, z, st)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    ctx.close()
    return n / (best / 1e3), best


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--preset", default="c4", choices=("c4", "c5"))
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--level-batch", type=int, default=1024, help="samples per level for the per-level rates")
    ap.add_argument("--slots", type=int, default=6, help="continuous batching: concurrent requests")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    cfg, mix = mix_config(a.preset)
    Nc = cfg["n0"] << (cfg["n_levels"] - 1)
    z = torch.tensor(inputs.z_test(Nc), dtype=torch.float64, device="cuda")
    out = {"preset": a.preset, "mix": list(mix)}
    for conc in (False, True):
        srv = MixServer(cfg, mix, concurrent=conc)
        srv.serve(a.warmup, z, first_request=10000)
        t = srv.serve(a.requests, z)
        srv.close()
        mean = statistics.mean(t)
        key = "concurrent_levels" if conc else "one_stream"
        out[key] = {"service_ms": {"p50": statistics.median(t), "p99": pct(t, 0.99), "mean": mean},
                    "sample_gradients_per_s": sum(mix) / (mean / 1e3)}
        if conc:
            cap = 1000.0 / mean
            out["latency_under_load"] = []
            for f in (0.25, 0.5, 0.75, 0.9, 0.97):
                lat = fifo_latency(t * 20, f * cap, seed=1)[len(t):]  # repeat the measured services, drop warm-up
                out["latency_under_load"].append({"load": f, "requests_per_s": f * cap,
                                                  "p50_ms": statistics.median(lat), "p99_ms": pct(lat, 0.99)})
    # continuous batching: estimates arrive as a Poisson process, level requests overlap
    srv = ContinuousServer(cfg, a.slots, [(l, m) for l, m in enumerate(mix)])
    sat = srv.run(poisson_mix_requests(mix, a.requests, 0.0, first_estimate=20000), z)  # all at t = 0
    span = max(r["done"] for r in sat) - min(r["start"] for r in sat)
    cap = a.requests / span  # estimates per second at saturation
    out["continuous"] = {"slots": a.slots, "hbm_budget_bytes": srv.budget, "saturated_estimates_per_s": cap,
                         "saturated_sample_gradients_per_s": cap * sum(mix), "device_overlap": device_overlap(sat),
                         "deferred_by_hbm": srv.deferred, "load": []}
    for f in (0.25, 0.5, 0.75, 0.9):
        res = srv.run(poisson_mix_requests(mix, a.requests, f * cap, seed=2, first_estimate=30000), z)
        est = {}
        for r in res:
            est.setdefault(r["estimate"], []).append(r)
        lat_e = [1e3 * (max(x["done"] for x in v) - v[0]["arrival"]) for v in est.values()]
        lat_r = [r["latency_ms"] for r in res]
        out["continuous"]["load"].append({"load": f, "estimates_per_s": f * cap,
                                          "estimate_p50_ms": statistics.median(lat_e), "estimate_p99_ms": pct(lat_e, 0.99),
                                          "request_p50_ms": statistics.median(lat_r), "request_p99_ms": pct(lat_r, 0.99)})
    srv.close()
    out["per_level"] = []
    for l in range(len(mix)):
        n = max(1, min(a.level_batch, a.level_batch >> (2 * max(0, l - 2))))
        rate, ms = level_throughput(cfg, l, n, z=z)
        out["per_level"].append({"level": l, "N": cfg["n0"] << l, "samples": n, "ms": ms,
                                 "sample_gradients_per_s": rate})
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
