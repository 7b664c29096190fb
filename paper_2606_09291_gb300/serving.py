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


class ContinuousServer:
    """Continuous batching of per-level sample-solve requests.

    A request is (estimate id, level, sample count): one level batch of one
    multilevel estimate, computed by mlsgd_level_gradient into its own level record
    (sample identity (seed, estimate id, level, index), so a request's result does
    not depend on what else runs).  The server owns n_slots slots, each a library
    context with its own scratch and its own CUDA stream.  Requests wait in arrival
    order; the head of the queue is admitted to a free slot as soon as one frees up
    and the workspace bytes of the requests in flight plus its own fit the HBM
    budget, so work arriving while the GPU is busy starts without waiting for the
    running requests to end and overlaps them on the device.  Every slot's scratch
    is sized once for the largest request before serving (no allocation, hence no
    device synchronisation, while serving)."""

    def __init__(self, cfg, n_slots, largest_requests, hbm_budget=None):
        self.cfg = dict(cfg)
        self.slots = []
        L = self.cfg["n_levels"]
        Nc = self.cfg["n0"] << self.cfg.get("ctrl_level", L - 1)
        zwarm = torch.zeros(Nc ** 3, dtype=torch.float64, device="cuda")
        for _ in range(n_slots):
            ctx = mlsgd.Context(**self.cfg)
            stream = torch.cuda.Stream()
            stats = [ctx.new_stats(l) for l in range(L)]
            for (level, n) in largest_requests:  # size the scratch and build the per-grid tables
                ctx.mlsgd_level_gradient(0, level, 0, n, zwarm, stats[level], stream=stream)
            self.slots.append(dict(ctx=ctx, stream=stream, stats=stats, req=None, ev=None, t0=None))
        torch.cuda.synchronize()
        # bytes of library scratch the requests in flight may need together (None: no
        # limit beyond the slots, whose scratch is already reserved)
        self.budget = float("inf") if hbm_budget is None else hbm_budget

    @staticmethod
    def _new_event():
        return torch.cuda.Event(enable_timing=True)

    def close(self):
        for s in self.slots:
            s["ctx"].close()

    def footprint(self, level, n):
        return self.slots[0]["ctx"].mlsgd_workspace_bytes(level, n)

    def run(self, requests, z, keep=False):
        """requests: list of (arrival_s, estimate_id, level, n), sorted by arrival.
        Returns one dict per request (arrival, start, done, latency_ms, service_ms) and,
        with keep, copies of the level records (field, scalars).  A request whose
        workspace alone exceeds the HBM budget could never be admitted: ValueError."""
        import collections
        import time
        for (a, eid, level, n) in requests:
            if self.footprint(level, n) > self.budget:
                raise ValueError("request (estimate %d, level %d, %d samples) needs %d workspace bytes, over the "
                                 "budget of %d" % (eid, level, n, self.footprint(level, n), self.budget))
        pending = collections.deque(range(len(requests)))
        queue = collections.deque()
        out = [None] * len(requests)
        in_flight = 0
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
                               service_ms=s["e0"].elapsed_time(s["ev"]), level=level, n=n, estimate=eid)
                    if keep:
                        st = s["stats"][level]
                        rec["field"], rec["scalars"] = st.field.clone(), st.scalars.clone()
                    out[i] = rec
                    in_flight -= self.footprint(level, n)
                    s["req"] = None
            for s in self.slots:  # admissions, in arrival order
                if not queue:
                    break
                if s["req"] is not None:
                    continue
                i = queue[0]
                a, eid, level, n = requests[i]
                fp = self.footprint(level, n)
                if in_flight + fp > self.budget:
                    break
                queue.popleft()
                in_flight += fp
                st = s["stats"][level]
                s["e0"] = self._new_event()
                s["e0"].record(s["stream"])
                s["ctx"].mlsgd_stats_reset(st, stream=s["stream"])
                s["ctx"].mlsgd_level_gradient(eid, level, 0, n, z, st, stream=s["stream"])
                s["ev"] = self._new_event()
                s["ev"].record(s["stream"])
                s["req"], s["t0"] = i, now
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
    out["continuous"] = {"slots": a.slots, "saturated_estimates_per_s": cap,
                         "saturated_sample_gradients_per_s": cap * sum(mix), "load": []}
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
