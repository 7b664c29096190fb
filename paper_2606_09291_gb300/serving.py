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

Latency under load: requests arrive as a Poisson process; they are served one
at a time in arrival order, each taking its measured service time (CUDA events
around the request's work, GPU otherwise idle), so the completion time of
request i is max(arrival_i, completion_{i-1}) + service_i.  Throughput is the
number of sample-gradients of the mix per second of service.

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
