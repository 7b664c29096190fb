#!/usr/bin/env python
"""Benchmark of the multilevel entropic-risk gradient hot path on GB300.

Default workload (c3): 4096 sample-gradients per step at level 3 (64^3 cells,
250,047 interior dofs) with their level-2 partners on the same draws, 256 KL
modes (corr length 0.2, sigma 1), theta = 10, mixed precision (BF16
coefficient for the V-cycle, FP32 MG-PCG, FP64 iterative refinement to rtol
1e-8).  One step = one call of mlsgd_level_gradient over the whole batch: xi,
fields on both grids, state and adjoint solves on both grids, B*q, entropic
weights, level differences and the Chan merge.

Prints ONE JSON line (rank 0).  --impl reference times the CPU FP64 oracle
on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sample-gradients/s (state+adjoint) at rtol 1e-8 vs plain FP64; p99 latency"
# DRAM bytes (read + write) over algorithmic bytes of the dominant kernel class, from
# one ncu capture of its 64^3 fine launch on a smaller batch of this workload (inputs
# larger than L2); a full launch processes more samples of the same grid, so its
# traffic is this ratio times its algorithmic bytes (ncu on the 64^3 slab launches of a
# 256-sample batch, profiles/slab_passes_c3_ncu.md).  Only valid for the kernel as
# captured: emptied with each change of that kernel until it is captured again.
TRAFFIC_RATIO = {"apply_f32": 0.996, "pre_f32": 1.037, "post_f32": 1.017}
# ALU-bound classes: the operations their launch sites count, against the issue rate of
# the units that execute them (152 SMs at 2070 MHz: 128 FP32 lanes per SM; FP64 at the
# nominal 1.25 TFLOP/s, i.e. 0.625 T operations/s)
ALU_PEAK = {"resid64": (152 * 128 * 2.07e9 / 1e12, "T FP32 ops/s", "FP32 lanes x max SM clock"),
            "level_field": (0.625, "T FP64 ops/s", "nominal FP64 rate")}
UNIT = "sample-gradients/s"


def workload_cfg(args):
    """The c3 configuration; the mixed path takes the autotuner's knobs for this batch
    from the committed cache (paper_2606_09291_gb300/tuned.json) when it has them."""
    from paper_2606_09291_gb300 import autotune, inputs
    p = dict(inputs.PRESETS["c3"])
    cfg = dict(n_levels=p["n_levels"], n0=p["n0"], n_modes=p["n_modes"], corr_len=p["corr_len"], sigma=p["sigma"],
               theta=p["theta"], alpha=p["alpha"], seed=p["seed"], rtol=1e-8, max_iter=50,
               precision=args.precision, max_batch=args.samples, ctrl_level=p["n_levels"] - 1,
               field_tc=1 if args.precision == "mixed" else 0, ir_steps=args.ir_steps)
    if args.precision == "mixed" and not getattr(args, "no_tuned", False):
        knobs = autotune.lookup(cfg, p["level"], args.samples)
        if knobs:
            if args.ir_steps:  # an explicit --ir-steps wins over the tuned schedule
                knobs["ir_steps"] = args.ir_steps
            cfg = autotune.context_cfg(cfg, knobs, args.samples)
    return cfg


def workload_name(args):
    return ("c3: %d samples/step at level 3 (64^3 cells) + level-2 partners, K=256 modes, corr 0.2, sigma 1, "
            "theta 10, %s, rtol 1e-8" % (args.samples, "tensor-core BF16 coef / FP32 MG-PCG / FP64 IR"
                                          if args.precision == "mixed"
                                          else "plain FP64 MG-PCG"))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(device_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [t.strip() for t in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6], swt=parts[7],
                                     pcap=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            if r["hw"].lower() == "active":
                reasons.add("hw_slowdown")
            if r["hwt"].lower() == "active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"].lower() == "active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"].lower() == "active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle legs
def oracle_rate(n_samples, it0=0):
    """Oracle sample-gradients/s on n_samples level-3 samples of the workload (rtol 1e-8)."""
    from oracle import mlmc
    from paper_2606_09291_gb300 import inputs
    p = inputs.PRESETS["c3"]
    W = mlmc.Workload(n0=p["n0"], n_levels=p["n_levels"], n_modes=p["n_modes"], corr_len=p["corr_len"],
                      sigma=p["sigma"], theta=p["theta"], alpha=p["alpha"], seed=p["seed"], rtol=1e-8)
    z = inputs.z_test(64)
    W.level(3), W.level(2)  # operators' static parts, outside the timing
    t = time.perf_counter()
    mlmc.level_batch(W, it0, 3, range(n_samples), z)
    dt = time.perf_counter() - t
    return n_samples / dt, dt


# all host cores: the unchanged oracle over disjoint sample ranges, one process per
# core (started with spawn: nothing is forked from a process that has used the GPU);
# each worker builds the operators' static parts before the timed map
_POOL_STATE = {}


def _oracle_worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import mlmc
    from paper_2606_09291_gb300 import inputs
    p = inputs.PRESETS["c3"]
    W = mlmc.Workload(n0=p["n0"], n_levels=p["n_levels"], n_modes=p["n_modes"], corr_len=p["corr_len"],
                      sigma=p["sigma"], theta=p["theta"], alpha=p["alpha"], seed=p["seed"], rtol=1e-8)
    W.level(3), W.level(2)
    _POOL_STATE.update(W=W, z=inputs.z_test(64), mlmc=mlmc)


def _oracle_worker_batch(task):
    it, first, count = task
    st = _POOL_STATE
    st["mlmc"].level_batch(st["W"], it, 3, range(first, first + count), st["z"])
    return count


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """A spawn-started pool of oracle processes, one per host core."""

    def __init__(self, procs):
        import multiprocessing as mp
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init)
        self.pool.map(_oracle_worker_batch, [(0, 10 ** 6 + i, 1) for i in range(procs)], chunksize=1)

    def rate(self, per_proc, it0):
        """Sample-gradients/s over procs * per_proc level-3 samples (wall time of the map)."""
        tasks = [(it0, i * per_proc, per_proc) for i in range(self.procs)]
        t = time.perf_counter()
        n = sum(self.pool.map(_oracle_worker_batch, tasks, chunksize=1))
        dt = time.perf_counter() - t
        return n / dt, dt, n

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_threads():
    try:
        import numpy  # noqa: F401
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return 1


def run_reference(args, rank):
    if rank != 0:
        return
    procs = host_cores()
    pool = OraclePool(procs)
    for k in range(args.warmup):
        pool.rate(1, it0=1000 + k)
    times, count = [], 0
    for k in range(args.steps):
        _, dt, n = pool.rate(args.ref_samples, it0=k + 1)
        times.append(dt)
        count += n
    pool.close()
    value = count / sum(times)
    sample = ("%d level-3 samples (+ level-2 partners) of the c3 workload per step, %d per process on %d "
              "processes (one per host core), rtol 1e-8" % (args.ref_samples * procs, args.ref_samples, procs))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "reference": "CPU FP64 oracle (numpy/scipy), bounded sample"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2606_09291_gb300 import distributed, inputs, mlsgd

    if world > 1:  # one rank compiles (in-tree outputs are shared), the others load after it
        if rank == 0:
            __graft_entry__.build()
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    else:
        __graft_entry__.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    cfg = workload_cfg(args)
    ctx = mlsgd.Context(**cfg)
    Nc = 8 << 3
    z_host = torch.tensor(inputs.z_test(Nc), dtype=torch.float64).pin_memory()
    z = z_host.to("cuda")
    S = args.samples
    level = 3
    stats = ctx.new_stats(level)
    first = rank * S  # weak scaling: each rank owns its own sample range

    def step(k):
        ctx.mlsgd_stats_reset(stats)
        ctx.mlsgd_level_gradient(k, level, first, S, z, stats)
        if world > 1:  # the level record of all ranks' samples (all-gather + the library's Chan merge)
            distributed.allgather_merge(ctx, stats)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up; the last warm-up step profiles every kernel class to find the dominant one
    for k in range(args.warmup):
        if k == args.warmup - 1:
            mlsgd.mlsgd_profile_start("*")
        step(k)
    torch.cuda.synchronize()
    prof_all = mlsgd.mlsgd_profile_stop()
    dominant = max(prof_all.items(), key=lambda kv: kv[1]["total_ms"])[0]
    total_prof = sum(v["total_ms"] for v in prof_all.values())
    h = stats.host()
    if h["noconv"] > 0:
        raise RuntimeError("warm-up: %d solves hit max_iter" % h["noconv"])

    # timed region
    sampler = ClockSampler(dev) if rank == 0 else None
    launches0 = mlsgd.mlsgd_launch_count()
    mlsgd.mlsgd_profile_start(dominant)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    ev[0].record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
        ev[k + 1].record(stream)
    barrier()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    prof = mlsgd.mlsgd_profile_stop().get(dominant)
    gpu_launches = mlsgd.mlsgd_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    ws_bytes = ctx.mlsgd_workspace_bytes(level, S)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = S * world * args.steps / (total_ms / 1e3)
    iters_per_sample = stats.host()["iters"] / S

    # end to end through the public API with host buffers: z H2D, stats D2H each step
    out_field = torch.empty(stats.field.numel(), dtype=torch.float64).pin_memory()
    out_sc = torch.empty(mlsgd.NSCALARS, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(e2e_steps):
        z.copy_(z_host, non_blocking=True)
        step(100 + k)
        out_field.copy_(stats.field, non_blocking=True)
        out_sc.copy_(stats.scalars, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = S * world * e2e_steps / (e2e_ms / 1e3)

    # plain FP64 path on the same batch (the metric's "vs plain FP64"): same sample
    # count per step, one warm-up step, then fp64_steps timed steps between barriers
    fp64 = None
    if args.fp64_samples > 0 and args.precision == "mixed":
        c64 = dict(cfg, precision="fp64", max_batch=min(args.fp64_chunk, args.fp64_samples), max_iter=200)
        ctx64 = mlsgd.Context(**c64)
        st64 = ctx64.new_stats(level)
        ctx64.mlsgd_level_gradient(0, level, first, args.fp64_samples, z, st64)  # warm-up
        barrier()
        fev = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps + 1)]
        fev[0].record(stream)
        for k in range(args.fp64_steps):
            ctx64.mlsgd_stats_reset(st64)
            ctx64.mlsgd_level_gradient(1 + k, level, first, args.fp64_samples, z, st64)
            fev[k + 1].record(stream)
        barrier()
        ms64 = fev[0].elapsed_time(fev[-1])
        if world > 1:
            t = torch.tensor([ms64], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms64 = float(t.item())
        fp64 = {"value": args.fp64_samples * world * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                "samples_per_step": args.fp64_samples, "steps": args.fp64_steps, "chunk": c64["max_batch"],
                "ms_per_step": ms64 / args.fp64_steps,
                "iters_per_sample": st64.host()["iters"] / args.fp64_samples}
        ctx64.close()

    # serving: the C4 mix (levels 0..5) through the continuous-batching server with its
    # HBM arena; estimates arrive all at once (saturation) and as a Poisson stream at
    # half that rate; latency from arrival to the last level's completion
    serve = None
    if args.serving and rank == 0 and world == 1:
        ctx.close()
        torch.cuda.empty_cache()
        serve = serving_leg(args)

    peaks, peak_kind = load_peaks()
    roof = None
    if prof and prof["launches"] > 0:
        per_launch_ms = prof["total_ms"] / prof["launches"]
        if dominant in ALU_PEAK and prof["flops"] > 0:
            peak, unit, kind = ALU_PEAK[dominant]
            ach = prof["flops"] / (prof["total_ms"] / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                    "traffic": None, "kernel": dominant, "peak_kind": kind}
        else:
            ach = prof["bytes"] / (prof["total_ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"],
                    "traffic": args.traffic_bytes if args.traffic_bytes is not None else (
                        TRAFFIC_RATIO[dominant] * prof["bytes"] / prof["launches"] if dominant in TRAFFIC_RATIO
                        else None),
                    "kernel": dominant, "peak_kind": peak_kind, "launches": prof["launches"],
                    "avg_launch_ms": per_launch_ms, "alg_bytes_per_launch": prof["bytes"] / prof["launches"],
                    "share_of_step": prof_all[dominant]["total_ms"] / total_prof}

    gemm = prof_all.get("kl_gemm")
    roof_gemm = None
    if gemm and gemm["launches"] > 0:
        tf = gemm["flops"] / (gemm["total_ms"] / 1e3) / 1e12
        roof_gemm = {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": tf / peaks["bf16_tflops"], "kernel": "kl_gemm (tcgen05, BF16 in / FP32 acc)",
                     "launches": gemm["launches"], "avg_launch_ms": gemm["total_ms"] / gemm["launches"],
                     "share_of_step": gemm["total_ms"] / total_prof, "peak_kind": peak_kind + " (burst)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r1, dt1 = oracle_rate(args.cpu_samples)
        single = {"value": r1, "cores": cpu_threads(),
                  "sample": "%d level-3 samples (+ level-2 partners) of this workload, rtol 1e-8, %.1f s" % (
                      args.cpu_samples, dt1)}
        procs = host_cores()
        pool = OraclePool(procs)
        r, dt, n = pool.rate(args.cpu_pool_samples, it0=1)
        pool.close()
        cpu = {"value": r, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": "%d level-3 samples (+ level-2 partners) of this workload, %d per process on %d processes "
                         "(one per host core; batches merged within each process), rtol 1e-8, %.1f s" % (
                             n, args.cpu_pool_samples, procs, dt),
               "single_thread": single}

    if rank == 0:
        sm = sorted(step_ms)
        p99 = sm[min(len(sm) - 1, int(np.ceil(0.99 * len(sm))) - 1)]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64 (bf16 coefficient)" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": workload_name(args), "samples_per_step_per_gpu": S, "level": level,
                           "partner_level": level - 1, "n_modes": 256, "l2": "inputs larger than L2 (batch working "
                           "set %.0f GB)" % (ws_bytes / 1e9),
                           "parallelism": ("samples sharded over ranks, records all-gathered and merged "
                                           "every step") if world > 1 else "single GPU",
                           "knobs": {k: cfg.get(k) for k in ("stencil", "z_chunks", "inner_iters",
                                                             "inner_iters_next", "omega", "ir_steps",
                                                             "max_batch")},
                           "knobs_source": "autotuner cache" if any(k in cfg for k in ("inner_iters", "omega"))
                           else "defaults"},
                "latency_ms": {"p50": statistics.median(step_ms), "p99": p99, "per": "step (one batch)"},
                "solver_iters_per_sample": iters_per_sample,
                "roofline": roof, "roofline_kl_gemm": roof_gemm, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": z.numel() * 8,
                        "d2h_bytes_per_step": (stats.field.numel() + mlsgd.NSCALARS) * 8},
                "gpu_launches": gpu_launches, "clocks": clocks, "fp64_path": fp64, "serving": serve,
                "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
                "kernel_shares": {k: round(v["total_ms"] / total_prof, 4) for k, v in
                                  sorted(prof_all.items(), key=lambda kv: -kv[1]["total_ms"])[:8]},
                # every class of the last warm-up step over 1% of it: algorithmic bytes per
                # second of its launches (CUDA events around each launch) against the HBM peak
                "kernel_roofline": {k: dict({"share": round(v["total_ms"] / total_prof, 4), "launches": v["launches"],
                                             "gbs": round(v["bytes"] / (v["total_ms"] / 1e3) / 1e9, 1),
                                             "frac": round(v["bytes"] / (v["total_ms"] / 1e3) / 1e9 /
                                                           peaks["hbm_gbs"], 3)},
                                            **({"alu": {"achieved": round(v["flops"] / (v["total_ms"] / 1e3) / 1e12, 3),
                                                        "peak": round(ALU_PEAK[k][0], 3), "unit": ALU_PEAK[k][1],
                                                        "frac": round(v["flops"] / (v["total_ms"] / 1e3) / 1e12 /
                                                                      ALU_PEAK[k][0], 3)}}
                                               if k in ALU_PEAK and v["flops"] > 0 else {}))
                                    for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1]["total_ms"])
                                    if v["total_ms"] > 0.01 * total_prof and v["bytes"] > 0}}
        print(json.dumps(line), flush=True)
    ctx.close()


def serving_leg(args):
    import numpy as np
    import torch

    from paper_2606_09291_gb300 import inputs, serving
    cfg, mix = serving.mix_config("c4")
    Nc = cfg["n0"] << (cfg["n_levels"] - 1)
    z = torch.tensor(inputs.z_test(Nc), dtype=torch.float64, device="cuda")
    srv = serving.ContinuousServer(cfg, args.serve_slots, [(l, m) for l, m in enumerate(mix)])
    srv.run(serving.poisson_mix_requests(mix, 2, 0.0, first_estimate=50000), z)  # warm-up
    sat = srv.run(serving.poisson_mix_requests(mix, args.serve_estimates, 0.0, first_estimate=60000), z)
    span = max(r["done"] for r in sat) - min(r["start"] for r in sat)
    cap = args.serve_estimates / span
    res = srv.run(serving.poisson_mix_requests(mix, args.serve_estimates, 0.5 * cap, seed=3, first_estimate=70000), z)
    est = {}
    for r in res:
        est.setdefault(r["estimate"], []).append(r)
    lat = [1e3 * (max(x["done"] for x in v) - v[0]["arrival"]) for v in est.values()]
    out = {"workload": "c4 mix %s over levels 0..5 (8^3 .. 256^3), K=128, theta 10, mixed, rtol 1e-8" % (list(mix),),
           "slots": args.serve_slots, "hbm_budget_bytes": srv.budget,
           "saturated_sample_gradients_per_s": cap * sum(mix), "saturated_estimates_per_s": cap,
           "device_overlap_saturated": serving.device_overlap(sat),
           "at_half_load": {"estimates_per_s": 0.5 * cap, "estimate_p50_ms": float(np.median(lat)),
                            "estimate_p99_ms": serving.pct(lat, 0.99), "deferred_by_hbm": srv.deferred},
           "estimates": args.serve_estimates}
    srv.close()
    return out


def parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-samples", type=int, default=4096,
                    help="samples per step of the plain FP64 leg (same batch as the mixed arm by default)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--fp64-chunk", type=int, default=1024, help="FP64 leg: samples per internal chunk")
    ap.add_argument("--cpu-samples", type=int, default=12, help="oracle samples of the one-thread leg (about 11 s)")
    ap.add_argument("--ref-samples", type=int, default=1, help="oracle samples per process per reference step")
    ap.add_argument("--cpu-pool-samples", type=int, default=8,
                    help="oracle samples per process, all-cores leg (about 10 s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ir-steps", type=int, default=0,
                    help="mixed path: 0 = refine until converged, launching only the samples still above rtol "
                         "(host check per step); k > 0 = exactly k masked steps (no host sync)")
    ap.add_argument("--no-tuned", action="store_true", help="default kernel and smoother knobs, not the tuned ones")
    ap.add_argument("--serving", type=int, default=1, help="1: also time the C4 serving mix (continuous batching)")
    ap.add_argument("--serve-slots", type=int, default=6)
    ap.add_argument("--serve-estimates", type=int, default=16)
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="ncu dram read+write bytes per launch of the dominant kernel, if captured")
    return ap


def main():
    args = parser().parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_gpu(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
