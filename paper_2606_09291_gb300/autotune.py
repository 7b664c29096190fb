"""Autotuner of the solver's kernel and smoother choices for one level's batch.

The knobs change how a batch of level-l samples is solved, never what a
converged solve returns beyond the solver tolerance (the level record stays
within the mixed path's 1e-6 of the oracle for every choice; tests/
test_gpu_autotune.py checks each one):

* stencil      0 = whole-row slab passes on 32^3 / 64^3 grids, 1 = z-marching tiles
* z_chunks     z chunks per sample in the fused passes (0 = chosen from the batch)
* batch_chunks the level batch is solved in this many sequential sub-batches
               (the context's max_batch = ceil(S / batch_chunks))
* inner_iters  FP32 PCG iterations per refinement step
* omega        damping of the Jacobi smoother of the V-cycle
* ir_steps     0 = refine until every sample converges (host check per step, the
               still-active samples compacted); k > 0 = exactly k masked steps
               (no host round trip; rejected when a sample is left unconverged)
* inner_iters_next  inner iterations of the refinement steps after the first, which
               start from a residual the first step has already reduced (0 = inner_iters)

Search: time candidate configurations on a probe batch of the level with CUDA
events (one warm-up call, then `reps` timed calls of mlsgd_level_gradient), keep
only candidates whose solves all converge, and go coordinate-wise: launch shape
(stencil x z_chunks x batch_chunks) first, then the smoother schedule (inner_iters x
omega), then the refinement schedule (ir_steps x inner_iters_next).  The cost is time per converged sample-gradient.  Winners are
stored per (grid, batch size, precision, modes) in a JSON cache; a cached entry is
returned as is, so a run is deterministic given its cache.  The paper's own
analogue is choosing the batch width per level by memory and cost (Sec. 4.2,
eq:optimal-parallelization); here the GPU's launch and smoother choices are picked
by measurement.

    python -m paper_2606_09291_gb300.autotune --preset c3 --level 3 --samples 4096
"""
import argparse
import itertools
import json
import os

import torch

from . import mlsgd

KNOBS = ("stencil", "z_chunks", "batch_chunks", "inner_iters", "omega", "ir_steps", "inner_iters_next")
DEFAULTS = dict(stencil=0, z_chunks=0, batch_chunks=1, inner_iters=6, omega=0.6, ir_steps=0, inner_iters_next=0)
SHAPES = dict(stencil=(0, 1), z_chunks=(0, 1, 2, 4), batch_chunks=(1, 2, 4))
SCHEDULES = dict(inner_iters=(4, 5, 6, 7, 8), omega=(0.5, 0.6, 0.7), ir_steps=(0, 2, 3),
                 inner_iters_next=(0, 3, 4, 5))
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def key(cfg, level, n_samples):
    N = cfg.get("n0", 8) << level
    prec = cfg.get("precision", "fp64")
    prec = {0: "fp64", 1: "mixed"}.get(prec, prec)
    return "N%d-S%d-%s-K%d" % (N, n_samples, prec, cfg.get("n_modes", 0))


def load_cache(path=CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def context_cfg(base_cfg, knobs, n_samples):
    """The context configuration of base_cfg with the knobs applied to batches of
    n_samples (knobs missing from an older cache entry take their defaults)."""
    k = dict(DEFAULTS, **knobs)
    cfg = dict(base_cfg)
    cfg.update({name: k[name] for name in KNOBS if name != "batch_chunks"})
    cfg["max_batch"] = max(1, -(-n_samples // k["batch_chunks"]))
    return cfg


def lookup(cfg, level, n_samples, path=CACHE):
    """The tuned knobs for this batch (all of KNOBS), or None (no entry: use DEFAULTS)."""
    e = load_cache(path).get(key(cfg, level, n_samples))
    return dict(DEFAULTS, **e["knobs"]) if e else None


def measure(base_cfg, knobs, level, n_samples, z, reps=2, it0=1000):
    """ms per sample-gradient of knobs on a batch of n_samples, and whether every solve converged."""
    ctx = mlsgd.Context(**context_cfg(base_cfg, knobs, n_samples))
    st = ctx.new_stats(level)
    ctx.mlsgd_level_gradient(it0, level, 0, n_samples, z, st)  # warm-up (scratch, kernels)
    noconv = st.host()["noconv"]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for r in range(reps):
        ctx.mlsgd_stats_reset(st)
        ctx.mlsgd_level_gradient(it0 + 1 + r, level, 0, n_samples, z, st)
        noconv += st.host()["noconv"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps * n_samples)
    iters = st.host()["iters"] / n_samples
    ctx.close()
    return dict(ms_per_sample=ms, noconv=int(noconv), iters_per_sample=iters)


def tune(base_cfg, level, n_samples, z, probe=None, reps=2, cache_path=CACHE, log=None, retune=False):
    """Pick the knobs for batches of n_samples on `level` (timed on a probe batch of
    min(n_samples, probe) samples).  Returns (knobs, report); report["source"] is
    "cache" when the entry came from the cache."""
    k = key(base_cfg, level, n_samples)
    cache = load_cache(cache_path) if cache_path else {}
    if k in cache and not retune:
        return dict(cache[k]["knobs"]), dict(cache[k], source="cache")
    m = min(n_samples, probe) if probe else n_samples
    tried = []

    def run(knobs):
        r = measure(base_cfg, knobs, level, m, z, reps)
        r["knobs"] = dict(knobs)
        tried.append(r)
        if log:
            log(r)
        return r

    def best(rs):
        ok = [r for r in rs if r["noconv"] == 0]
        return min(ok, key=lambda r: r["ms_per_sample"]) if ok else None

    shape = best([run(dict(DEFAULTS, stencil=s, z_chunks=c, batch_chunks=b))
                  for s, c, b in itertools.product(SHAPES["stencil"], SHAPES["z_chunks"], SHAPES["batch_chunks"])])
    if shape is None:
        raise RuntimeError("autotune: no launch shape converged")
    sched = best([run(dict(shape["knobs"], inner_iters=i, omega=w))
                  for i, w in itertools.product(SCHEDULES["inner_iters"], SCHEDULES["omega"])])
    win = sched if sched is not None and sched["ms_per_sample"] < shape["ms_per_sample"] else shape
    refine = best([run(dict(win["knobs"], ir_steps=k, inner_iters_next=i2))
                   for k, i2 in itertools.product(SCHEDULES["ir_steps"], SCHEDULES["inner_iters_next"])])
    if refine is not None and refine["ms_per_sample"] < win["ms_per_sample"]:
        win = refine
    entry = dict(knobs=win["knobs"], ms_per_sample=win["ms_per_sample"], probe_samples=m,
                 default_ms_per_sample=next(r["ms_per_sample"] for r in tried if r["knobs"] == DEFAULTS),
                 candidates=len(tried), device=torch.cuda.get_device_name())
    if cache_path:
        cache[k] = entry
        with open(cache_path + ".tmp", "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(cache_path + ".tmp", cache_path)
    return dict(win["knobs"]), dict(entry, source="measured")


def main():
    from . import inputs
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", default="c3")
    ap.add_argument("--level", type=int, default=3)
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--probe", type=int, default=1024)
    ap.add_argument("--cache", default=CACHE)
    ap.add_argument("--retune", action="store_true")
    args = ap.parse_args()
    p = dict(inputs.PRESETS[args.preset])
    cfg = dict(n_levels=p["n_levels"], n0=p["n0"], n_modes=p["n_modes"], corr_len=p["corr_len"], sigma=p["sigma"],
               theta=p["theta"], alpha=p["alpha"], seed=p["seed"], rtol=1e-8, max_iter=50,
               precision=p.get("precision", "mixed"), field_tc=1, ctrl_level=p["n_levels"] - 1)
    z = torch.tensor(inputs.z_test(p["n0"] << (p["n_levels"] - 1)), dtype=torch.float64, device="cuda")
    knobs, rep = tune(cfg, args.level, args.samples, z, probe=args.probe, cache_path=args.cache, retune=args.retune,
                      log=lambda r: print(json.dumps(r), flush=True))
    print(json.dumps(dict(knobs=knobs, **{k: v for k, v in rep.items() if k != "knobs"})))


if __name__ == "__main__":
    main()
