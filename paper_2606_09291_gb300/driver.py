"""MLSGD outer loop over the C ABI (Algorithm 1, function MLSGD).

Orchestration only: each iteration calls mlsgd_level_gradient for every
level with the current batch sizes (fresh draws per iteration, sample
identity (seed, iteration, level, index)) and mlsgd_step, which combines the
levels, takes the projected gradient step and plans the next level count
and batch sizes (eq:optimal-level, eq:optimal-batch-size).  All arithmetic
runs in libmlsgd.
"""
import torch

from . import mlsgd


def fixed_step(alpha):
    """Fixed step of the MLSGD workload: tau = 0.5 / (alpha + (3 pi^2)^-2), the
    'alpha-scaled' step read so that |1 - tau (alpha + ||S||^2)| < 1 for a ~ 1."""
    import math
    return 0.5 / (alpha + (3.0 * math.pi ** 2) ** -2)


def run_mlsgd(ctx, z, counts, iterations, tau, eta=0.9, max_levels=None, adapt=True, stream=None, log=None):
    """Run `iterations` MLSGD steps from control z (device FP64 tensor, updated in
    place).  counts: initial per-level batch sizes (levels 0..len-1).
    Returns the list of per-iteration reports (host dicts)."""
    max_levels = ctx.cfg["n_levels"] if max_levels is None else max_levels
    counts = list(counts)
    history = []
    stats = [ctx.new_stats(l) for l in range(ctx.cfg["n_levels"])]
    for k in range(iterations):
        for l, m in enumerate(counts):
            ctx.mlsgd_stats_reset(stats[l], stream=stream)
            ctx.mlsgd_level_gradient(k, l, 0, m, z, stats[l], stream=stream)
        rep = ctx.mlsgd_step(stats[:len(counts)], tau, z, eta=eta, max_levels=max_levels, stream=stream)
        rep["iteration"] = k
        rep["counts"] = list(counts)
        history.append(rep)
        if log is not None:
            log(rep)
        if adapt:
            counts = list(rep["next_counts"])
    return history
