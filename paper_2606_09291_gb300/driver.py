"""MLSGD outer loop over the C ABI (Algorithm 1, function MLSGD).

Orchestration only: each iteration calls mlsgd_level_gradient for every
level with the current batch sizes (fresh draws per iteration, sample
identity (seed, iteration, level, index)) and mlsgd_step, which combines the
levels, takes the projected gradient step and plans the next level count
and batch sizes (eq:optimal-level, eq:optimal-batch-size), with a fixed or
the adaptive step size (eq:adaptive-step-size).  All arithmetic of the method
runs in libmlsgd; the host only fits the exponent of the measured cost per
sample when asked to time the levels.
"""
import json
import math
import os
import time

import numpy as np
import torch

from . import mlsgd


def fixed_step(alpha):
    """Fixed step of the MLSGD workload: tau = 0.5 / (alpha + (3 pi^2)^-2), the
    'alpha-scaled' step read so that |1 - tau (alpha + ||S||^2)| < 1 for a ~ 1."""
    import math
    return 0.5 / (alpha + (3.0 * math.pi ** 2) ** -2)


def _event():
    return torch.cuda.Event(enable_timing=True)


def _slope(ls, vals):
    """Least-squares slope of log2(vals) against ls (NaN with fewer than two points)."""
    if len(ls) < 2:
        return float("nan")
    x = [float(l) for l in ls]
    y = [math.log2(v) if v > 0 else float("nan") for v in vals]
    xm, ym = sum(x) / len(x), sum(y) / len(y)
    return sum((a - xm) * (b - ym) for a, b in zip(x, y)) / sum((a - xm) ** 2 for a in x)


# ---------------------------------------------------------------- checkpoint and log
# A checkpoint holds everything the next iteration depends on: the iteration index
# k, the control u_k, the planned batch sizes {M_{k,l}} (their number is L_k), the
# previous step size and gradient of the adaptive rule, the elapsed time and the
# seed.  Sample identity is (seed, iteration, level, index), so an MLSGD run resumed
# from it repeats bit for bit what the uninterrupted run computes.
def save_checkpoint(path, k_next, z, counts, tau_prev, g_prev, elapsed_s, seed):
    meta = dict(k_next=int(k_next), counts=[int(m) for m in counts], tau_prev=float(tau_prev),
                elapsed_s=float(elapsed_s), seed=int(seed), adaptive=g_prev is not None)
    tmp = path + ".tmp.npz"
    np.savez(tmp, z=z.detach().cpu().numpy(),
             g_prev=(g_prev.detach().cpu().numpy() if g_prev is not None else np.zeros(0)),
             meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8))
    os.replace(tmp, path)


def load_checkpoint(path):
    with np.load(path) as f:
        meta = json.loads(bytes(f["meta"]).decode())
        meta["z"] = f["z"].copy()
        meta["g_prev"] = f["g_prev"].copy() if meta["adaptive"] else None
    return meta


def log_line(rep):
    """One JSON line per iteration with the quantities of the paper's Sec. 5.1
    figures: objective J^ML(u_k), ||grad J^ML||, batch sizes per level, the rate
    estimates (alpha, beta per X and Y, gamma when timed), the error bar
    sqrt(MSE) = sqrt(err_sam + err_num) (eq:mse-estimate-mlmc), the step."""
    keys = ("iteration", "objective", "risk", "grad_norm", "counts", "next_levels", "next_counts", "err_sam", "err_num",
            "alpha_hat", "alpha_x", "alpha_y", "beta_x", "beta_y", "gamma_hat", "tau", "l_hat", "tau_fallback",
            "truncated", "elapsed_s", "level_ms")
    line = {k: rep[k] for k in keys if k in rep}
    line["sqrt_mse"] = math.sqrt(max(rep["err_sam"] + rep["err_num"], 0.0))
    return json.dumps(line)


def run_mlsgd(ctx, z, counts, iterations, tau, eta=0.9, max_levels=None, adapt=True, stream=None, log=None,
              step="fixed", time_levels=False, grad_tol=None, budget_s=None, count_cap=None, checkpoint=None,
              resume=None, log_path=None):
    """Run `iterations` MLSGD steps from control z (device FP64 tensor, updated in
    place).  counts: initial per-level batch sizes (levels 0..len-1).
    step: "fixed" (tau every iteration) or "adaptive" (eq:adaptive-step-size with
    tau_0 = tau; mlsgd_step_adaptive keeps the previous gradient in a device buffer).
    time_levels: time each level's batch with CUDA events and report the cost per
    sample and its exponent gamma_hat (eq:assumption_gamma, cost ~ h_l^-gamma,
    fitted over l >= 1; this synchronises after every level).
    Stops after `iterations` steps, or earlier once the gradient norm of an
    iteration is <= grad_tol (the loop condition of Algorithm 1, MLSGD; that
    iteration's step is still taken, so the result is u_{k+1}), or once budget_s
    wall-clock seconds have passed at the end of an iteration (a plain time budget:
    the budgeting scheme the paper cites for choosing its tolerance is not restated).
    count_cap: optional upper bound on every planned batch size.
    checkpoint: path written after every iteration (save_checkpoint); resume: path of
    a checkpoint to continue from (iterations counts from its k; z is overwritten
    with its control); log_path: JSON-lines file, one log_line per iteration
    (appended).
    With budget_s and adapt, the planned batches of the next iteration are scaled
    down together (keeping their ratios, at least 2 each) when their estimated
    time, from this iteration's measured cost per sample (a new level: 8 times the
    last), exceeds the budget left; this turns on time_levels.
    Returns the list of per-iteration reports (host dicts)."""
    assert step in ("fixed", "adaptive")
    if budget_s is not None and adapt:
        time_levels = True
    max_levels = ctx.cfg["n_levels"] if max_levels is None else max_levels
    counts = list(counts)
    history = []
    stats = [ctx.new_stats(l) for l in range(ctx.cfg["n_levels"])]
    g_prev = torch.zeros_like(z) if step == "adaptive" else None
    tau_prev = 0.0
    k0, elapsed0 = 0, 0.0
    if resume is not None:
        st = load_checkpoint(resume)
        if st["seed"] != ctx.cfg.get("seed", st["seed"]) or st["adaptive"] != (step == "adaptive"):
            raise ValueError("checkpoint is of another run (seed or step rule differ)")
        k0, counts, tau_prev, elapsed0 = st["k_next"], st["counts"], st["tau_prev"], st["elapsed_s"]
        z.copy_(torch.as_tensor(st["z"], dtype=z.dtype))
        if g_prev is not None:
            g_prev.copy_(torch.as_tensor(st["g_prev"], dtype=z.dtype))
    strm = stream if stream is not None or not time_levels else torch.cuda.current_stream()
    t0 = time.perf_counter() - elapsed0
    for k in range(k0, iterations):
        level_ms = []
        for l, m in enumerate(counts):
            ctx.mlsgd_stats_reset(stats[l], stream=stream)
            if time_levels:
                e0, e1 = _event(), _event()
                e0.record(strm)
            ctx.mlsgd_level_gradient(k, l, 0, m, z, stats[l], stream=stream)
            if time_levels:
                e1.record(strm)
                e1.synchronize()
                level_ms.append(e0.elapsed_time(e1))
        if step == "adaptive":
            rep = ctx.mlsgd_step_adaptive(stats[:len(counts)], tau, tau_prev, z, g_prev, eta=eta,
                                          max_levels=max_levels, stream=stream)
            tau_prev = rep["tau"]
        else:
            rep = ctx.mlsgd_step(stats[:len(counts)], tau, z, eta=eta, max_levels=max_levels, stream=stream)
        rep["iteration"] = k
        rep["counts"] = list(counts)
        if time_levels:
            rep["level_ms"] = level_ms
            rep["cost_per_sample_ms"] = [t / m for t, m in zip(level_ms, counts)]
            rep["gamma_hat"] = _slope(range(1, len(counts)), rep["cost_per_sample_ms"][1:])
        history.append(rep)
        rep["elapsed_s"] = time.perf_counter() - t0
        if log is not None:
            log(rep)
        if log_path is not None:
            with open(log_path, "a") as f:
                f.write(log_line(rep) + "\n")
        if adapt:
            counts = list(rep["next_counts"])
            if count_cap is not None:
                counts = [min(m, count_cap) for m in counts]
            if budget_s is not None:
                cps = list(rep["cost_per_sample_ms"])
                while len(cps) < len(counts):
                    cps.append(8.0 * cps[-1])
                left_ms = 1000.0 * (budget_s - rep["elapsed_s"])
                est_ms = sum(m * c for m, c in zip(counts, cps))
                if left_ms > 0 and est_ms > left_ms:
                    f = left_ms / est_ms
                    counts = [max(2, int(m * f)) for m in counts]
        if checkpoint is not None:
            save_checkpoint(checkpoint, k + 1, z, counts, tau_prev, g_prev, rep["elapsed_s"],
                            ctx.cfg.get("seed", 0))
        if grad_tol is not None and rep["grad_norm"] <= grad_tol:
            break
        if budget_s is not None and rep["elapsed_s"] >= budget_s:
            break
    return history
