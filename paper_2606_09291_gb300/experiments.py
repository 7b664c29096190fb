"""The risk-aversion sweep of Sec. 5 on synthetic draws (the run behind the
paper's theta experiment, without its four-hour budget).

For every theta in {1, 8, 16, ..., 72} the paper's workload (cos-product field,
125 modes, rho = 0.15, xi ~ U(-4, 4), target prod sin(2 pi x_i), initial batches
{128, 16, 2} on the 16^3, 32^3 and 64^3 grids, one further level allowed) runs
adaptive MLSGD (eq:optimal-level, eq:optimal-batch-size, eq:adaptive-step-size,
eta = 0.9) from u_0 = 0 for a wall-clock budget per theta, and reports what the
paper plots: the objective and gradient norm at the last iterate, the number of
steps, the total samples per level, when the extra level was added, and the
rate exponents of the last batch.

    python -m paper_2606_09291_gb300.experiments --budget 30 --precision mixed

The same module runs the full FP64 MLSGD workload (run_c2):

    python -m paper_2606_09291_gb300.experiments --workload c2 --iterations 100 --log c2.jsonl
"""
import argparse
import json
import math
import sys

import torch

from . import driver, inputs, mlsgd


def paper_config(theta, precision="mixed", seed=0, rtol=None):
    p = dict(inputs.PRESETS["paper"])
    for k in ("counts", "thetas"):
        p.pop(k)
    p.update(theta=float(theta), seed=seed, precision=precision,
             rtol=(1e-8 if precision == "mixed" else 1e-10) if rtol is None else rtol, max_iter=400)
    return p


def run_theta(theta, budget_s, precision="mixed", max_iters=10000, count_cap=1 << 16, seed=0, log=None, tau0=1.0):
    cfg = paper_config(theta, precision, seed)
    ctx = mlsgd.Context(**cfg)
    try:
        Nc = cfg["n0"] << cfg["ctrl_level"]
        z = torch.zeros(Nc ** 3, dtype=torch.float64, device="cuda")
        hist = driver.run_mlsgd(ctx, z, inputs.PRESETS["paper"]["counts"], max_iters, tau0, eta=0.9,
                                max_levels=cfg["n_levels"], adapt=True, step="adaptive", time_levels=True,
                                budget_s=budget_s, count_cap=count_cap, log=log)
    finally:
        ctx.close()
    last = hist[-1]
    totals = [0] * cfg["n_levels"]
    level_added_s = None
    for h in hist:
        for l, m in enumerate(h["counts"]):
            totals[l] += m
        if level_added_s is None and len(h["counts"]) > len(hist[0]["counts"]):
            level_added_s = h["elapsed_s"]
    return dict(theta=theta, steps=len(hist), objective=last["objective"], risk=last["risk"],
                grad_norm=last["grad_norm"], elapsed_s=last["elapsed_s"], total_samples=totals,
                levels=len(last["counts"]), level_added_s=level_added_s, tau=last["tau"],
                beta_x=last["beta_x"], beta_y=last["beta_y"], alpha_x=last["alpha_x"], alpha_y=last["alpha_y"],
                gamma=last.get("gamma_hat", math.nan), cost_per_sample_ms=last.get("cost_per_sample_ms"))


def run_c2(iterations=100, log_path=None, checkpoint=None, resume=None, count_cap=1 << 14, precision="fp64"):
    """The full MLSGD workload c2: levels 0..4 (8^3 .. 128^3 cells), 128 KL modes of
    the exponential covariance (corr length 0.2, sigma 1), theta 10, alpha 1e-4,
    control on the 128^3 grid from u_0 = 0, the fixed step driver.fixed_step(alpha),
    adaptive level count and batch sizes (eq:optimal-level, eq:optimal-batch-size,
    eta = 0.9) from {128, 16, 2} on levels 0..2, `iterations` iterations, plain FP64.
    Writes one JSON line per iteration to log_path (driver.log_line); returns a
    summary of the history."""
    p = dict(inputs.PRESETS["c2"])
    counts = p.pop("counts")
    p.pop("iterations")
    p.update(precision=precision, rtol=1e-8, max_iter=400)
    ctx = mlsgd.Context(**p)
    try:
        Nc = p["n0"] << (p["n_levels"] - 1)
        z = torch.zeros(Nc ** 3, dtype=torch.float64, device="cuda")
        hist = driver.run_mlsgd(ctx, z, counts, iterations, driver.fixed_step(p["alpha"]), eta=0.9,
                                max_levels=p["n_levels"], adapt=True, step="fixed", time_levels=True,
                                count_cap=count_cap, log_path=log_path, checkpoint=checkpoint, resume=resume)
    finally:
        ctx.close()
    totals = [0] * p["n_levels"]
    for h in hist:
        for l, m in enumerate(h["counts"]):
            totals[l] += m
    pick = lambda h: dict(iteration=h["iteration"], objective=h["objective"], grad_norm=h["grad_norm"],  # noqa: E731
                          levels=len(h["counts"]), counts=h["counts"],
                          sqrt_mse=math.sqrt(max(h["err_sam"] + h["err_num"], 0.0)), elapsed_s=h["elapsed_s"])
    return dict(workload="c2", iterations=len(hist), count_cap=count_cap, precision=precision,
                total_samples=totals, first=pick(hist[0]), last=pick(hist[-1]),
                every_10th=[pick(h) for h in hist[::10]], elapsed_s=hist[-1]["elapsed_s"],
                levels_added_at=[h["iteration"] for a, h in zip(hist, hist[1:]) if len(h["counts"]) > len(a["counts"])])


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="sweep", choices=("sweep", "c2"),
                    help="sweep: the theta sweep of the paper's workload; c2: the full FP64 MLSGD run")
    ap.add_argument("--iterations", type=int, default=100, help="c2: MLSGD iterations")
    ap.add_argument("--log", default=None, help="c2: JSON-lines iteration log")
    ap.add_argument("--thetas", default=",".join(str(t) for t in inputs.PRESETS["paper"]["thetas"]))
    ap.add_argument("--budget", type=float, default=30.0, help="wall-clock seconds per theta")
    ap.add_argument("--precision", default="mixed", choices=("mixed", "fp64"))
    ap.add_argument("--max-iters", type=int, default=10000)
    ap.add_argument("--count-cap", type=int, default=1 << 16)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tau0", type=float, default=1.0,
                    help="first step; the adaptive rule sets the later ones")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.workload == "c2":
        print(json.dumps(run_c2(a.iterations, log_path=a.log, count_cap=a.count_cap)), flush=True)
        return 0
    for t in [float(x) for x in a.thetas.split(",")]:
        r = run_theta(t, a.budget, a.precision, a.max_iters, a.count_cap, a.seed, tau0=a.tau0)
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
