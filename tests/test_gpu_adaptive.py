"""GPU parity of the adaptive step size (eq:adaptive-step-size) and of the rate
diagnostics: a few MLSGD iterations through mlsgd_step_adaptive against the
oracle's MLSGD loop on the same draws (FP64 path, rtol 1e-13, <= 1e-10)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402

TOL64 = 1e-10


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("workload", ["expcov", "paper"])
def test_adaptive_steps_match_oracle(lib, workload):
    from paper_2606_09291_gb300 import driver
    if workload == "paper":
        cfg = dict(n_levels=3, n0=4, n_modes=27, corr_len=0.15, sigma=1.0, theta=8.0, alpha=1e-4, seed=3,
                   field_model=1, target_freq=2)
        z0 = inputs.z_test(16, freq=2)
    else:
        cfg = dict(n_levels=3, n0=4, n_modes=16, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=1)
        z0 = inputs.z_test(16)
    counts, iters, tau0 = (6, 4, 3), 3, 200.0
    ctx = lib.Context(**dict(cfg, rtol=1e-13, max_iter=400, precision="fp64"))
    z = torch.tensor(z0, dtype=torch.float64, device="cuda")
    hist = driver.run_mlsgd(ctx, z, counts, iters, tau0, adapt=False, step="adaptive", time_levels=True)
    W = mlmc.Workload(**{k: cfg[k] for k in ("n0", "n_levels", "n_modes", "corr_len", "sigma", "theta", "alpha",
                                             "seed")}, field_model=cfg.get("field_model", 0),
                      target_freq=cfg.get("target_freq", 1))
    z_ref, ref = mlmc.mlsgd(W, z0, counts, iters, tau0, adaptive=True)
    assert hist[0]["tau"] == tau0 and math.isnan(hist[0]["l_hat"])
    for g, r in zip(hist, ref):
        assert rel(g["grad_norm"], r["grad_norm"]) <= TOL64
        assert rel(g["objective"], r["objective"]) <= TOL64
        assert g["tau_fallback"] == int(r["fallback"])
        assert rel(g["tau"], r["tau"]) <= TOL64
        if not math.isnan(r["l_hat"]):
            assert rel(g["l_hat"], r["l_hat"]) <= TOL64
        assert rel(g["err_sam"], r["err_sam"]) <= 1e-8
        for key in ("m2_dx", "m2_dy", "mean_dx_norm", "mean_dy_abs"):
            for l in range(len(counts)):
                assert rel(g[key][l], r["rates"][key][l]) <= 1e-8, (key, l)
        for key in ("beta_x", "beta_y", "alpha_x", "alpha_y"):
            assert abs(g[key] - r["rates"][key]) <= 1e-7, key
        assert len(g["cost_per_sample_ms"]) == len(counts) and all(t > 0 for t in g["cost_per_sample_ms"])
    zg = z.cpu().numpy()
    assert np.abs(zg - z_ref).max() <= TOL64 * np.abs(z_ref).max()
    ctx.close()


def test_fixed_step_reports_tau(lib):
    ctx = lib.Context(n_levels=2, n0=4, n_modes=16, corr_len=0.3, sigma=1.0, theta=2.0, alpha=1e-4, seed=0,
                      rtol=1e-12)
    z = torch.tensor(inputs.z_test(8), dtype=torch.float64, device="cuda")
    st = [ctx.new_stats(l) for l in range(2)]
    for l in range(2):
        ctx.mlsgd_level_gradient(0, l, 0, 3, z, st[l])
    rep = ctx.mlsgd_step(st, 123.0, z)
    assert rep["tau"] == 123.0 and math.isnan(rep["l_hat"]) and rep["tau_fallback"] == 0
    # two levels: one difference level, so no exponent fits
    assert math.isnan(rep["beta_x"]) and math.isnan(rep["alpha_y"])
    g = torch.zeros_like(z)
    with pytest.raises(lib.MlsgdError):
        ctx.mlsgd_step_adaptive(st, -1.0, 0.0, z, g)
    ctx.close()


def test_stop_rules_and_count_cap(lib):
    from paper_2606_09291_gb300 import driver
    ctx = lib.Context(n_levels=3, n0=4, n_modes=16, corr_len=0.3, sigma=1.0, theta=2.0, alpha=1e-4, seed=0,
                      rtol=1e-8, precision="mixed")
    z = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    # gradient tolerance above any gradient: one iteration, its step taken
    h = driver.run_mlsgd(ctx, z, (4, 2), 5, 100.0, grad_tol=float("inf"))
    assert len(h) == 1 and torch.any(z != 0)
    # zero budget: one iteration
    h = driver.run_mlsgd(ctx, z, (4, 2), 5, 100.0, budget_s=0.0, step="adaptive")
    assert len(h) == 1
    # planned batches capped
    h = driver.run_mlsgd(ctx, z, (4, 2), 3, 100.0, count_cap=3, step="adaptive")
    assert all(m <= 3 for r in h[1:] for m in r["counts"])
    ctx.close()
