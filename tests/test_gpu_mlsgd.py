"""GPU parity of the multilevel combine, the adaptive plan and the MLSGD loop.

* the host controller of mlsgd_step, fed the GPU's level statistics, makes the
  same plan (level count and batch sizes, bit-exact) as the oracle's
  controller fed the same numbers (eq:sec-order-sum .. eq:mse-estimate-mlmc);
* three MLSGD iterations (Algorithm 1) with adaptive batch sizes follow the
  oracle's iterates (FP64 path, 1e-10) and its batch sizes (exactly);
* the large-risk-aversion workload (theta = 100, 512 modes, corr length 0.1,
  sigma = 1.5, mixed precision) on levels 0..2 matches the oracle within 1e-6.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import controller, mlmc  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _oracle(c):
    return mlmc.Workload(n0=8, n_levels=c["n_levels"], n_modes=c["n_modes"], corr_len=c["corr_len"], sigma=c["sigma"],
                         theta=c["theta"], alpha=c["alpha"], seed=c["seed"], rtol=1e-13)


def _info_from_gpu(stats, rep, theta):
    infos = []
    for l, st in enumerate(stats):
        h = st.host()
        infos.append(dict(n=int(h["count"]), shift=h["shift"], theta=theta, s2_x=h["s2_dx"], s2_y=h["s2_dy"],
                          mean_x_norm2=rep["mean_dx_norm2"][l], mean_y=h["mean_dy"]))
    return infos


def test_controller_matches_oracle(lib):
    cfg = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=10.0, alpha=1e-4, seed=3, rtol=1e-12,
               max_iter=400, precision="fp64")
    ctx = lib.Context(**cfg)
    z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    stats = [ctx.new_stats(l) for l in range(3)]
    for l, m in enumerate((16, 8, 4)):
        ctx.mlsgd_level_gradient(0, l, 0, m, z, stats[l])
    for max_levels in (3, 5):
        rep = ctx.mlsgd_step(stats, 0.0, z.clone(), eta=0.9, max_levels=max_levels)
        ref = controller.plan(_info_from_gpu(stats, rep, cfg["theta"]), EX_norm2=rep["ex_norm2"], EY=rep["ey"],
                              grad_norm=rep["grad_norm"], eta=0.9, n0=8, L_max=min(max_levels, 3))
        assert rep["next_levels"] == ref["L"]
        assert rep["next_counts"] == ref["M"]
        for k in ("err_sam", "err_num", "alpha_hat", "eps2"):
            assert abs(rep[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
        assert abs(rep["c_hat"] - ref["C_hat"]) <= 1e-13 * ref["C_hat"]
    ctx.close()


def test_mlsgd_iterations_match_oracle(lib):
    from paper_2606_09291_gb300 import driver
    cfg = dict(n_levels=2, n0=8, n_modes=32, corr_len=0.2, sigma=1.0, theta=10.0, alpha=1e-4, seed=0, rtol=1e-13,
               max_iter=400, precision="fp64", max_batch=64)
    ctx = lib.Context(**cfg)
    tau = driver.fixed_step(cfg["alpha"])
    z0 = inputs.z_random(16, seed=5, scale=30.0)
    z = torch.tensor(z0, dtype=torch.float64, device="cuda")
    hist = driver.run_mlsgd(ctx, z, counts=(8, 4), iterations=3, tau=tau, eta=0.9, max_levels=2)
    W = _oracle(cfg)
    zo = z0.copy()
    counts = [8, 4]
    for k in range(3):
        assert hist[k]["counts"] == counts, (k, hist[k]["counts"], counts)
        rs = [mlmc.level_batch(W, k, l, range(m), zo) for l, m in enumerate(counts)]
        out = mlmc.combine(W, [r["stats"] for r in rs], [r["shift"] for r in rs], zo, tau)
        assert abs(hist[k]["grad_norm"] - out["grad_norm"]) <= 1e-10 * out["grad_norm"]
        assert abs(hist[k]["risk"] - out["risk"]) <= 1e-10 * abs(out["risk"])
        infos = [dict(n=r["stats"].n, shift=r["shift"], theta=W.theta, s2_x=r["stats"].s2_x, s2_y=r["stats"].s2_y,
                      mean_x_norm2=W.hc3 * (r["stats"].mean_x @ r["stats"].mean_x), mean_y=r["stats"].mean_y)
                 for r in rs]
        plan = controller.plan(infos, EX_norm2=W.hc3 * (out["EX"] @ out["EX"]), EY=out["EY"],
                               grad_norm=out["grad_norm"], eta=0.9, n0=8, L_max=2)
        zo = out["z_new"]
        counts = plan["M"]
        assert hist[k]["next_counts"] == counts, (k, hist[k]["next_counts"], counts)
    assert rel_err(z.cpu().numpy(), zo) <= 1e-10
    ctx.close()


def test_large_risk_aversion_levels_0_to_2(lib):
    """theta = 100, 512 modes, corr length 0.1, sigma = 1.5, mixed precision (rtol 1e-8): the
    max-shifted FP64 weights and level-difference sums against the oracle on levels 0..2."""
    p = inputs.PRESETS["c5"]
    cfg = dict(n_levels=3, n0=8, n_modes=p["n_modes"], corr_len=p["corr_len"], sigma=p["sigma"], theta=p["theta"],
               alpha=p["alpha"], seed=p["seed"], rtol=1e-8, max_iter=50, precision="mixed")
    ctx = lib.Context(**cfg)
    W = _oracle(cfg)
    zn = inputs.z_test(32)
    z = torch.tensor(zn, dtype=torch.float64, device="cuda")
    counts = (6, 3, 2)
    stats, refs = [], []
    for l, m in enumerate(counts):
        st = ctx.new_stats(l)
        ctx.mlsgd_level_gradient(0, l, 0, m, z, st)
        stats.append(st)
        refs.append(mlmc.level_batch(W, 0, l, range(m), zn))
        h = st.host()
        assert h["count"] == m and h["noconv"] == 0
        # theta * Phi is O(1) here; compare in unshifted units
        fg, fo = math.exp(W.theta * h["shift"]), math.exp(W.theta * refs[-1]["shift"])
        assert rel_err(st.field.cpu().numpy() * fg, refs[-1]["stats"].mean_x * fo) <= 1e-6
        assert abs(h["mean_dy"] * fg - refs[-1]["stats"].mean_y * fo) <= 1e-6 * abs(refs[-1]["stats"].mean_y * fo)
    grad = torch.zeros_like(z)
    rep = ctx.mlsgd_step(stats, 1.0, z.clone(), grad=grad)
    out = mlmc.combine(W, [r["stats"] for r in refs], [r["shift"] for r in refs], zn, 1.0)
    assert rel_err(grad.cpu().numpy(), out["grad"]) <= 1e-6
    assert abs(rep["risk"] - out["risk"]) <= 1e-6 * abs(out["risk"])
    ctx.close()


@pytest.mark.parametrize("step", ["fixed", "adaptive"])
def test_resume_from_checkpoint_is_bit_exact(lib, tmp_path, step):
    """Four MLSGD iterations against two, a checkpoint, and two more from it: the
    counter-based draws make the resumed run repeat the uninterrupted one bit for bit
    (control, gradient norms, batch sizes and plans)."""
    from paper_2606_09291_gb300 import driver
    cfg = dict(n_levels=3, n0=8, n_modes=32, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=4, rtol=1e-10,
               max_iter=300, precision="fp64")
    tau = 0.5 if step == "adaptive" else driver.fixed_step(1e-4)
    runs = []
    for plan in (dict(iterations=4), dict(iterations=2, checkpoint=str(tmp_path / "ck.npz"))):
        ctx = lib.Context(**cfg)
        z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
        runs.append((driver.run_mlsgd(ctx, z, [8, 4, 2], tau=tau, step=step, count_cap=16, **plan), z))
        ctx.close()
    ctx = lib.Context(**cfg)
    z = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    tail = driver.run_mlsgd(ctx, z, [8], 4, tau=tau, step=step, count_cap=16, resume=str(tmp_path / "ck.npz"))
    ctx.close()
    (full, zf), (head, _) = runs
    assert torch.equal(z, zf)
    for a, b in zip(full, head + tail):
        assert a["iteration"] == b["iteration"] and a["counts"] == b["counts"]
        assert a["grad_norm"] == b["grad_norm"] and a["next_counts"] == b["next_counts"] and a["tau"] == b["tau"]
