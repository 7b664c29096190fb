"""Parity at the full size of the benchmark workload, in the configuration the
benchmark times (bench.workload_cfg with the benchmark's default arguments):
4096 level-3 samples (64^3 cells) with their level-2 partners, 256 KL modes,
mixed precision at rtol 1e-8, one batch of 4096 per call.

(a) The timed call itself, mlsgd_level_gradient over samples 0..4095 of step 0,
    against the oracle's record of the same samples (tests/golden/
    c3_level3_record.npz, written by tests/golden/make_c3_record.py, which calls
    only oracle/; oracle solves at rtol 1e-12): count bit-exact, the mean of dX~
    element by element, the mean of dY~ and both second-order sums within the
    mixed path's bar 1e-6, compared in unshifted units.
(b) The same full-batch field and solve through mlsgd_solve_state_adjoint against
    the oracle on sampled samples (first, middle, last): xi and log a to rounding;
    the state and adjoint solutions through the solver's contract,
    ||b - A y|| <= rtol ||b|| with the oracle's assembled operator on the
    coefficient the mixed path solves with (exp(log a) rounded to FP32), and
    against the oracle's own solutions (rtol 1e-12) at the mixed path's bar (1e-6);
    Phi from the returned state.
(c) The full-batch level record equals the Chan merge of the records of its two
    halves (each sample's contribution depends only on its identity; the level
    differences are accumulated in FP64), a property that holds at any size.
Named to run after the other GPU tests (they are cheaper and say more when they
fail); the allocation-free entry point's test stays last."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402
from oracle import mlmc, philox  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402

S = 4096
LEVEL = 3
SAMPLED = (0, 2047, 4095)
RTOL = 1e-8
TOLMIX = 1e-6


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3_level3_record.npz")


def bench_cfg():
    args = bench.parser().parse_args([])
    assert args.samples == S and args.precision == "mixed"
    return bench.workload_cfg(args)


def test_timed_call_matches_oracle_record(lib):
    ref = np.load(GOLDEN)
    assert int(ref["count"]) == S and int(ref["level"]) == LEVEL and int(ref["first_sample"]) == 0
    cfg = bench_cfg()
    ctx = lib.Context(**cfg)
    zt = torch.tensor(inputs.z_test(8 << LEVEL), dtype=torch.float64, device="cuda")
    st = ctx.new_stats(LEVEL)
    ctx.mlsgd_level_gradient(int(ref["iteration"]), LEVEL, 0, S, zt, st)
    h = st.host()
    field = st.field.cpu().numpy()
    ctx.close()
    assert h["count"] == S and h["noconv"] == 0
    theta = cfg["theta"]
    fg, fo = np.exp(theta * h["shift"]), np.exp(theta * float(ref["shift"]))
    my = float(ref["mean_y"]) * fo
    err = {"shift": abs(h["shift"] - float(ref["shift"])) / abs(float(ref["shift"])),
           "mean_dx": rel_err(field * fg, ref["mean_x"] * fo),
           "mean_dy": abs(h["mean_dy"] * fg - my) / abs(my)}
    for k_gpu, k_ref in (("s2_dx", "s2_x"), ("s2_dy", "s2_y")):
        r = float(ref[k_ref]) * fo ** 2
        err[k_gpu] = abs(h[k_gpu] * fg ** 2 - r) / r
    print("measured relative error per result (4096-sample timed call vs oracle):",
          {k: "%.2e" % v for k, v in err.items()})
    for k, v in err.items():
        assert v <= TOLMIX, (k, v)


def oracle_workload():
    p = inputs.PRESETS["c3"]
    return mlmc.Workload(n0=p["n0"], n_levels=p["n_levels"], n_modes=p["n_modes"], corr_len=p["corr_len"],
                         sigma=p["sigma"], theta=p["theta"], alpha=p["alpha"], seed=p["seed"], rtol=1e-12)


def rel_err(gpu, ref):
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return np.abs(gpu - ref).max() / (scale if scale > 0 else 1.0)


def test_full_batch_solve_on_sampled_samples(lib):
    cfg = bench_cfg()
    assert cfg["max_batch"] == S and cfg["precision"] == "mixed" and cfg["rtol"] == RTOL
    ctx = lib.Context(**cfg)
    N, K = 8 << LEVEL, cfg["n_modes"]
    z = inputs.z_test(N)
    zt = torch.tensor(z, dtype=torch.float64, device="cuda")
    xi = torch.zeros(S, K, dtype=torch.float64, device="cuda")
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    ctx.mlsgd_sample_field(0, LEVEL, LEVEL, 0, S, xi=xi, log_a=la)
    nn = (N + 1) ** 3
    y = torch.zeros(S, nn, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(y)
    phi = torch.zeros(S, dtype=torch.float64, device="cuda")
    it = torch.zeros(S, dtype=torch.int32, device="cuda")
    stt = torch.zeros(S, dtype=torch.int32, device="cuda")
    st = ctx.mlsgd_solve_state_adjoint(LEVEL, S, la, zt, y, q, phi, it, stt)
    assert st == 0, ctx.L.mlsgd_last_error(ctx.h)
    assert int(stt.sum()) == 0 and int(it.min()) > 0
    idx = torch.tensor(SAMPLED, device="cuda")
    xs, las = xi[idx].cpu().numpy(), la[idx].cpu().numpy()
    ys, qs, phis = y[idx].cpu().numpy(), q[idx].cpu().numpy(), phi[idx].cpu().numpy()
    del xi, la, y, q
    torch.cuda.empty_cache()
    ctx.close()

    W = oracle_workload()
    lev = W.level(LEVEL)
    I = lev.interior
    b = W.rhs_state(z, LEVEL)
    ref_xi = philox.normals(W.seed, 0, LEVEL, np.array(SAMPLED), K)
    assert np.abs(xs - ref_xi).max() <= 4e-15 * np.abs(ref_xi).max()
    err = {"y": 0.0, "q": 0.0, "phi": 0.0, "res_y/rtol": 0.0, "res_q/rtol": 0.0}
    for k, m in enumerate(SAMPLED):
        assert rel_err(las[k], W.log_a(ref_xi[k][None], LEVEL)[0]) <= 1e-12
        # the operator the mixed path solves with: the coefficient rounded to FP32
        a32 = np.exp(las[k]).astype(np.float32).astype(np.float64)
        A32 = lev.restrict(lev.stiffness(a32))
        ry = b[I] - A32 @ ys[k][I]
        assert np.linalg.norm(ry) <= 1.05 * RTOL * np.linalg.norm(b[I])
        e = ys[k] - lev.g
        Me = lev.M_full @ e
        assert abs(phis[k] - 0.5 * e @ Me) <= 1e-12 * abs(0.5 * e @ Me)
        rq = Me[I] - A32 @ qs[k][I]
        assert np.linalg.norm(rq) <= 1.05 * RTOL * np.linalg.norm(Me[I])
        # against the oracle's own solutions (FP64 coefficient, rtol 1e-12)
        ref = W.solve_state_adjoint(las[k], z, LEVEL)
        e_k = {"y": rel_err(ys[k], ref["y"]), "q": rel_err(qs[k], ref["q"]),
               "phi": abs(phis[k] - ref["phi"]) / abs(ref["phi"]),
               "res_y/rtol": np.linalg.norm(ry) / (RTOL * np.linalg.norm(b[I])),
               "res_q/rtol": np.linalg.norm(rq) / (RTOL * np.linalg.norm(Me[I]))}
        err = {key: max(err[key], v) for key, v in e_k.items()}
        assert e_k["y"] <= TOLMIX and e_k["q"] <= TOLMIX and e_k["phi"] <= TOLMIX
    print("measured error per result over the sampled samples (max):", {k: "%.2e" % v for k, v in err.items()})


def test_full_batch_record_equals_merged_halves(lib):
    cfg = bench_cfg()
    ctx = lib.Context(**cfg)
    zt = torch.tensor(inputs.z_test(8 << LEVEL), dtype=torch.float64, device="cuda")
    theta = cfg["theta"]
    full = ctx.new_stats(LEVEL)
    ctx.mlsgd_level_gradient(7, LEVEL, 0, S, zt, full)
    half = ctx.new_stats(LEVEL)
    ctx.mlsgd_level_gradient(7, LEVEL, 0, S // 2, zt, half)
    other = ctx.new_stats(LEVEL)
    ctx.mlsgd_level_gradient(7, LEVEL, S // 2, S // 2, zt, other)
    ctx.mlsgd_stats_merge(half, other)
    hf, hm = full.host(), half.host()
    assert hf["count"] == hm["count"] == S and hf["noconv"] == hm["noconv"] == 0
    ff = full.field.cpu().numpy() * np.exp(theta * hf["shift"])
    fm = half.field.cpu().numpy() * np.exp(theta * hm["shift"])
    assert rel_err(fm, ff) <= 1e-12
    gf, gm = np.exp(theta * hf["shift"]), np.exp(theta * hm["shift"])
    assert abs(hm["mean_dy"] * gm - hf["mean_dy"] * gf) <= 1e-12 * abs(hf["mean_dy"] * gf)
    assert abs(hm["s2_dx"] * gm ** 2 - hf["s2_dx"] * gf ** 2) <= 1e-10 * hf["s2_dx"] * gf ** 2
    assert abs(hm["s2_dy"] * gm ** 2 - hf["s2_dy"] * gf ** 2) <= 1e-10 * hf["s2_dy"] * gf ** 2
    ctx.close()
