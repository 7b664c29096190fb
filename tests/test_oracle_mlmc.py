"""Pins of the oracle's estimator: gradient, entropic limits, telescoping, Chan merge."""
import numpy as np
import pytest

from oracle import controller, mlmc


def _ctrl_field(Nc, kind, seed=0):
    c = np.arange(Nc ** 3)
    x, y, z = (c % Nc + 0.5) / Nc, ((c // Nc) % Nc + 0.5) / Nc, (c // Nc ** 2 + 0.5) / Nc
    if kind == "test":
        return 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    rng = np.random.default_rng(seed)
    return rng.standard_normal(Nc ** 3)


def _small(theta=5.0, sigma=1.0, n0=4, n_levels=1, **kw):
    return mlmc.Workload(n0=n0, n_levels=n_levels, n_modes=16, corr_len=0.3, sigma=sigma,
                         theta=theta, alpha=1e-2, seed=7, **kw)


def _objective(W, z, xis, level=0):
    """Sampled single-level objective J_N(z) = theta^-1 log(mean exp(theta Phi_m)) + alpha/2 ||z||_U^2."""
    phis = np.array([W.solve_state_adjoint(W.log_a(x[None], level)[0], z, level)["phi"] for x in xis])
    c = phis.max()
    return c + np.log(np.mean(np.exp(W.theta * (phis - c)))) / W.theta + 0.5 * W.alpha * W.hc3 * (z @ z)


def _single_level_grad(W, z, samples):
    r = mlmc.level_batch(W, 0, 0, samples, z)
    return mlmc.combine(W, [r["stats"]], [r["shift"]], z, tau=0.0), r


@pytest.mark.parametrize("theta", [0.5, 20.0])
def test_gradient_matches_finite_differences(theta):
    W = _small(theta=theta)
    z = _ctrl_field(W.Nc, "test") + 5.0 * _ctrl_field(W.Nc, "rand", 1)
    samples = list(range(4))
    out, _ = _single_level_grad(W, z, samples)
    xis = W.xi(0, 0, samples)
    for seed in (2, 3):
        dz = _ctrl_field(W.Nc, "rand", seed)
        dz /= np.sqrt(W.hc3 * (dz @ dz))
        eps = 1e-4
        fd = (_objective(W, z + eps * dz, xis) - _objective(W, z - eps * dz, xis)) / (2 * eps)
        an = W.hc3 * (out["grad"] @ dz)
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3), (fd, an)


def test_theta_to_zero_gives_the_mean():
    z = _ctrl_field(4, "test")
    samples = list(range(6))
    W = _small(theta=1e-8)
    out, r = _single_level_grad(W, z, samples)
    mean_bq = np.mean([p["fine"]["bq"] for p in r["per_sample"]], axis=0)
    assert np.abs(out["grad"] - (mean_bq + W.alpha * z)).max() < 1e-9 * np.abs(mean_bq).max()
    # R_theta = mean + theta/2 var + O(theta^2) for the empirical measure
    W = _small(theta=1e-2)
    out, r = _single_level_grad(W, z, samples)
    phis = np.array([p["fine"]["phi"] for p in r["per_sample"]])
    approx = phis.mean() + 0.5 * W.theta * phis.var()
    assert abs(out["risk"] - approx) < 10 * W.theta ** 2 * np.abs(phis).max() ** 3 + 1e-15
    assert out["risk"] > phis.mean()  # strictly increasing in theta for non-constant Phi


def test_one_sample_gradient_independent_of_theta():
    z = _ctrl_field(4, "test")
    g = [_single_level_grad(_small(theta=t), z, [3])[0]["grad"] for t in (0.1, 10.0, 100.0)]
    assert np.abs(g[0] - g[1]).max() < 1e-13 * np.abs(g[0]).max()
    assert np.abs(g[0] - g[2]).max() < 1e-13 * np.abs(g[0]).max()


def test_sigma_zero_has_zero_variance():
    z = _ctrl_field(8, "test")
    W = _small(sigma=0.0, n_levels=2)
    for l in (0, 1):
        r = mlmc.level_batch(W, 0, l, range(5), z)
        assert r["stats"].s2_x == 0.0 and r["stats"].s2_y == 0.0
    # theta-independent gradient when all samples agree
    gs = []
    for th in (1.0, 50.0):
        W = _small(sigma=0.0, n_levels=2, theta=th)
        rs = [mlmc.level_batch(W, 0, l, range(3), z) for l in (0, 1)]
        gs.append(mlmc.combine(W, [r["stats"] for r in rs], [r["shift"] for r in rs], z, 0.0)["grad"])
    assert np.abs(gs[0] - gs[1]).max() < 1e-12 * np.abs(gs[0]).max()


def test_telescoping_sum():
    """Same draws on every level: sum_l mean(X_l - X_{l-1}) = mean X_L."""
    W = _small(n_levels=3)
    z = _ctrl_field(W.Nc, "test")
    samples = list(range(3))
    c = 0.05
    rs = [mlmc.level_batch(W, 0, l, samples, z, shift=c, xi_level=0) for l in range(3)]
    out = mlmc.combine(W, [r["stats"] for r in rs], [c] * 3, z, 0.0)
    top = rs[2]["per_sample"]
    wX = np.mean([np.exp(W.theta * (p["fine"]["phi"] - c)) * p["fine"]["bq"] for p in top], axis=0)
    wY = np.mean([np.exp(W.theta * (p["fine"]["phi"] - c)) for p in top])
    assert np.abs(out["EX"] - wX).max() < 1e-14 * np.abs(wX).max()
    assert abs(out["EY"] - wY) < 1e-14
    # and the coarse partner of level l is exactly level l-1 on the same draw
    for m in samples:
        assert rs[1]["per_sample"][m]["coarse"]["phi"] == rs[0]["per_sample"][m]["fine"]["phi"]


def test_shift_invariance():
    W = _small(n_levels=2, theta=30.0)
    z = _ctrl_field(W.Nc, "test")
    outs = []
    for c in (None, 0.0, 0.3):
        rs = [mlmc.level_batch(W, 0, l, range(3), z, shift=c) for l in (0, 1)]
        outs.append(mlmc.combine(W, [r["stats"] for r in rs], [r["shift"] for r in rs], z, 0.1))
    for o in outs[1:]:
        assert np.abs(o["grad"] - outs[0]["grad"]).max() < 1e-12 * np.abs(outs[0]["grad"]).max()
        assert abs(o["risk"] - outs[0]["risk"]) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 7, 8, 13])
def test_chan_merge_matches_two_pass(n):
    rng = np.random.default_rng(n)
    hc3 = 0.125
    X = rng.standard_normal((n, 5)) * 3 + 10
    Y = rng.standard_normal(n) + 4
    S = mlmc.pairwise_reduce([mlmc.Stats.single(x, y) for x, y in zip(X, Y)], hc3)
    assert S.n == n
    assert np.abs(S.mean_x - X.mean(0)).max() < 1e-13
    assert abs(S.mean_y - Y.mean()) < 1e-13
    assert abs(S.s2_x - hc3 * ((X - X.mean(0)) ** 2).sum()) < 1e-11
    assert abs(S.s2_y - ((Y - Y.mean()) ** 2).sum()) < 1e-11
    # batch split and merge order do not matter
    if n >= 2:
        k = n // 2
        A = mlmc.pairwise_reduce([mlmc.Stats.single(x, y) for x, y in zip(X[:k], Y[:k])], hc3)
        B = mlmc.pairwise_reduce([mlmc.Stats.single(x, y) for x, y in zip(X[k:], Y[k:])], hc3)
        for AB in (mlmc.chan_merge(A, B, hc3), mlmc.chan_merge(B, A, hc3)):
            assert np.abs(AB.mean_x - S.mean_x).max() < 1e-13
            assert abs(AB.s2_x - S.s2_x) < 1e-11 and abs(AB.s2_y - S.s2_y) < 1e-11


def test_merge_of_records_at_different_shifts():
    """Records of disjoint sample ranges, each at its own shift (the largest Phi of
    its own samples), merge into the record of the whole range at its shift."""
    W = _small(n_levels=2, theta=40.0)
    z = _ctrl_field(W.Nc, "test") + 3.0 * _ctrl_field(W.Nc, "rand", 2)
    whole = mlmc.level_batch(W, 1, 1, range(7), z)
    parts = [mlmc.level_batch(W, 1, 1, r, z) for r in (range(0, 2), range(2, 3), range(3, 7))]
    assert len({p["shift"] for p in parts}) > 1  # the parts' shifts differ
    m = mlmc.merge_shifted(parts, W.theta, W.hc3)
    a, b = m["stats"], whole["stats"]
    assert m["shift"] == whole["shift"] and a.n == b.n == 7
    assert np.abs(a.mean_x - b.mean_x).max() <= 1e-13 * np.abs(b.mean_x).max()
    assert abs(a.mean_y - b.mean_y) <= 1e-13 * abs(b.mean_y)
    assert abs(a.s2_x - b.s2_x) <= 1e-11 * b.s2_x and abs(a.s2_y - b.s2_y) <= 1e-11 * b.s2_y


def test_truncation_of_denominator():
    W = _small(theta=2.0)
    S = mlmc.Stats(4, np.ones(W.Nc ** 3), 0.0, 1e-6, 0.0)  # E^ML[Y~] far below exp(-theta c)
    out = mlmc.combine(W, [S], [0.1], np.zeros(W.Nc ** 3), 1.0)
    assert out["truncated"]
    assert np.allclose(out["grad"], np.exp(2.0 * 0.1))


# ---------------------------------------------------------------- controller

def _info(n, s2x, s2y, mx2, my, shift=0.0, theta=1.0):
    return dict(n=n, shift=shift, theta=theta, s2_x=s2x, s2_y=s2y, mean_x_norm2=mx2, mean_y=my)


def test_batch_sizes_meet_the_sampling_target():
    infos = [_info(64, 6.3, 0.4, 1.0, 1.0), _info(16, 0.2, 0.01, 1e-2, 1e-3), _info(4, 0.01, 1e-4, 5e-4, 1e-4)]
    p = controller.plan(infos, EX_norm2=1.0, EY=1.0, grad_norm=0.5, eta=0.9, n0=8, L_max=3)
    V = [p["v2"][l] / (infos[l]["n"] - 1) for l in range(3)]
    assert sum(V[l] / p["M"][l] for l in range(3)) <= p["eps2"] / 2
    # near-optimal cost: compare with exhaustive search over integer (M0, M1) for L = 2
    C = [controller.cost_model(8, l) for l in range(3)]
    best = min(M0 * C[0] + M1 * C[1] + M2 * C[2]
               for M0 in range(2, 400) for M1 in range(2, 200) for M2 in (p["M"][2],)
               if V[0] / M0 + V[1] / M1 + V[2] / M2 <= p["eps2"] / 2)
    got = sum(p["M"][l] * C[l] for l in range(3))
    assert got <= best + C[0] + C[1] + C[2]


def test_alpha_fit_and_level_update():
    # bias^2 decays like 4^-(2 l)  ->  alpha_hat = 2 exactly
    infos = [_info(8, 1.0, 0.0, 1.0, 0.0)] + [_info(8, 1.0, 0.0, 16.0 ** -l, 0.0) for l in (1, 2, 3)]
    p = controller.plan(infos, EX_norm2=1.0, EY=1.0, grad_norm=1.0, eta=0.9, n0=8, L_max=6)
    assert abs(p["alpha_hat"] - 2.0) < 1e-12
    # err_num = bias2_L / (2^2 - 1)^2 at the finest level dominates
    assert abs(p["err_num"] - 16.0 ** -3 / 9.0) < 1e-15
    assert p["L"] == 4  # 16^-3/9 < 0.81/2: no refinement
    p = controller.plan(infos, EX_norm2=1.0, EY=1.0, grad_norm=1e-3, eta=0.9, n0=8, L_max=6)
    assert p["L"] == 5 and len(p["M"]) == 5
    p = controller.plan(infos, EX_norm2=1.0, EY=1.0, grad_norm=1e-3, eta=0.9, n0=8, L_max=4)
    assert p["L"] == 4


def test_plan_undoes_the_shift():
    """v^2, err_sam and the plan are in unshifted units (eq:sec-order-sum,
    eq:mse-estimate-mlmc, eq:optimal-batch-size): records kept with nonzero shifts
    c_l (X~ = exp(-theta c_l) X) must give the plan that the unshifted per-sample data
    give, and v^2 must equal the second-order sums formed directly from the unshifted
    data.  Converting back with exp(theta c) instead of exp(2 theta c) fails this."""
    rng = np.random.default_rng(11)
    theta, hc3, ncell = 7.0, 1.0 / 512, 512
    shifts = [0.31, 0.27, 0.33]
    counts = [40, 12, 5]
    raw, shifted = [], []
    for l, (c, n) in enumerate(zip(shifts, counts)):
        dX = rng.standard_normal((n, ncell)) * 2.0 ** -l + 0.3 * 4.0 ** -l
        dY = rng.standard_normal(n) * 0.1 * 2.0 ** -l + 4.0 ** -l
        mx, my = dX.mean(0), dY.mean()
        s2x = hc3 * float(((dX - mx) ** 2).sum())  # sum_m ||dX_m - mean||_U^2, two passes
        s2y = float(((dY - my) ** 2).sum())
        raw.append(dict(n=n, mx=mx, my=my, s2x=s2x, s2y=s2y))
        f = np.exp(-theta * c)
        shifted.append(_info(n, s2x * f * f, s2y * f * f, hc3 * float(mx @ mx) * f * f, my * f, shift=c,
                             theta=theta))
    EX = sum(r["mx"] for r in raw)
    EY = sum(r["my"] for r in raw)
    cstar = max(shifts)
    g = 0.05
    p = controller.plan(shifted, EX_norm2=hc3 * float(EX @ EX) * np.exp(-2 * theta * cstar),
                        EY=EY * np.exp(-theta * cstar), grad_norm=g, eta=0.9, n0=8, L_max=4)
    C_hat = hc3 * float(EX @ EX) / EY ** 2
    v2 = [r["s2x"] + C_hat * r["s2y"] for r in raw]
    assert np.allclose(p["v2"], v2, rtol=1e-12, atol=0)
    err_sam = sum(v / (r["n"] * (r["n"] - 1)) for v, r in zip(v2, raw))
    assert abs(p["err_sam"] - err_sam) <= 1e-12 * err_sam
    q = controller.plan([_info(r["n"], r["s2x"], r["s2y"], hc3 * float(r["mx"] @ r["mx"]), r["my"], theta=theta)
                         for r in raw], EX_norm2=hc3 * float(EX @ EX), EY=EY, grad_norm=g, eta=0.9, n0=8, L_max=4)
    assert p["M"] == q["M"] and p["L"] == q["L"]
    assert abs(p["err_num"] - q["err_num"]) <= 1e-12 * q["err_num"]


def inputs_z_test(Nc):
    from paper_2606_09291_gb300 import inputs
    return inputs.z_test(Nc)


def test_adaptive_tau_quadratic_closed_form():
    """J(u) = lam/2 ||u||^2 with exact gradients (err_sam = 0): L_hat = lam and the
    adaptive step is 1/lam, which lands on the minimiser in one step."""
    from oracle import controller
    rng = np.random.default_rng(1)
    lam, hc3 = 7.5, 1.0 / 64
    u0 = rng.standard_normal(64)
    tau0 = 0.01
    g0 = lam * u0
    u1 = u0 - tau0 * g0
    g1 = lam * u1
    tau, l_hat, fb = controller.adaptive_tau(g1, g0, tau0, 0.0, hc3, tau0)
    assert not fb and abs(l_hat - lam) <= 1e-12 * lam and abs(tau - 1.0 / lam) <= 1e-12 / lam
    assert np.abs(u1 - tau * g1).max() <= 1e-13 * np.abs(u0).max()
    # sampling error shortens the step by (1 - err_sam / ||g||^2)
    g2 = hc3 * float(g1 @ g1)
    tau_e, _, _ = controller.adaptive_tau(g1, g0, tau0, 0.25 * g2, hc3, tau0)
    assert abs(tau_e - 0.75 / lam) <= 1e-12 / lam
    # no positive step: min(tau_prev, 1 / L_hat)
    tau_f, _, fb = controller.adaptive_tau(g1, g0, tau0, 2.0 * g2, hc3, tau0)
    assert fb and tau_f == tau0
    big = 0.5  # a previous step longer than 1 / lam: u1' = u0 - big lam u0
    u1b = u0 - big * g0
    tau_b, l_b, fb = controller.adaptive_tau(lam * u1b, g0, big, 2.0 * hc3 * float((lam * u1b) @ (lam * u1b)),
                                             hc3, big)
    assert fb and abs(l_b - lam) <= 1e-12 * lam and abs(tau_b - 1.0 / lam) <= 1e-12 / lam
    # first iteration
    assert controller.adaptive_tau(g1, None, 0.0, 0.0, hc3, 0.3)[0] == 0.3


def test_adaptive_mlsgd_sigma0_lipschitz_bounds():
    """sigma = 0: every sample is the deterministic a = 1 problem, err_sam = 0 and
    the gradient u -> S*(S u - g) + alpha u is affine with symmetric Hessian
    H = S*S + alpha, so L_hat is a Rayleigh-type quotient ||H d|| / ||d|| inside
    [alpha, alpha + ||S||^2] with ||S|| <= 1/lambda_1 <= 1/(3 pi^2) (Q1 Ritz values
    lie above the continuous ones); the steps drive the gradient to rounding level."""
    W = mlmc.Workload(n0=4, n_levels=2, n_modes=8, corr_len=0.3, sigma=0.0, theta=3.0, alpha=1e-3, seed=0)
    z0 = inputs_z_test(8)
    tau0 = 50.0
    z, hist = mlmc.mlsgd(W, z0, (3, 2), 4, tau0, adaptive=True)
    top = W.alpha + (3 * np.pi ** 2) ** -2
    for h in hist[1:]:
        assert abs(h["err_sam"]) <= 1e-20
        assert W.alpha * (1 - 1e-9) <= h["l_hat"] <= top * (1 + 1e-9)
        assert not h["fallback"] and abs(h["tau"] - 1.0 / h["l_hat"]) <= 1e-12 * h["tau"]
    assert hist[-1]["grad_norm"] <= 1e-8 * hist[0]["grad_norm"]


def test_rates_second_moment_definition():
    """The rate diagnostics' second moments equal (1/M) sum of the per-sample
    squared norms, recomputed from the unshifted per-sample records."""
    from oracle import controller
    W = mlmc.Workload(n0=4, n_levels=3, n_modes=8, corr_len=0.3, sigma=1.0, theta=4.0, alpha=1e-4, seed=2)
    z = inputs_z_test(16)
    recs = [mlmc.level_batch(W, 0, l, range(4), z) for l in range(3)]
    r = controller.rates([x["stats"] for x in recs], [x["shift"] for x in recs], W.theta, W.hc3)
    for l, rec in enumerate(recs):
        dX = [ps["dX"] * np.exp(W.theta * rec["shift"]) for ps in rec["per_sample"]]
        dY = [ps["dY"] * np.exp(W.theta * rec["shift"]) for ps in rec["per_sample"]]
        m2x = np.mean([W.hc3 * float(d @ d) for d in dX])
        m2y = np.mean([d * d for d in dY])
        assert abs(r["m2_dx"][l] - m2x) <= 1e-12 * m2x
        assert abs(r["m2_dy"][l] - m2y) <= 1e-12 * m2y
        mx = np.mean(dX, axis=0)
        assert abs(r["mean_dx_norm"][l] - np.sqrt(W.hc3 * float(mx @ mx))) <= 1e-12 * r["mean_dx_norm"][l]
    assert np.isfinite(r["beta_x"]) and np.isfinite(r["alpha_y"])
