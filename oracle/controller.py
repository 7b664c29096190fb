"""Adaptive batch size and level selection (oracle, test infrastructure only).

Sec. 4.1 of the paper, with the readings this workload takes where the
printed formulas are garbled:

* second-order sums v^2_l = sum ||dX - mean||_U^2 + C_hat sum |dY - mean|^2
  (eq:sec-order-sum), C_hat = ||E^ML[X]||_U^2 / E^ML[Y]^2.  Sums are kept in
  shifted units (factor exp(-theta c_l) on X and Y) and are converted back by
  exp(2 theta c_l) before use, so that they are compared with the unshifted
  accuracy target eps^2.
* optimal batch (eq:optimal-batch-size), read as the Giles form
  M_l = ceil( 2 eps^-2 sqrt(V_l / C_l) sum_l' sqrt(V_l' C_l') ),
  V_l = v^2_l / (M_l - 1), so that sum_l V_l / M_l = eps^2 / 2 (the stated
  target err_sam = eps^2/2; the printed constant (sqrt2 eps)^-2 would give
  2 eps^2).  M_l >= 2.
* bias estimate (eq:squared-bias-estimate-mlmc), read with the Giles
  extrapolation factor ((2^alpha - 1) (h_l / h_L)^alpha)^2, maximised over the
  difference levels l >= 1; alpha_hat from a least-squares fit of
  log2 sqrt(||E dX_l||^2 + C_hat |E dY_l|^2) against l over l >= 1 (default
  alpha_hat = 2 when fewer than two difference levels exist).
* level update (eq:optimal-level): L grows by one when err_num > eps^2 / 2,
  up to the configured finest level.  A new level's variance is extrapolated
  from the last one by 2^-beta_hat (beta_hat fitted like alpha_hat from
  log2 V_l; default 4).
* err_sam = sum_l v^2_l / (M_l (M_l - 1)) (eq:mse-estimate-mlmc).
* cost per sample C_l (measured CPU seconds in the paper) is replaced by the
  deterministic model C_l = dofs_l (1 + 1/8 for l >= 1), dofs_l = (N_l - 1)^3.
"""
import math

import numpy as np


def cost_model(n0, l):
    N = n0 * 2 ** l
    return float((N - 1) ** 3) * (1.0 + (0.125 if l >= 1 else 0.0))


def _fit_slope(ls, vals):
    """Least-squares slope of log2(vals) against ls."""
    x = np.asarray(ls, dtype=np.float64)
    y = np.log2(np.asarray(vals, dtype=np.float64))
    xm, ym = x.mean(), y.mean()
    return float(((x - xm) * (y - ym)).sum() / ((x - xm) ** 2).sum())


def plan(level_info, EX_norm2, EY, grad_norm, eta, n0, L_max):
    """Next level count and batch sizes.

    level_info: list over l = 0..L-1 of dict(n, shift, theta, s2_x, s2_y,
    mean_x_norm2, mean_y) in shifted units.  EX_norm2 = ||E^ML[X~]||_U^2 and EY
    = E^ML[Y~] at the common shift (C_hat is a ratio, shift independent).
    Returns dict(L, M, err_sam, err_num, alpha_hat, eps2, C_hat, v2).
    """
    L = len(level_info)
    C_hat = EX_norm2 / (EY * EY)
    eps2 = (eta * grad_norm) ** 2
    v2, bias2 = [], []
    for info in level_info:
        s = math.exp(2.0 * info["theta"] * info["shift"])
        v2.append(s * (info["s2_x"] + C_hat * info["s2_y"]))
        bias2.append(s * (info["mean_x_norm2"] + C_hat * info["mean_y"] ** 2))
    M = [info["n"] for info in level_info]
    err_sam = sum(v2[l] / (M[l] * (M[l] - 1)) for l in range(L))
    diff_levels = list(range(1, L))
    if len(diff_levels) >= 2:
        alpha = -_fit_slope(diff_levels, [math.sqrt(bias2[l]) for l in diff_levels])
    else:
        alpha = 2.0
    err_num = 0.0
    for l in diff_levels:
        f = (2.0 ** alpha - 1.0) * (2.0 ** (L - 1 - l)) ** alpha
        err_num = max(err_num, bias2[l] / (f * f))
    V = [v2[l] / (M[l] - 1) for l in range(L)]
    C = [cost_model(n0, l) for l in range(L)]
    L_next = L + 1 if (err_num > eps2 / 2.0 and L < L_max) else L
    if L_next > L:
        if len(diff_levels) >= 2:
            beta = -_fit_slope(diff_levels, [V[l] for l in diff_levels])
        else:
            beta = 4.0
        V.append(V[-1] * 2.0 ** (-beta))
        C.append(cost_model(n0, L))
    total = sum(math.sqrt(V[l] * C[l]) for l in range(L_next))
    M_next = [max(2, int(math.ceil(2.0 / eps2 * math.sqrt(V[l] / C[l]) * total)))
              for l in range(L_next)]
    return dict(L=L_next, M=M_next, err_sam=err_sam, err_num=err_num, alpha_hat=alpha,
                eps2=eps2, C_hat=C_hat, v2=v2)


def adaptive_tau(grad, grad_prev, tau_prev, err_sam, hc3, tau0):
    """Adaptive step size of Sec. 5 (eq:adaptive-step-size).

    tau_k = (||g_k||^2 - err_sam_k) / (L_hat ||g_k||^2) with
    L_hat = ||g_k - g_{k-1}||_U / ||tau_{k-1} g_{k-1}||_U; the printed t_{k-1} is
    read as tau_{k-1}.  First iteration (grad_prev None): tau0.  Reading where
    the rule gives no positive finite step (sampling error estimate at or above
    ||g_k||^2): min(tau_{k-1}, 1 / L_hat), the rule without its sampling
    correction but never longer than the last step; tau_{k-1} if L_hat is not
    positive and finite.
    Returns (tau, L_hat, fell_back)."""
    if grad_prev is None:
        return tau0, float("nan"), False
    norm = lambda v: math.sqrt(hc3 * float(v @ v))
    g2 = hc3 * float(grad @ grad)
    l_hat = norm(grad - grad_prev) / (tau_prev * norm(grad_prev)) if norm(grad_prev) > 0 else float("inf")
    with np.errstate(all="ignore"):
        tau = (g2 - err_sam) / (l_hat * g2) if l_hat > 0 and g2 > 0 else float("nan")
    if not (math.isfinite(tau) and tau > 0):
        if math.isfinite(l_hat) and l_hat > 0:
            return min(tau_prev, 1.0 / l_hat), l_hat, True
        return tau_prev, l_hat, True
    return tau, l_hat, False


def rates(level_stats, level_shifts, theta, hc3):
    """Rate diagnostics of one batch (unshifted): per level the second moments
    (1/M) sum ||dX_l||_U^2 and (1/M) sum |dY_l|^2 (the left sides of eq:decayNum and
    eq:decayDenom), ||mean dX_l||_U and |mean dY_l| (eq:weakerror2, eq:weakerror),
    and the exponents beta_x, beta_y, alpha_x, alpha_y fitted over l >= 1 with
    h_l = h_0 2^-l (NaN with fewer than two difference levels)."""
    out = dict(m2_dx=[], m2_dy=[], mean_dx_norm=[], mean_dy_abs=[])
    for S, c in zip(level_stats, level_shifts):
        f = math.exp(theta * c)
        mx2 = hc3 * float(S.mean_x @ S.mean_x)
        out["m2_dx"].append(f * f * (S.s2_x / S.n + mx2))
        out["m2_dy"].append(f * f * (S.s2_y / S.n + S.mean_y ** 2))
        out["mean_dx_norm"].append(f * math.sqrt(mx2))
        out["mean_dy_abs"].append(f * abs(S.mean_y))
    L = len(level_stats)
    for key, name in (("m2_dx", "beta_x"), ("m2_dy", "beta_y"), ("mean_dx_norm", "alpha_x"),
                      ("mean_dy_abs", "alpha_y")):
        out[name] = -_fit_slope(range(1, L), out[key][1:]) if L >= 3 else float("nan")
    return out
