"""Per-sample MLMC gradient pieces and the estimator (oracle, test infrastructure only).

Follows the paper's notation:
* state y_l = S_l[xi](u), adjoint q_l with right-hand side <y_l - g, v>_H
  (Sec. 2.2, discrete state and adjoint problems);
* Phi(y) = 1/2 ||y - g||_H^2 (eq:cost); here g is replaced by its nodal
  interpolant g_h and ||e||_H^2 = e^T M e with the consistent Q1 mass M;
* X_l = exp(theta Phi(y_l)) B* q_l, Y_l = exp(theta Phi(y_l))
  (eq:definition_Xell_Yell), evaluated with a shift c:
  Ytilde = exp(theta (Phi - c)), Xtilde = Ytilde B* q, which multiplies X and Y
  by the same factor exp(-theta c);
* Delta X_l = X_l - X_{l-1} on the SAME draw xi^(m,l), with X_{-1} = 0 on the
  coarsest level (eq:shorthand-notation, eq:delta-notation; the paper's
  coarsest level is l = 1 with X_0 = 0, here it is level 0);
* per-level sample statistics merged pairwise with the Chan update
  (Algorithm 1, PairwiseUpdate; Sec. 4.2 b): M_AB = M_A + M_B,
  delta = E_A - E_B, E_AB = E_B + (M_A / M_AB) delta, and the second-order
  sums S_AB = S_A + S_B + |delta|^2 M_A M_B / M_AB (Chan, Golub, LeVeque);
* E^ML[X] = sum_l mean(Delta X_l) (eq:ml_estimator_numerator, and likewise Y,
  eq:ml_estimator_denominator), gradient
  E^ML[X] / max{1, E^ML[Y]} + lambda u (eq:gradient_estimator, with the
  truncation below it), and u <- Pi(u - tau grad) (eq:gradientdescentMLMC).
  With shifted sums the truncation max{1, E^ML[Y]} becomes
  max{exp(-theta c*), E^ML[Ytilde]} for the common shift c*.

Norms on U: <z, w>_U = h_c^3 sum_c z_c w_c on the control grid.
"""
import numpy as np

from . import fem, kl, philox, solve as solvers


class Workload:
    """Fixed data of one workload: levels, KL table, control grid."""

    def __init__(self, n0, n_levels, n_modes, corr_len, sigma, theta, alpha, seed,
                 ctrl_level=None, rtol=1e-13, method="auto", field_model=0, target_freq=1):
        self.n0, self.n_levels = n0, n_levels
        self.ctrl_level = n_levels - 1 if ctrl_level is None else ctrl_level
        self.Nc = n0 * 2 ** self.ctrl_level
        self.hc3 = (1.0 / self.Nc) ** 3
        self.sigma, self.theta, self.alpha, self.seed = sigma, theta, alpha, seed
        self.n_modes = n_modes
        self.field_model, self.target_freq = field_model, target_freq
        if field_model == 1:  # the paper's Sec. 5 field with n_modes = m^3
            m = round(n_modes ** (1.0 / 3.0))
            assert m ** 3 == n_modes
            self.kl = kl.PaperKLTable(corr_len, m)
        else:
            self.kl = kl.KLTable(corr_len, n_modes)
        self.rtol, self.method = rtol, method
        self._levels = {}

    def level(self, l):
        if l not in self._levels:
            lev = fem.Level(self.n0 * 2 ** l)
            lev.M_full = lev.mass()
            lev.g = lev.nodal_target(self.target_freq)
            lev.I = lev.interpolation(self.Nc)
            lev.phi = self.kl.cell_modes(lev.N)
            self._levels[l] = lev
        return self._levels[l]

    def xi(self, iteration, level, samples):
        if self.field_model == 1:  # xi ~ U(-4, 4) (Sec. 5)
            return philox.uniforms(self.seed, iteration, level, samples, self.n_modes, 4.0)
        return philox.normals(self.seed, iteration, level, samples, self.n_modes)

    def log_a(self, xi, grid_level):
        lev = self.level(grid_level)
        return (self.sigma * self.kl.sqrt_lam3[None, :] * xi) @ lev.phi

    def rhs_state(self, z, grid_level):
        """Full node vector B_l z."""
        lev = self.level(grid_level)
        return self.hc3 * (lev.I.T @ z)

    def solve_state_adjoint(self, log_a, z, grid_level):
        """One sample on one grid: returns dict(y, q (full node vectors), phi, bq, iters)."""
        lev = self.level(grid_level)
        a = np.exp(log_a)
        A = lev.restrict(lev.stiffness(a))
        I = lev.interior
        b = self.rhs_state(z, grid_level)
        y = np.zeros(lev.nn)
        y[I], it_y = solvers.solve(A, b[I], lev.N, self.rtol, self.method)
        e = y - lev.g
        Me = lev.M_full @ e
        phi = 0.5 * e @ Me
        q = np.zeros(lev.nn)
        q[I], it_q = solvers.solve(A, Me[I], lev.N, self.rtol, self.method)
        return dict(y=y, q=q, phi=phi, bq=lev.I @ q, iters=(it_y, it_q))

    def sample(self, iteration, level, m, z, xi_level=None):
        """Everything for sample m of level `level`: fine and (if level > 0) coarse grid.

        xi is drawn with the counter of `level` (or of `xi_level` if given)."""
        xi = self.xi(iteration, level if xi_level is None else xi_level, [m])[0]
        out = {"xi": xi, "fine": self.solve_state_adjoint(self.log_a(xi[None], level)[0], z, level)}
        if level > 0:
            out["coarse"] = self.solve_state_adjoint(self.log_a(xi[None], level - 1)[0], z, level - 1)
        return out


# ---------------------------------------------------------------- statistics

class Stats:
    """Sample count, mean and second-order sum of a field and of a scalar."""

    def __init__(self, n, mean_x, s2_x, mean_y, s2_y):
        self.n, self.mean_x, self.s2_x, self.mean_y, self.s2_y = n, mean_x, s2_x, mean_y, s2_y

    @staticmethod
    def single(x, y):
        return Stats(1, np.array(x, dtype=np.float64), 0.0, float(y), 0.0)


def chan_merge(A, B, hc3):
    """Pairwise update of two groups (Algorithm 1, PairwiseUpdate)."""
    n = A.n + B.n
    dx = A.mean_x - B.mean_x
    dy = A.mean_y - B.mean_y
    mean_x = B.mean_x + (A.n / n) * dx
    mean_y = B.mean_y + (A.n / n) * dy
    s2_x = A.s2_x + B.s2_x + hc3 * (dx @ dx) * A.n * B.n / n
    s2_y = A.s2_y + B.s2_y + dy * dy * A.n * B.n / n
    return Stats(n, mean_x, s2_x, mean_y, s2_y)


def pairwise_reduce(items, hc3):
    """Merge a list of Stats pairwise at distances d = 2^k, largest first
    (the process-pairing pattern of Algorithm 1 / Sec. 4.2 b); a list whose
    length is not a power of two folds its tail onto the head first."""
    items = list(items)
    P = 1
    while 2 * P <= len(items):
        P *= 2
    for j in range(P, len(items)):  # fold the remainder
        items[j - P] = chan_merge(items[j - P], items[j], hc3)
    items = items[:P]
    d = P // 2
    while d >= 1:
        items = [chan_merge(items[i], items[i + d], hc3) for i in range(d)]
        d //= 2
    return items[0]


def merge_shifted(records, theta, hc3):
    """Merge level records kept at different shifts (each a dict(stats, shift) as
    level_batch returns): every record is rescaled to the largest shift c* (means by
    exp(theta (c - c*)), second-order sums by its square; X~ and Y~ carry the factor
    exp(-theta c)) and the rescaled records are merged pairwise (Algorithm 1,
    PairwiseUpdate).  Returns dict(stats, shift)."""
    cstar = max(r["shift"] for r in records)
    items = []
    for r in records:
        f = np.exp(theta * (r["shift"] - cstar))
        S = r["stats"]
        items.append(Stats(S.n, S.mean_x * f, S.s2_x * f * f, S.mean_y * f, S.s2_y * f * f))
    return dict(stats=pairwise_reduce(items, hc3), shift=cstar)


def level_batch(W, iteration, level, samples, z, shift=None, xi_level=None):
    """Samples of one level: per-sample records and their merged statistics.

    Returns dict(stats, shift, per_sample=[...]).  The shift c is
    max over the batch of Phi on both grids unless given."""
    recs = [W.sample(iteration, level, m, z, xi_level) for m in samples]
    phis = [r["fine"]["phi"] for r in recs] + [r["coarse"]["phi"] for r in recs if "coarse" in r]
    c = max(phis) if shift is None else shift
    th = W.theta
    items = []
    for r in recs:
        yf = np.exp(th * (r["fine"]["phi"] - c))
        dX = yf * r["fine"]["bq"]
        dY = yf
        if "coarse" in r:
            yc = np.exp(th * (r["coarse"]["phi"] - c))
            dX = dX - yc * r["coarse"]["bq"]
            dY = dY - yc
        r["dX"], r["dY"] = dX, dY
        items.append(Stats.single(dX, dY))
    return dict(stats=pairwise_reduce(items, W.hc3), shift=c, per_sample=recs)


def combine(W, level_stats, level_shifts, z, tau, project=None):
    """Cross-level sums, gradient and projected step.

    level_stats[l] / level_shifts[l]: Stats and shift c_l of level l.
    Returns dict(grad, z_new, grad_norm, EX, EY, shift, risk)."""
    cstar = max(level_shifts)
    th = W.theta
    EX = np.zeros(W.Nc ** 3)
    EY = 0.0
    for S, c in zip(level_stats, level_shifts):
        f = np.exp(th * (c - cstar))
        EX = EX + f * S.mean_x
        EY = EY + f * S.mean_y
    denom = max(np.exp(-th * cstar), EY)
    grad = EX / denom + W.alpha * z
    z_new = z - tau * grad
    if project is not None:
        z_new = project(z_new)
    gnorm = np.sqrt(W.hc3 * (grad @ grad))
    risk = cstar + np.log(EY) / th if EY > 0 else float("nan")
    return dict(grad=grad, z_new=z_new, grad_norm=gnorm, EX=EX, EY=EY, shift=cstar,
                risk=risk, truncated=EY < np.exp(-th * cstar))


def mlsgd(W, z, counts, iterations, tau0, adaptive=False, eta=0.9, L_max=None, adapt_counts=False):
    """MLSGD outer loop (Algorithm 1, function MLSGD): per iteration k, fresh draws
    on every level with the current batch sizes, the multilevel gradient, the step
    (fixed tau0, or eq:adaptive-step-size with tau_0 = tau0), and optionally the
    next level count and batch sizes from the controller.
    Returns (z, history) with one dict per iteration (tau, L_hat, grad_norm, risk,
    err_sam, counts, rates)."""
    from . import controller
    L_max = W.n_levels if L_max is None else L_max
    counts = list(counts)
    z = np.array(z, dtype=np.float64)
    g_prev, tau_prev, hist = None, 0.0, []
    for k in range(iterations):
        recs = [level_batch(W, k, l, range(m), z) for l, m in enumerate(counts)]
        stats, shifts = [r["stats"] for r in recs], [r["shift"] for r in recs]
        res = combine(W, stats, shifts, z, 0.0)
        info = [dict(n=s.n, shift=c, theta=W.theta, s2_x=s.s2_x, s2_y=s.s2_y,
                     mean_x_norm2=W.hc3 * float(s.mean_x @ s.mean_x), mean_y=s.mean_y)
                for s, c in zip(stats, shifts)]
        p = controller.plan(info, W.hc3 * float(res["EX"] @ res["EX"]), res["EY"], res["grad_norm"], eta, W.n0, L_max)
        if adaptive:
            tau, l_hat, fb = controller.adaptive_tau(res["grad"], g_prev, tau_prev, p["err_sam"], W.hc3, tau0)
        else:
            tau, l_hat, fb = tau0, float("nan"), False
        objective = res["risk"] + 0.5 * W.alpha * W.hc3 * float(z @ z)  # J^ML(u_k), eq:cost
        z = z - tau * res["grad"]
        hist.append(dict(tau=tau, l_hat=l_hat, fallback=fb, grad_norm=res["grad_norm"], risk=res["risk"],
                         objective=objective,
                         err_sam=p["err_sam"], counts=list(counts), plan=p,
                         rates=controller.rates(stats, shifts, W.theta, W.hc3)))
        g_prev, tau_prev = res["grad"], tau
        if adapt_counts:
            counts = p["M"]
    return z, hist
