"""Host logic of the MLSGD driver (Algorithm 1 outer loop) on the CPU.

The library context is a fake that records the level launches and returns
scripted step reports, so what is checked is the driver's own logic: batch
sizes taken from each step's plan, the count cap, the two stop rules, the
adaptive step's previous step size, the cost-exponent fit and the time-budget
scaling of the next batches."""
import math

import pytest

torch = pytest.importorskip("torch")
from paper_2606_09291_gb300 import driver  # noqa: E402


class FakeCtx:
    def __init__(self, n_levels, reports, cost_ms=None):
        self.cfg = dict(n_levels=n_levels)
        self.reports = list(reports)
        self.launches, self.steps = [], []
        self.cost_ms = cost_ms
        self.last_ms = 0.0

    def new_stats(self, level):
        return ("stats", level)

    def mlsgd_stats_reset(self, st, stream=None):
        pass

    def mlsgd_level_gradient(self, it, level, first, n, z, st, stream=None):
        assert st == ("stats", level) and first == 0
        self.launches.append((it, level, n))
        if self.cost_ms is not None:
            self.last_ms = n * self.cost_ms[level]

    def _report(self, stats_list):
        rep = dict(self.reports.pop(0))
        rep.setdefault("tau", 0.5)
        return rep

    def mlsgd_step(self, stats_list, tau, z, eta=0.9, max_levels=None, grad=None, stream=None):
        self.steps.append(("fixed", len(stats_list), tau, None))
        return self._report(stats_list)

    def mlsgd_step_adaptive(self, stats_list, tau0, tau_prev, z, grad_prev, eta=0.9, max_levels=None, stream=None):
        assert grad_prev.shape == z.shape
        self.steps.append(("adaptive", len(stats_list), tau0, tau_prev))
        return self._report(stats_list)


def test_slope_and_fixed_step():
    assert driver._slope([1, 2, 3], [4.0 ** l for l in (1, 2, 3)]) == pytest.approx(2.0)
    assert driver._slope([0, 1, 2, 3], [3.0 * 2.0 ** (-1.5 * l) for l in range(4)]) == pytest.approx(-1.5)
    assert math.isnan(driver._slope([1], [2.0]))
    alpha = 1e-4
    tau = driver.fixed_step(alpha)
    assert tau == pytest.approx(0.5 / (alpha + 1.0 / (3 * math.pi ** 2) ** 2))


def test_counts_follow_the_plan_with_cap():
    reps = [dict(grad_norm=1.0, next_counts=[40, 8]), dict(grad_norm=1.0, next_counts=[80, 16, 4]),
            dict(grad_norm=1.0, next_counts=[1000, 32, 8])]
    ctx = FakeCtx(4, reps)
    z = torch.zeros(8, dtype=torch.float64)
    hist = driver.run_mlsgd(ctx, z, [16, 4], 3, tau=0.25, count_cap=500)
    assert [h["counts"] for h in hist] == [[16, 4], [40, 8], [80, 16, 4]]
    assert ctx.launches == [(0, 0, 16), (0, 1, 4), (1, 0, 40), (1, 1, 8), (2, 0, 80), (2, 1, 16), (2, 2, 4)]
    assert [s[1] for s in ctx.steps] == [2, 2, 3] and all(s[2] == 0.25 for s in ctx.steps)
    # without adaptation the batches stay fixed
    ctx = FakeCtx(4, [dict(grad_norm=1.0, next_counts=[99])] * 2)
    hist = driver.run_mlsgd(ctx, z, [16, 4], 2, tau=0.25, adapt=False)
    assert [h["counts"] for h in hist] == [[16, 4], [16, 4]]
    # the cap applies to the planned batches
    ctx = FakeCtx(2, [dict(grad_norm=1.0, next_counts=[1000, 600]), dict(grad_norm=1.0, next_counts=[1, 1])])
    hist = driver.run_mlsgd(ctx, z, [2, 2], 2, tau=0.1, count_cap=500)
    assert hist[1]["counts"] == [500, 500]


def test_gradient_tolerance_stops_after_that_step():
    reps = [dict(grad_norm=g, next_counts=[8]) for g in (1.0, 0.5, 1e-3, 1e-4)]
    ctx = FakeCtx(1, reps)
    hist = driver.run_mlsgd(ctx, torch.zeros(4, dtype=torch.float64), [8], 10, tau=0.1, grad_tol=1e-2)
    assert len(hist) == 3 and hist[-1]["grad_norm"] == 1e-3 and len(ctx.steps) == 3


def test_adaptive_step_passes_the_previous_step_size():
    reps = [dict(grad_norm=1.0, next_counts=[8], tau=t) for t in (0.7, 0.3, 0.2)]
    ctx = FakeCtx(1, reps)
    driver.run_mlsgd(ctx, torch.zeros(4, dtype=torch.float64), [8], 3, tau=1.0, step="adaptive")
    assert [(s[0], s[2], s[3]) for s in ctx.steps] == [("adaptive", 1.0, 0.0), ("adaptive", 1.0, 0.7),
                                                        ("adaptive", 1.0, 0.3)]


class FakeEvent:
    ctx = None

    def record(self, stream):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, end):
        return FakeEvent.ctx.last_ms


def test_time_budget_scales_the_next_batches(monkeypatch):
    cost = [1.0, 4.0, 16.0]  # ms per sample on levels 0..2; a new level 3 is estimated at 8 x 16
    reps = [dict(grad_norm=1.0, next_counts=[10000, 1000, 100, 10]), dict(grad_norm=1.0, next_counts=[2, 2])]
    ctx = FakeCtx(4, reps, cost_ms=cost + [128.0])
    FakeEvent.ctx = ctx
    monkeypatch.setattr(driver, "_event", FakeEvent)
    budget = 10.0
    hist = driver.run_mlsgd(ctx, torch.zeros(4, dtype=torch.float64), [100, 10, 1], 2, tau=0.1, budget_s=budget,
                            stream="s")
    h0 = hist[0]
    assert h0["level_ms"] == [100.0, 40.0, 16.0]
    assert h0["cost_per_sample_ms"] == [1.0, 4.0, 16.0]
    assert h0["gamma_hat"] == pytest.approx(2.0)  # cost ~ 4^l on levels 1, 2
    planned = [10000, 1000, 100, 10]
    est = sum(m * c for m, c in zip(planned, cost + [128.0]))  # 21,880 ms > 10 s left
    f = 1000.0 * (budget - h0["elapsed_s"]) / est
    got = hist[1]["counts"]
    assert got == [max(2, int(m * f)) for m in planned]
    assert sum(m * c for m, c in zip(got, cost + [128.0])) <= 1000.0 * budget


class StepCtx(FakeCtx):
    """A fake whose step moves z by an amount that depends on the iteration, the batch
    sizes and the previous step size, and whose plan depends on the iteration, so
    that any state lost at a checkpoint changes the continuation."""

    def __init__(self, n_levels, seed=3):
        super().__init__(n_levels, [])
        self.cfg["seed"] = seed

    def _report(self, stats_list):
        it = self.launches[-1][0]
        n = [m for (i, l, m) in self.launches if i == it]
        return dict(grad_norm=1.0 / (it + 1), tau=0.1 + 0.01 * it, next_counts=[8 + it + l for l in range(len(n))],
                    err_sam=0.01 * it, err_num=1e-4, objective=0.5 + it, risk=0.4)

    def mlsgd_step(self, stats_list, tau, z, eta=0.9, max_levels=None, grad=None, stream=None):
        self.steps.append(("fixed", len(stats_list), tau, None))
        rep = self._report(stats_list)
        it = self.launches[-1][0]
        z += tau * (it + 1) * torch.arange(z.numel(), dtype=z.dtype) + sum(m for (i, l, m) in self.launches if i == it)
        return rep

    def mlsgd_step_adaptive(self, stats_list, tau0, tau_prev, z, grad_prev, eta=0.9, max_levels=None, stream=None):
        self.steps.append(("adaptive", len(stats_list), tau0, tau_prev))
        rep = self._report(stats_list)
        z -= (tau_prev + 1.0) * grad_prev
        grad_prev += 0.5 * z
        return rep


@pytest.mark.parametrize("step", ["fixed", "adaptive"])
def test_checkpoint_resume_is_bit_exact(tmp_path, step):
    ck = str(tmp_path / "ck.npz")
    a = StepCtx(3)
    za = torch.linspace(0, 1, 16, dtype=torch.float64)
    ha = driver.run_mlsgd(a, za, [6, 2], 5, tau=0.3, step=step)
    b = StepCtx(3)
    zb = torch.linspace(0, 1, 16, dtype=torch.float64)
    hb = driver.run_mlsgd(b, zb, [6, 2], 3, tau=0.3, step=step, checkpoint=ck)
    c = StepCtx(3)
    zc = torch.zeros(16, dtype=torch.float64)  # overwritten from the checkpoint
    hc = driver.run_mlsgd(c, zc, [99], 5, tau=0.3, step=step, resume=ck)
    assert torch.equal(zc, za)
    assert b.launches + c.launches == a.launches and b.steps + c.steps == a.steps
    assert [h["counts"] for h in hb + hc] == [h["counts"] for h in ha]
    assert [h["iteration"] for h in hc] == [3, 4]
    with pytest.raises(ValueError):
        driver.run_mlsgd(StepCtx(3, seed=4), torch.zeros(16, dtype=torch.float64), [6], 5, tau=0.3, step=step,
                         resume=ck)


def test_iteration_log_lines(tmp_path):
    import json
    log = str(tmp_path / "log.jsonl")
    ctx = StepCtx(2)
    driver.run_mlsgd(ctx, torch.zeros(4, dtype=torch.float64), [6, 2], 3, tau=0.3, log_path=log)
    lines = [json.loads(x) for x in open(log)]
    assert [d["iteration"] for d in lines] == [0, 1, 2]
    assert [d["counts"] for d in lines] == [[6, 2], [8, 9], [9, 10]]
    for d in lines:
        assert d["sqrt_mse"] == pytest.approx(math.sqrt(d["err_sam"] + d["err_num"]))
        assert {"objective", "grad_norm", "tau", "elapsed_s"} <= set(d)
