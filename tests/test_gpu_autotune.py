"""GPU tests of the autotuner: every knob value it can choose keeps the level
record within the mixed path's bar of the oracle (a fixed refinement-step count that
leaves a sample unconverged is reported as such, and the tuner rejects it), and a
tuned entry, once cached, is returned as is (a run is deterministic given its
cache)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402

TOLMIX = 1e-6
CFG = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=0, rtol=1e-8,
           max_iter=50, precision="mixed")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def _choices():
    from paper_2606_09291_gb300 import autotune as T
    out = []
    for name, values in list(T.SHAPES.items()) + list(T.SCHEDULES.items()):
        for v in values:
            if v != T.DEFAULTS[name]:
                out.append(dict(T.DEFAULTS, **{name: v}))
    return [dict(T.DEFAULTS)] + out


def test_every_choice_matches_the_oracle(lib):
    z = inputs.z_test(32)
    zt = torch.tensor(z, dtype=torch.float64, device="cuda")
    W = mlmc.Workload(n0=8, n_levels=3, n_modes=64, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=0)
    ref = mlmc.level_batch(W, 2, 2, range(5), z)
    fo = ref["stats"].mean_x * np.exp(W.theta * ref["shift"])
    yo = ref["stats"].mean_y * np.exp(W.theta * ref["shift"])
    from paper_2606_09291_gb300 import autotune as T
    for knobs in _choices():
        ctx = lib.Context(**T.context_cfg(CFG, knobs, 5))
        st = ctx.new_stats(2)
        ctx.mlsgd_level_gradient(2, 2, 0, 5, zt, st)
        h = st.host()
        f = st.field.cpu().numpy() * np.exp(W.theta * h["shift"])
        ctx.close()
        assert h["count"] == 5, knobs
        if h["noconv"]:  # only a fixed step count may stop short of rtol
            assert knobs["ir_steps"] > 0, knobs
            continue
        assert np.abs(f - fo).max() <= TOLMIX * np.abs(fo).max(), knobs
        assert abs(h["mean_dy"] * np.exp(W.theta * h["shift"]) - yo) <= TOLMIX * abs(yo), knobs


def test_tuned_entry_is_cached(lib, tmp_path):
    from paper_2606_09291_gb300 import autotune as T
    cache = str(tmp_path / "tuned.json")
    zt = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    knobs, rep = T.tune(CFG, 2, 16, zt, reps=1, cache_path=cache)
    assert rep["source"] == "measured" and set(knobs) == set(T.KNOBS)
    assert knobs["stencil"] in T.SHAPES["stencil"] and knobs["inner_iters"] in T.SCHEDULES["inner_iters"]
    assert rep["ms_per_sample"] <= rep["default_ms_per_sample"]
    with open(cache) as f:
        assert T.key(CFG, 2, 16) in json.load(f)
    again, rep2 = T.tune(CFG, 2, 16, zt, reps=1, cache_path=cache)
    assert again == knobs and rep2["source"] == "cache"
    assert T.lookup(CFG, 2, 16, path=cache) == knobs
