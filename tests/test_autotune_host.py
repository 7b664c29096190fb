"""Host logic of the autotuner (no GPU): cache keys, the knobs-to-configuration
mapping, lookups that fill knobs an older cache entry lacks, and the committed cache
entry of the benchmark batch."""
import json

import pytest

pytest.importorskip("torch")
from paper_2606_09291_gb300 import autotune as T  # noqa: E402

CFG = dict(n_levels=4, n0=8, n_modes=256, precision="mixed", rtol=1e-8)


def test_key_names_grid_batch_precision_modes():
    assert T.key(CFG, 3, 4096) == "N64-S4096-mixed-K256"
    assert T.key(dict(CFG, precision=0), 2, 16) == "N32-S16-fp64-K256"


def test_context_cfg_maps_batch_chunks_to_max_batch():
    for chunks, want in ((1, 4096), (2, 2048), (4, 1024), (3, 1366)):
        cfg = T.context_cfg(CFG, dict(T.DEFAULTS, batch_chunks=chunks), 4096)
        assert cfg["max_batch"] == want and "batch_chunks" not in cfg
    cfg = T.context_cfg(CFG, dict(inner_iters=5, omega=0.7), 100)  # missing knobs take their defaults
    assert cfg["inner_iters"] == 5 and cfg["omega"] == 0.7 and cfg["ir_steps"] == 0
    assert cfg["inner_iters_next"] == 0 and cfg["max_batch"] == 100
    assert all(cfg[k] == v for k, v in CFG.items())


def test_lookup_fills_missing_knobs(tmp_path):
    path = str(tmp_path / "tuned.json")
    with open(path, "w") as f:
        json.dump({T.key(CFG, 3, 4096): {"knobs": {"stencil": 0, "z_chunks": 2, "inner_iters": 5, "omega": 0.7}}}, f)
    got = T.lookup(CFG, 3, 4096, path=path)
    assert set(got) == set(T.KNOBS)
    assert got["z_chunks"] == 2 and got["batch_chunks"] == 1 and got["inner_iters_next"] == 0
    assert T.lookup(CFG, 3, 2048, path=path) is None
    assert T.load_cache(str(tmp_path / "missing.json")) == {}


def test_committed_entry_is_a_valid_choice():
    got = T.lookup(CFG, 3, 4096)
    assert got is not None
    for name, values in list(T.SHAPES.items()) + list(T.SCHEDULES.items()):
        assert got[name] in values, (name, got[name])
