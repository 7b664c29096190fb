"""A whole level batch (fields, both grids' state and adjoint solves, statistics) as
one CUDA graph: with a fixed number of refinement steps mlsgd_level_gradient enqueues
only stream work, so it can be captured once and replayed; the replay reproduces
the direct call bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_09291_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def test_level_gradient_captured_in_a_graph(lib):
    cfg = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=0, rtol=1e-8,
               max_iter=50, precision="mixed", field_tc=1, ir_steps=3, max_batch=16)
    ctx = lib.Context(**cfg)
    z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    direct = ctx.new_stats(2)
    ctx.mlsgd_level_gradient(7, 2, 0, 16, z, direct)  # also sizes the scratch and builds tables
    torch.cuda.synchronize()
    st = ctx.new_stats(2)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.mlsgd_stats_reset(st)
        ctx.mlsgd_level_gradient(7, 2, 0, 16, z, st)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(st.field, direct.field)
        assert torch.equal(st.scalars, direct.scalars)
    h = direct.host()
    assert h["count"] == 16 and h["noconv"] == 0
    ctx.close()
