"""Oracle check of the large-risk-aversion workload on levels 0-2: 512 modes,
correlation length 0.1, sigma 1.5, theta = 100 (the entropic weights span many
orders of magnitude, so the per-level shifts and their rescaling at the combine
step are exercised), FP64 (<= 1e-10 at rtol 1e-13) and mixed (<= 1e-6 at rtol
1e-8) paths through the C ABI against the CPU FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402

CFG = dict(n_levels=3, n0=8, n_modes=512, corr_len=0.1, sigma=1.5, theta=100.0, alpha=1e-4, seed=11)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def rel_err(gpu, ref):
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return np.abs(gpu - ref).max() / (scale if scale > 0 else 1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c5_levels_0_to_2(lib, precision):
    rtol, tol = (1e-13, 1e-10) if precision == "fp64" else (1e-8, 1e-6)
    ctx = lib.Context(**dict(CFG, rtol=rtol, max_iter=600, precision=precision))
    W = mlmc.Workload(**CFG)
    z = inputs.z_test(32)
    zt = torch.tensor(z, dtype=torch.float64, device="cuda")
    counts = (6, 3, 2)
    stats, refs = [], []
    for l in range(3):
        st = ctx.new_stats(l)
        ctx.mlsgd_level_gradient(2, l, 0, counts[l], zt, st)
        ref = mlmc.level_batch(W, 2, l, range(counts[l]), z)
        h = st.host()
        assert h["count"] == counts[l] and h["noconv"] == 0
        fg, fo = np.exp(W.theta * h["shift"]), np.exp(W.theta * ref["shift"])
        assert rel_err(st.field.cpu().numpy() * fg, ref["stats"].mean_x * fo) <= tol
        assert abs(h["mean_dy"] * fg - ref["stats"].mean_y * fo) <= tol * abs(ref["stats"].mean_y * fo)
        t2 = max(tol, 1e-8)
        assert abs(h["s2_dx"] * fg ** 2 - ref["stats"].s2_x * fo ** 2) <= t2 * ref["stats"].s2_x * fo ** 2
        stats.append(st)
        refs.append(ref)
    z_new = zt.clone()
    grad = torch.zeros_like(zt)
    rep = ctx.mlsgd_step(stats, 10.0, z_new, grad=grad)
    ref = mlmc.combine(W, [r["stats"] for r in refs], [r["shift"] for r in refs], z, 10.0)
    assert rel_err(grad.cpu().numpy(), ref["grad"]) <= tol
    assert abs(rep["risk"] - ref["risk"]) <= tol * abs(ref["risk"])
    assert rep["truncated"] == int(ref["truncated"])
    ctx.close()
