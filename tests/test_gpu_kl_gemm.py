"""GPU tests of the tensor-core KL synthesis (tcgen05 GEMM, BF16 in, FP32 accumulate).

* log a from the GEMM equals the FP64 sum of the same BF16-rounded operands
  (sigma sqrt(lambda_k) xi_k rounded to FP32 then BF16; phi_k(x_c) likewise) up to
  FP32 accumulation error: this pins the operand layouts, the swizzle, the
  descriptors and the tile mapping (a transposed or permuted tile would be off
  by O(1));
* against the exact FP64 field the error stays within the BF16 input rounding;
* a ragged sample count (tail tile) and both grids of a level difference;
* the mixed path with the tensor-core coefficient still matches the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc, philox  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def bf16_round(x):
    """Round-to-nearest-even of float32 values to BF16, returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


CFG = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0)


@pytest.mark.parametrize("level,grid,S", [(2, 2, 37), (2, 1, 130), (1, 1, 4)])
def test_gemm_matches_bf16_reference(lib, level, grid, S):
    ctx = lib.Context(**CFG)
    N = 8 << grid
    la = torch.zeros(S, N ** 3, dtype=torch.float32, device="cuda")
    ab = torch.zeros(S, N ** 3, dtype=torch.bfloat16, device="cuda")
    ctx.mlsgd_sample_field_tc(2, level, grid, 5, S, log_a_f32=la, a_bf16=ab)
    W = mlmc.Workload(n0=8, n_levels=3, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0)
    xi = philox.normals(0, 2, level, np.arange(5, 5 + S), 64)
    A = bf16_round((W.sigma * W.kl.sqrt_lam3[None, :] * xi).astype(np.float32))
    B = bf16_round(W.kl.cell_modes(N).astype(np.float32))
    ref = A @ B
    got = la.cpu().numpy().astype(np.float64)
    scale = np.abs(A) @ np.abs(B)
    # FP32 accumulation of 64 products: error well below 1e-5 of the absolute sum
    assert np.abs(got - ref).max() <= 1e-5 * scale.max()
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-6)
    exact = W.log_a(xi, grid)
    assert np.abs(got - exact).max() <= 2.0 ** -7 * scale.max()
    # the BF16 coefficient is exp of the FP32 log a, rounded
    a = ab.float().cpu().numpy().astype(np.float64)
    assert np.abs(a / np.exp(got) - 1.0).max() <= 2.0 ** -8
    ctx.close()


def test_mixed_path_with_tensor_core_coefficient(lib):
    counts = (6, 3, 2)
    cfg = dict(CFG, rtol=1e-8, max_iter=50, precision="mixed", field_tc=1, theta=5.0)
    ctx = lib.Context(**cfg)
    W = mlmc.Workload(n0=8, n_levels=3, n_modes=64, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=0)
    zn = inputs.z_test(32)
    z = torch.tensor(zn, dtype=torch.float64, device="cuda")
    stats, refs = [], []
    for l, m in enumerate(counts):
        st = ctx.new_stats(l)
        ctx.mlsgd_level_gradient(0, l, 0, m, z, st)
        stats.append(st)
        refs.append(mlmc.level_batch(W, 0, l, range(m), zn))
        h = st.host()
        assert h["noconv"] == 0
        fg, fo = np.exp(5.0 * h["shift"]), np.exp(5.0 * refs[-1]["shift"])
        f, o = st.field.cpu().numpy() * fg, refs[-1]["stats"].mean_x * fo
        assert np.abs(f - o).max() <= 1e-6 * np.abs(o).max()
    grad = torch.zeros_like(z)
    ctx.mlsgd_step(stats, 0.0, z.clone(), grad=grad)
    out = mlmc.combine(W, [r["stats"] for r in refs], [r["shift"] for r in refs], zn, 0.0)
    g = grad.cpu().numpy()
    assert np.abs(g - out["grad"]).max() <= 1e-6 * np.abs(out["grad"]).max()
    ctx.close()
