"""GPU parity on the paper's Sec. 5 workload: cos-product KL field with m^3 = 125
modes, lambda_jkl = exp(-pi (j + k + l) rho), rho = 0.15, xi ~ U(-4, 4), target
g = prod sin(2 pi x_i); the CUDA path through the C ABI against the CPU FP64
oracle, FP64 (<= 1e-10 at rtol 1e-13) and mixed (<= 1e-6 at rtol 1e-8)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc, philox  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402

TOL64 = 1e-10
TOLMIX = 1e-6
CFG = dict(n_levels=3, n0=8, n_modes=125, corr_len=0.15, sigma=1.0, theta=8.0, alpha=1e-4, seed=5,
           field_model=1, target_freq=2)


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


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def oracle_workload(**over):
    c = dict(CFG)
    c.update(over)
    return mlmc.Workload(n0=c["n0"], n_levels=c["n_levels"], n_modes=c["n_modes"], corr_len=c["corr_len"],
                         sigma=c["sigma"], theta=c["theta"], alpha=c["alpha"], seed=c["seed"],
                         field_model=1, target_freq=2)


def test_paper_mode_table(lib):
    ctx = lib.Context(**CFG)
    idx, lam, n1d = ctx.mlsgd_mode_table()
    W = oracle_workload()
    assert n1d == 5
    assert [tuple(map(int, r)) for r in W.kl.idx] == idx
    assert np.abs(np.array(lam) - W.kl.lam3).max() <= 1e-15 * W.kl.lam3.max()
    ctx.close()


@pytest.mark.parametrize("S", [1, 6])
def test_uniform_xi_and_cos_field(lib, S):
    ctx = lib.Context(**CFG)
    K = CFG["n_modes"]
    W = oracle_workload()
    xi = torch.zeros(S, K, dtype=torch.float64, device="cuda")
    for level, grid in [(0, 0), (2, 1), (2, 2)]:
        N = 8 << grid
        la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
        ctx.mlsgd_sample_field(3, level, grid, 20, S, xi=xi, log_a=la)
        ref_xi = philox.uniforms(CFG["seed"], 3, level, np.arange(20, 20 + S), K, 4.0)
        g = xi.cpu().numpy()
        assert np.abs(g - ref_xi).max() <= 4e-15 * 4.0
        assert g.min() > -4.0 and g.max() <= 4.0
        assert rel_err(la.cpu().numpy(), W.log_a(ref_xi, grid)) <= 1e-13
    ctx.close()


def _solve_both(lib, precision, grid, S, rtol):
    ctx = lib.Context(**dict(CFG, rtol=rtol, max_iter=600, precision=precision))
    N = 8 << grid
    z = inputs.z_test(32, freq=2)
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    ctx.mlsgd_sample_field(0, grid, grid, 0, S, log_a=la)
    nn = (N + 1) ** 3
    y = torch.zeros(S, nn, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(y)
    phi = torch.zeros(S, dtype=torch.float64, device="cuda")
    it = torch.zeros(S, dtype=torch.int32, device="cuda")
    stt = torch.zeros(S, dtype=torch.int32, device="cuda")
    st = ctx.mlsgd_solve_state_adjoint(grid, S, la, cuda(z), y, q, phi, it, stt)
    assert st == 0, ctx.L.mlsgd_last_error(ctx.h)
    W = oracle_workload()
    las = la.cpu().numpy()
    refs = [W.solve_state_adjoint(las[s], z, grid) for s in range(S)]
    ctx.close()
    return y.cpu().numpy(), q.cpu().numpy(), phi.cpu().numpy(), stt.cpu().numpy(), refs


@pytest.mark.parametrize("precision,grid,S", [("fp64", 0, 3), ("fp64", 2, 2), ("mixed", 1, 3), ("mixed", 2, 2)])
def test_paper_state_adjoint(lib, precision, grid, S):
    rtol, tol = (1e-13, TOL64) if precision == "fp64" else (1e-8, TOLMIX)
    y, q, phi, st, refs = _solve_both(lib, precision, grid, S, rtol)
    assert np.all(st == 0)
    for s in range(S):
        assert rel_err(y[s], refs[s]["y"]) <= tol
        assert rel_err(q[s], refs[s]["q"]) <= tol
        assert abs(phi[s] - refs[s]["phi"]) <= tol * abs(refs[s]["phi"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_level_gradient_and_step(lib, precision):
    rtol, tol = (1e-13, TOL64) if precision == "fp64" else (1e-8, TOLMIX)
    counts = (6, 3, 2)
    ctx = lib.Context(**dict(CFG, rtol=rtol, max_iter=600, precision=precision))
    W = oracle_workload()
    z = inputs.z_test(32, freq=2)
    zt = cuda(z)
    stats, refs = [], []
    for l in range(3):
        st = ctx.new_stats(l)
        ctx.mlsgd_level_gradient(1, l, 0, counts[l], zt, st)
        ref = mlmc.level_batch(W, 1, l, range(counts[l]), z)
        h = st.host()
        assert h["count"] == ref["stats"].n
        fg, fo = np.exp(W.theta * h["shift"]), np.exp(W.theta * ref["shift"])
        assert rel_err(st.field.cpu().numpy() * fg, ref["stats"].mean_x * fo) <= tol
        assert abs(h["mean_dy"] * fg - ref["stats"].mean_y * fo) <= tol * abs(ref["stats"].mean_y * fo)
        stats.append(st)
        refs.append(ref)
    z_new = zt.clone()
    grad = torch.zeros_like(zt)
    rep = ctx.mlsgd_step(stats, 50.0, z_new, grad=grad)
    ref = mlmc.combine(W, [r["stats"] for r in refs], [r["shift"] for r in refs], z, 50.0)
    assert rel_err(grad.cpu().numpy(), ref["grad"]) <= tol
    assert rel_err(z_new.cpu().numpy(), ref["z_new"]) <= tol
    assert abs(rep["risk"] - ref["risk"]) <= tol * abs(ref["risk"])
    ctx.close()
