"""GPU parity: libmlsgd (through the C ABI) against the CPU FP64 oracle.

Tolerances (from the workload contract): relative error <= 1e-10 for the FP64
path at solver rtol 1e-13 (oracle: direct / MG-PCG at 1e-13), <= 1e-6 for the
mixed path at rtol 1e-8; sample indices and counts bit-exact.  Fields are
compared element by element against the field's max-norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc, philox  # noqa: E402
from paper_2606_09291_gb300 import inputs  # noqa: E402

TOL64 = 1e-10
TOLMIX = 1e-6


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


CFG = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0)


def oracle_workload(**over):
    c = dict(CFG)
    c.update(over)
    return mlmc.Workload(n0=c["n0"], n_levels=c["n_levels"], n_modes=c["n_modes"], corr_len=c["corr_len"],
                         sigma=c["sigma"], theta=c["theta"], alpha=c["alpha"], seed=c["seed"],
                         ctrl_level=c.get("ctrl_level"))


def test_mode_table_matches_oracle(lib):
    ctx = lib.Context(**CFG)
    idx, lam, n1d = ctx.mlsgd_mode_table()
    W = oracle_workload()
    assert [tuple(map(int, r)) for r in W.kl.idx] == idx
    assert np.abs(np.array(lam) - W.kl.lam3).max() <= 1e-15 * W.kl.lam3.max()
    ctx.close()


@pytest.mark.parametrize("S", [1, 3, 37])
def test_xi_and_field(lib, S):
    ctx = lib.Context(**CFG)
    K = CFG["n_modes"]
    xi = torch.zeros(S, K, dtype=torch.float64, device="cuda")
    for level, grid in [(1, 1), (1, 0), (2, 2)]:
        N = 8 << grid
        la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
        ctx.mlsgd_sample_field(4, level, grid, 10, S, xi=xi, log_a=la)
        ref_xi = philox.normals(0, 4, level, np.arange(10, 10 + S), K)
        assert np.abs(xi.cpu().numpy() - ref_xi).max() <= 4e-15 * np.abs(ref_xi).max()
        W = oracle_workload()
        ref_la = W.log_a(ref_xi, grid)
        assert rel_err(la.cpu().numpy(), ref_la) <= 1e-13
    ctx.close()


def _solve_both(lib, precision, grid, S, rtol, z_kind="test", **over):
    cfg = dict(CFG, rtol=rtol, max_iter=400, precision=precision)
    cfg.update(over)
    ctx = lib.Context(**cfg)
    N = 8 << grid
    Nc = 8 << cfg.get("ctrl_level", cfg["n_levels"] - 1)
    z = inputs.z_test(Nc) if z_kind == "test" else (inputs.z_random(Nc, 1, 50.0) if z_kind == "rand" else inputs.z_zero(Nc))
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
    W = oracle_workload(**over)
    las = la.cpu().numpy()
    refs = [W.solve_state_adjoint(las[s], z, grid) for s in range(S)]
    ctx.close()
    return y.cpu().numpy(), q.cpu().numpy(), phi.cpu().numpy(), it.cpu().numpy(), stt.cpu().numpy(), refs


@pytest.mark.parametrize("grid,S", [(0, 5), (1, 3), (2, 2)])
def test_state_adjoint_fp64(lib, grid, S):
    y, q, phi, it, st, refs = _solve_both(lib, "fp64", grid, S, 1e-13)
    assert np.all(st == 0) and np.all(it > 0)
    for s in range(S):
        assert rel_err(y[s], refs[s]["y"]) <= TOL64
        assert rel_err(q[s], refs[s]["q"]) <= TOL64
        assert abs(phi[s] - refs[s]["phi"]) <= TOL64 * abs(refs[s]["phi"])


@pytest.mark.parametrize("grid,S", [(0, 4), (1, 3), (2, 2)])
def test_state_adjoint_mixed(lib, grid, S):
    y, q, phi, it, st, refs = _solve_both(lib, "mixed", grid, S, 1e-8)
    assert np.all(st == 0) and np.all(it > 0)
    for s in range(S):
        assert rel_err(y[s], refs[s]["y"]) <= TOLMIX
        assert rel_err(q[s], refs[s]["q"]) <= TOLMIX
        assert abs(phi[s] - refs[s]["phi"]) <= TOLMIX * abs(refs[s]["phi"])


def test_zero_control_and_rough_control(lib):
    # z = 0: b = 0, the state is exactly 0 and Phi = 1/2 g_h^T M g_h for every sample
    y, q, phi, it, st, refs = _solve_both(lib, "fp64", 1, 2, 1e-13, z_kind="zero")
    assert not np.any(y)
    assert np.all(st == 0)
    for s in range(2):
        assert abs(phi[s] - refs[s]["phi"]) <= 1e-13 * refs[s]["phi"]
        assert rel_err(q[s], refs[s]["q"]) <= TOL64
    # a rough control (white noise on the control grid)
    y, q, phi, it, st, refs = _solve_both(lib, "fp64", 1, 2, 1e-13, z_kind="rand")
    for s in range(2):
        assert rel_err(y[s], refs[s]["y"]) <= TOL64 and rel_err(q[s], refs[s]["q"]) <= TOL64


@pytest.mark.parametrize("grid", [2, 3])
def test_zero_control_mixed(lib, grid):
    # the mixed path on the slab grids (32^3, 64^3): b = 0 takes no refinement step, the
    # first step's pass writes y = 0 exactly; the adjoint (b = -M g_h) is solved as usual
    y, q, phi, it, st, refs = _solve_both(lib, "mixed", grid, 2, 1e-8, z_kind="zero", n_levels=grid + 1)
    assert not np.any(y)
    assert np.all(st == 0)
    for s in range(2):
        assert abs(phi[s] - refs[s]["phi"]) <= 1e-12 * refs[s]["phi"]
        assert rel_err(q[s], refs[s]["q"]) <= TOLMIX


def test_batch_composition_is_bitwise_irrelevant(lib):
    """A sample's solution does not depend on which batch it is solved in."""
    y1, q1, p1, *_ = _solve_both(lib, "fp64", 1, 5, 1e-10)
    y2, q2, p2, *_ = _solve_both(lib, "fp64", 1, 2, 1e-10)
    assert np.array_equal(y1[:2], y2) and np.array_equal(q1[:2], q2) and np.array_equal(p1[:2], p2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_size_does_not_change_a_sample(lib, precision):
    """Small batches split the tiled passes' z march into more chunks than large
    ones; the partial sums are formed per fixed 8-plane segment, so a sample's
    solution is bitwise the same in a batch of 2 and in a batch of 2600 (32^3 grid:
    4 chunks against 1)."""
    cfg = dict(CFG, rtol=1e-8 if precision == "mixed" else 1e-12, max_iter=200, precision=precision,
               max_batch=4096)
    ctx = lib.Context(**cfg)
    zt = cuda(inputs.z_test(32))
    outs = []
    for S in (2, 2600):
        la = torch.zeros(S, 32 ** 3, dtype=torch.float64, device="cuda")
        ctx.mlsgd_sample_field(3, 2, 2, 0, S, log_a=la)
        y = torch.zeros(S, 33 ** 3, dtype=torch.float64, device="cuda")
        q, phi = torch.zeros_like(y), torch.zeros(S, dtype=torch.float64, device="cuda")
        it, stt = torch.zeros(S, dtype=torch.int32, device="cuda"), torch.zeros(S, dtype=torch.int32, device="cuda")
        assert ctx.mlsgd_solve_state_adjoint(2, S, la, zt, y, q, phi, it, stt) == 0, ctx.L.mlsgd_last_error(ctx.h)
        outs.append((y[:2].cpu().numpy(), q[:2].cpu().numpy(), phi[:2].cpu().numpy(), it[:2].cpu().numpy()))
        del la, y, q
    ctx.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def _oracle_level(W, level, n, z, it=0):
    r = mlmc.level_batch(W, it, level, range(n), z)
    return r


def _gpu_level(ctx, level, n, zt, it=0, splits=None):
    st = ctx.new_stats(level)
    if splits is None:
        ctx.mlsgd_level_gradient(it, level, 0, n, zt, st)
    else:
        first = 0
        for m in splits:
            ctx.mlsgd_level_gradient(it, level, first, m, zt, st)
            first += m
    return st


def _compare_stats(gpu, ref, W, tol):
    h = gpu.host()
    assert h["count"] == ref["stats"].n
    # compare in unshifted units (shifts may differ by rounding)
    fg = np.exp(W.theta * h["shift"])
    fo = np.exp(W.theta * ref["shift"])
    assert rel_err(gpu.field.cpu().numpy() * fg, ref["stats"].mean_x * fo) <= tol
    assert abs(h["mean_dy"] * fg - ref["stats"].mean_y * fo) <= tol * abs(ref["stats"].mean_y * fo) + 1e-300
    if ref["stats"].n > 1:
        t2 = max(tol, 1e-8)  # second-order sums: the path's bar, but never looser than 1e-8 for FP64
        assert abs(h["s2_dx"] * fg ** 2 - ref["stats"].s2_x * fo ** 2) <= t2 * ref["stats"].s2_x * fo ** 2
        assert abs(h["s2_dy"] * fg ** 2 - ref["stats"].s2_y * fo ** 2) <= t2 * ref["stats"].s2_y * fo ** 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_level_gradient_and_step(lib, precision):
    """Config 1 shape (levels 0..2, K = 64) with reduced counts and z = z_test."""
    rtol, tol = (1e-13, TOL64) if precision == "fp64" else (1e-8, TOLMIX)
    counts = (8, 4, 2)
    ctx = lib.Context(**dict(CFG, rtol=rtol, max_iter=400, precision=precision, theta=5.0))
    W = oracle_workload(theta=5.0)
    z = inputs.z_test(32)
    zt = cuda(z)
    stats, refs = [], []
    for l in range(3):
        stats.append(_gpu_level(ctx, l, counts[l], zt))
        refs.append(_oracle_level(W, l, counts[l], z))
        _compare_stats(stats[-1], refs[-1], W, tol)
    z_new = zt.clone()
    grad = torch.zeros_like(zt)
    rep = ctx.mlsgd_step(stats, 100.0, z_new, grad=grad)
    ref = mlmc.combine(W, [r["stats"] for r in refs], [r["shift"] for r in refs], z, 100.0)
    assert rel_err(grad.cpu().numpy(), ref["grad"]) <= tol
    assert rel_err(z_new.cpu().numpy(), ref["z_new"]) <= tol
    assert abs(rep["grad_norm"] - ref["grad_norm"]) <= tol * ref["grad_norm"]
    assert abs(rep["risk"] - ref["risk"]) <= tol * abs(ref["risk"])
    ctx.close()


def test_split_batches_merge_like_one(lib):
    ctx = lib.Context(**dict(CFG, rtol=1e-12, theta=20.0, max_batch=3))
    zt = cuda(inputs.z_test(32))
    a = _gpu_level(ctx, 1, 7, zt)                  # internal chunks of 3 (max_batch)
    b = _gpu_level(ctx, 1, 7, zt, splits=[1, 4, 2])  # caller-side splits
    ha, hb = a.host(), b.host()
    assert ha["count"] == hb["count"] == 7
    fa = a.field.cpu().numpy() * np.exp(20.0 * ha["shift"])
    fb = b.field.cpu().numpy() * np.exp(20.0 * hb["shift"])
    assert rel_err(fa, fb) <= 1e-13
    assert abs(ha["s2_dx"] - hb["s2_dx"]) <= 1e-10 * ha["s2_dx"]
    # stats_merge of two disjoint halves equals one batch
    c1 = _gpu_level(ctx, 1, 3, zt)
    c2 = ctx.new_stats(1)
    ctx.mlsgd_level_gradient(0, 1, 3, 4, zt, c2)
    ctx.mlsgd_stats_merge(c1, c2)
    hc = c1.host()
    assert hc["count"] == 7
    fc = c1.field.cpu().numpy() * np.exp(20.0 * hc["shift"])
    assert rel_err(fc, fa) <= 1e-13
    assert abs(hc["s2_dx"] - ha["s2_dx"]) <= 1e-10 * ha["s2_dx"]
    ctx.close()


def test_invalid_arguments_and_empty(lib):
    ctx = lib.Context(**CFG)
    zt = cuda(inputs.z_test(32))
    st = ctx.new_stats(1)
    ctx.mlsgd_level_gradient(0, 1, 0, 0, zt, st)  # empty batch: no-op
    assert st.host()["count"] == 0
    with pytest.raises(lib.MlsgdError):
        ctx.mlsgd_level_gradient(0, 5, 0, 2, zt, st)  # level out of range
    with pytest.raises(lib.MlsgdError):
        ctx.mlsgd_level_gradient(0, 0, 0, 2, zt, st)  # stats of another level
    with pytest.raises(lib.MlsgdError):
        ctx.mlsgd_sample_field(0, 2, 0, 0, 1, log_a=torch.zeros(512, dtype=torch.float64, device="cuda"))
    ctx.close()
    with pytest.raises(lib.MlsgdError):
        lib.Context(**dict(CFG, n_modes=63))
    with pytest.raises(lib.MlsgdError):
        lib.Context(**dict(CFG, ctrl_level=3))


def test_iteration_cap_reports_noconv(lib):
    cfg = dict(CFG, rtol=1e-14, max_iter=2, precision="fp64")
    ctx = lib.Context(**cfg)
    N = 16
    la = torch.zeros(2, N ** 3, dtype=torch.float64, device="cuda")
    ctx.mlsgd_sample_field(0, 1, 1, 0, 2, log_a=la)
    nn = (N + 1) ** 3
    y = torch.zeros(2, nn, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(y)
    phi = torch.zeros(2, dtype=torch.float64, device="cuda")
    it = torch.zeros(2, dtype=torch.int32, device="cuda")
    stt = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = ctx.mlsgd_solve_state_adjoint(1, 2, la, cuda(inputs.z_test(32)), y, q, phi, it, stt)
    assert st == 3  # MLSGD_ENOCONV
    assert np.all(stt.cpu().numpy() == 1) and np.all(it.cpu().numpy() == 4)
    ctx.close()


@pytest.mark.parametrize("ctrl_level", [0, 1])
def test_control_coarser_than_grid(lib, ctrl_level):
    """Solves and level statistics on grids finer than the control grid: B z by
    exact integration of the cellwise control, B*q as control-cell averages."""
    y, q, phi, it, st, refs = _solve_both(lib, "fp64", 2, 2, 1e-13, z_kind="rand", ctrl_level=ctrl_level)
    assert np.all(st == 0)
    for s in range(2):
        assert rel_err(y[s], refs[s]["y"]) <= TOL64 and rel_err(q[s], refs[s]["q"]) <= TOL64
        assert abs(phi[s] - refs[s]["phi"]) <= TOL64 * abs(refs[s]["phi"])
    ctx = lib.Context(**dict(CFG, rtol=1e-13, max_iter=400, theta=5.0, ctrl_level=ctrl_level))
    W = oracle_workload(theta=5.0, ctrl_level=ctrl_level)
    z = inputs.z_random(8 << ctrl_level, 3, 20.0)
    zt = cuda(z)
    for level, n in ((2, 3), (1, 4)):
        st_ = _gpu_level(ctx, level, n, zt)
        _compare_stats(st_, _oracle_level(W, level, n, z), W, TOL64)
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOLMIX)])
def test_control_much_finer_than_grid(lib, precision, tol):
    """Grid 8 (r = 8) and 16 (r = 4) under a 64^3 control grid: B z summed over the
    (2r)^3 control cells of each node's support, one block per node for r >= 8."""
    rtol = 1e-13 if precision == "fp64" else 1e-8
    for grid, S in ((0, 3), (1, 2)):
        y, q, phi, it, st, refs = _solve_both(lib, precision, grid, S, rtol, z_kind="rand", n_levels=4, ctrl_level=3)
        assert np.all(st == 0)
        for s in range(S):
            assert rel_err(y[s], refs[s]["y"]) <= tol and rel_err(q[s], refs[s]["q"]) <= tol
            assert abs(phi[s] - refs[s]["phi"]) <= tol * abs(refs[s]["phi"])
    ctx = lib.Context(**dict(CFG, rtol=rtol, max_iter=400, theta=5.0, n_levels=4, ctrl_level=3, precision=precision))
    W = oracle_workload(theta=5.0, n_levels=4, ctrl_level=3)
    z = inputs.z_random(64, 3, 20.0)
    zt = cuda(z)
    for level, n in ((0, 6), (1, 3)):
        _compare_stats(_gpu_level(ctx, level, n, zt), _oracle_level(W, level, n, z), W, tol)
    ctx.close()
