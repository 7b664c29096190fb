"""GPU tests of the failure paths and of the compacted launches.

Failure detection is exercised without any GPU fault: a non-finite control
(the per-sample status flags and MLSGD_ENONFINITE), a scratch request the
device cannot satisfy (a failed cudaMalloc, MLSGD_ENOMEM, with the context
usable afterwards) and the iteration cap (in test_gpu_parity.py).  The
compaction test checks that launching only the still-active samples (the
host-checked refinement) gives bit for bit the records of the masked fixed-step
form, whose launches cover every sample.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_09291_gb300 import inputs  # noqa: E402

CFG = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0)
ENONFINITE, ENOMEM = 4, 2


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def _solve(ctx, grid, S, z):
    N = 8 << grid
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    ctx.mlsgd_sample_field(0, grid, grid, 0, S, log_a=la)
    nn = (N + 1) ** 3
    y = torch.zeros(S, nn, dtype=torch.float64, device="cuda")
    q, phi = torch.zeros_like(y), torch.zeros(S, dtype=torch.float64, device="cuda")
    it, stt = torch.zeros(S, dtype=torch.int32, device="cuda"), torch.zeros(S, dtype=torch.int32, device="cuda")
    st = ctx.mlsgd_solve_state_adjoint(grid, S, la, z, y, q, phi, it, stt)
    return st, stt.cpu().numpy(), y


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("mixed", 1e-8)])
def test_nonfinite_control(lib, precision, rtol):
    ctx = lib.Context(**dict(CFG, rtol=rtol, max_iter=100, precision=precision))
    z = inputs.z_test(32)
    z[1000] = np.nan
    zt = torch.tensor(z, dtype=torch.float64, device="cuda")
    for grid in (1, 2):  # plain kernels and tiled passes
        st, flags, _ = _solve(ctx, grid, 3, zt)
        assert st == ENONFINITE, ctx.L.mlsgd_last_error(ctx.h)
        assert np.all(flags & 2)
    # an infinite control value as well
    z[1000] = np.inf
    st, flags, _ = _solve(ctx, 2, 2, torch.tensor(z, dtype=torch.float64, device="cuda"))
    assert st == ENONFINITE and np.all(flags & 2)
    # through the level gradient the records turn non-finite and the step refuses them
    stats = [ctx.new_stats(l) for l in range(2)]
    for l in range(2):
        ctx.mlsgd_level_gradient(0, l, 0, 3, zt, stats[l])
    assert stats[1].host()["noconv"] > 0
    with pytest.raises(lib.MlsgdError) as e:
        ctx.mlsgd_step(stats, 1.0, zt.clone())
    assert e.value.status == ENONFINITE
    # the context still works with a finite control
    st, flags, y = _solve(ctx, 1, 2, torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda"))
    assert st == 0 and not np.any(flags) and bool(torch.isfinite(y).all())
    ctx.close()


def test_scratch_allocation_failure(lib):
    # one chunk of 2^20 level-2 samples asks for far more scratch than the device holds
    ctx = lib.Context(**dict(CFG, rtol=1e-8, precision="mixed", max_batch=1 << 20))
    need = ctx.mlsgd_workspace_bytes(2, 1 << 20)
    assert need > torch.cuda.get_device_properties(0).total_memory
    zt = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    st = ctx.new_stats(2)
    with pytest.raises(lib.MlsgdError) as e:
        ctx.mlsgd_level_gradient(0, 2, 0, 1 << 20, zt, st)
    assert e.value.status == ENOMEM
    assert st.host()["count"] == 0
    # the context recovers: a small batch runs afterwards
    ctx.mlsgd_level_gradient(0, 2, 0, 2, zt, st)
    assert st.host()["count"] == 2 and st.host()["noconv"] == 0
    ctx.close()


@pytest.mark.parametrize("level", [1, 2])
def test_compacted_launches_match_masked_steps(lib, level):
    """ir_steps = 0 launches only the samples still above rtol in each refinement step;
    ir_steps = 3 launches every sample and masks the converged ones.  A sample's
    arithmetic is the same in both, so the records agree bit for bit."""
    base = dict(CFG, rtol=1e-8, max_iter=50, precision="mixed", theta=5.0)
    zt = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    recs = []
    for ir in (3, 0):
        ctx = lib.Context(**dict(base, ir_steps=ir))
        st = ctx.new_stats(level)
        ctx.mlsgd_level_gradient(2, level, 0, 9, zt, st)
        recs.append((st.field.cpu().numpy(), st.scalars.cpu().numpy()))
        ctx.close()
    (f0, s0), (f1, s1) = recs
    assert s0[0] == s1[0] == 9 and s0[7] == s1[7] == 0  # count, no unconverged solve
    assert np.array_equal(f0, f1) and np.array_equal(s0, s1)
