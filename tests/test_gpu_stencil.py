"""GPU check of the two families of fused solver passes against each other.

The mixed path runs its FP32 passes on 32^3 and 64^3 grids as whole-row slab
kernels staged by bulk copies (stencil 0) and elsewhere as z-marching tile
kernels; stencil 1 forces the tile kernels everywhere.  Both evaluate the same
Q1 operator, Jacobi smoother and transfers in FP32, so after a fixed number of
refinement steps their iterates agree to FP32 rounding amplified by a few PCG
iterations, and converged solves agree within the solver tolerance with the
same iteration counts.  A wrong operator or a wrong preconditioner in either
family shows up as a large difference after one refinement step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_09291_gb300 import inputs  # noqa: E402

BASE = dict(n_levels=4, n0=8, n_modes=64, corr_len=0.2, sigma=1.0, theta=5.0, alpha=1e-4, seed=0, rtol=1e-8,
            max_iter=50, precision="mixed")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def _solve(lib, grid, S, **over):
    ctx = lib.Context(**dict(BASE, **over))
    N = 8 << grid
    zt = torch.tensor(inputs.z_test(64), dtype=torch.float64, device="cuda")
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    ctx.mlsgd_sample_field(1, grid, grid, 0, S, log_a=la)
    y = torch.zeros(S, (N + 1) ** 3, dtype=torch.float64, device="cuda")
    q, phi = torch.zeros_like(y), torch.zeros(S, dtype=torch.float64, device="cuda")
    it, stt = torch.zeros(S, dtype=torch.int32, device="cuda"), torch.zeros(S, dtype=torch.int32, device="cuda")
    st = ctx.mlsgd_solve_state_adjoint(grid, S, la, zt, y, q, phi, it, stt)
    ctx.close()
    return st, y.cpu().numpy(), q.cpu().numpy(), phi.cpu().numpy(), it.cpu().numpy(), stt.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("grid,S", [(2, 5), (3, 3)])
def test_one_refinement_step_agrees(lib, grid, S):
    outs = [_solve(lib, grid, S, ir_steps=1, stencil=v) for v in (0, 1)]
    (_, y0, q0, p0, i0, _), (_, y1, q1, p1, i1, _) = outs
    assert np.array_equal(i0, i1)
    assert _rel(y0, y1) <= 1e-4 and _rel(q0, q1) <= 1e-4
    assert np.abs(p0 - p1).max() <= 1e-4 * np.abs(p1).max()


@pytest.mark.parametrize("grid,S", [(2, 6), (3, 4)])
def test_converged_solves_agree(lib, grid, S):
    outs = [_solve(lib, grid, S, stencil=v) for v in (0, 1)]
    for st, *_rest, flags in outs:
        assert st == 0 and not np.any(flags)
    (_, y0, q0, p0, i0, _), (_, y1, q1, p1, i1, _) = outs
    assert _rel(y0, y1) <= 1e-7 and _rel(q0, q1) <= 1e-7
    assert np.abs(p0 - p1).max() <= 1e-7 * np.abs(p1).max()
    assert abs(int(i0.sum()) - int(i1.sum())) <= 12  # at most two extra refinement steps over the batch


@pytest.mark.parametrize("grid", [2, 3])
def test_z_chunks_and_omega_leave_the_solution(lib, grid):
    """Forced z chunking changes the launch only (bitwise: the fused restriction's
    chunks overlap by one plane, the coarse rows shared by two row blocks take exactly
    two additions); another smoother damping changes the iterates but not the
    converged solution beyond the tolerance."""
    ref = _solve(lib, grid, 2)
    for zc in (1, 2, 4, 8):
        out = _solve(lib, grid, 2, z_chunks=zc)
        assert all(np.array_equal(a, b) for a, b in zip(out[1:], ref[1:]))
    out = _solve(lib, grid, 2, omega=0.5)
    assert out[0] == 0 and _rel(out[1], ref[1]) <= 1e-7 and _rel(out[2], ref[2]) <= 1e-7
