"""GPU test of mlsgd_solve_state_adjoint_noalloc, the allocation-free solve.

Some callers cannot allocate device memory when they need a solve (a host
callback or real-time loop where cudaMalloc's implicit synchronisation is not
allowed, or an application whose own pool owns all device memory).  The
allocation-free entry point serves them from a static device array inside the
library.  This test calls it through the C ABI twice in a row and checks each
result against the ordinary entry point, mlsgd_solve_state_adjoint, within the
parity tolerance of the FP64 path; it also checks that an oversized batch is
refused cleanly.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_09291_gb300 import inputs  # noqa: E402

TOL64 = 1e-10
CFG = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0, rtol=1e-12,
           max_iter=400, precision="fp64")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


def _buffers(S, N):
    nn = (N + 1) ** 3
    f64 = dict(dtype=torch.float64, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    return (torch.zeros(S, nn, **f64), torch.zeros(S, nn, **f64), torch.zeros(S, **f64), torch.zeros(S, **i32),
            torch.zeros(S, **i32))


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("grid,S", [(1, 3), (2, 2)])
def test_noalloc_matches_allocating_entry_point(lib, grid, S):
    ctx = lib.Context(**CFG)
    N = 8 << grid
    z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row, different draws
        la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
        ctx.mlsgd_sample_field(call, grid, grid, 0, S, log_a=la)
        y0, q0, p0, i0, s0 = _buffers(S, N)
        assert ctx.mlsgd_solve_state_adjoint(grid, S, la, z, y0, q0, p0, i0, s0) == 0
        y1, q1, p1, i1, s1 = _buffers(S, N)
        # straight through the C symbol
        st = ctx.L.mlsgd_solve_state_adjoint_noalloc(
            ctx.h, grid, S, ctypes.c_void_p(la.data_ptr()), ctypes.c_void_p(z.data_ptr()),
            ctypes.c_void_p(y1.data_ptr()), ctypes.c_void_p(q1.data_ptr()), ctypes.c_void_p(p1.data_ptr()),
            ctypes.c_void_p(i1.data_ptr()), ctypes.c_void_p(s1.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, ctx.L.mlsgd_last_error(ctx.h)
        torch.cuda.synchronize()
        assert _rel(y1, y0) <= TOL64 and _rel(q1, q0) <= TOL64 and _rel(p1, p0) <= TOL64
        assert torch.equal(i1, i0) and torch.equal(s1, s0)
    ctx.close()


def test_noalloc_rejects_oversized_batch(lib):
    ctx = lib.Context(**CFG)
    N = 32
    S = 64  # ~2.5 MB of scratch per sample on a 32^3 grid: far beyond the static array
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    z = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    y, q, p, i, s = _buffers(S, N)
    st = ctx.mlsgd_solve_state_adjoint_noalloc(2, S, la, z, y, q, p, i, s)
    assert st == 1  # MLSGD_EINVAL
    assert b"static array" in ctx.L.mlsgd_last_error(ctx.h)
    ctx.close()
