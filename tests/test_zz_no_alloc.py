"""GPU test of mlsgd_solve_state_adjoint_noalloc, the allocation-free solve.

Some callers cannot allocate device memory when they need a solve: a
latency-critical loop in which cudaMalloc's implicit device-wide
synchronisation is not acceptable, or an application whose own allocator has
reserved the device memory and does not let libraries call the CUDA allocator.
The allocation-free entry point serves them from a static device array inside
the library.

The tests call it through the C ABI, two calls in a row, and check each result
against the ordinary entry point, mlsgd_solve_state_adjoint, within the parity
tolerance of the precision used (1e-10 FP64, 1e-6 mixed).  The allocation-free
calls run on a fresh context whose workspace was never grown, and the device's
free memory is compared before and after them, so an accidental allocation on
that path would show.  A larger call precedes a smaller one, so the smaller one
starts from the larger one's leftovers in the shared array.  A batch above 8192
samples checks the status read-back at any batch size, and an oversized batch
must be refused cleanly.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_09291_gb300 import inputs  # noqa: E402

TOL = {"fp64": 1e-10, "mixed": 1e-6}
BASE = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0)
CFG = {"fp64": dict(BASE, rtol=1e-12, max_iter=400, precision="fp64"),
       "mixed": dict(BASE, rtol=1e-8, max_iter=50, precision="mixed")}


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
    return [torch.zeros(S, nn, **f64), torch.zeros(S, nn, **f64), torch.zeros(S, **f64), torch.zeros(S, **i32),
            torch.zeros(S, **i32)]


def _noalloc(ctx, grid, S, la, z, out):
    """Straight through the C symbol (no binding helper in between)."""
    y, q, p, i, s = out
    return ctx.L.mlsgd_solve_state_adjoint_noalloc(
        ctx.h, grid, S, ctypes.c_void_p(la.data_ptr()), ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(y.data_ptr()),
        ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(i.data_ptr()),
        ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point(lib, precision):
    cfg = CFG[precision]
    tol = TOL[precision]
    # (grid, samples) per call: the larger call first, then a smaller one on another grid
    calls = [(2, 4 if precision == "mixed" else 2), (1, 3)]
    z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    ref_ctx, fresh = lib.Context(**cfg), lib.Context(**cfg)
    fields, refs, outs = [], [], []
    for k, (grid, S) in enumerate(calls):
        N = 8 << grid
        la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
        ref_ctx.mlsgd_sample_field(k, grid, grid, 0, S, log_a=la)
        ref = _buffers(S, N)
        assert ref_ctx.mlsgd_solve_state_adjoint(grid, S, la, z, *ref) == 0, ref_ctx.L.mlsgd_last_error(ref_ctx.h)
        fields.append(la)
        refs.append(ref)
        outs.append(_buffers(S, N))
    # the first call on this device (symbol look-up, kernels loaded) on a context of its own
    warm = lib.Context(**cfg)
    grid, S = calls[-1]
    assert _noalloc(warm, grid, S, fields[-1], z, _buffers(S, 8 << grid)) == 0, warm.L.mlsgd_last_error(warm.h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for (grid, S), la, out in zip(calls, fields, outs):  # two calls in a row on a context never grown
        st = _noalloc(fresh, grid, S, la, z, out)
        assert st == 0, fresh.L.mlsgd_last_error(fresh.h)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0, "the allocation-free path took %d bytes of device memory" % (free0 - free1)
    for ref, out in zip(refs, outs):
        y0, q0, p0, i0, s0 = ref
        y1, q1, p1, i1, s1 = out
        assert _rel(y1, y0) <= tol and _rel(q1, q0) <= tol and _rel(p1, p0) <= tol
        assert torch.equal(i1, i0) and torch.equal(s1, s0) and int(s1.abs().sum()) == 0
    for c in (ref_ctx, fresh, warm):
        c.close()


def test_noalloc_status_of_a_batch_above_8192_samples(lib):
    # 2^3 cells per sample (one unknown), mixed precision: about 1.6 KB of scratch per sample
    cfg = dict(n_levels=1, n0=2, ctrl_level=0, n_modes=8, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0,
               rtol=1e-8, max_iter=50, precision="mixed")
    S, N = 10000, 2
    ctx = lib.Context(**cfg)
    z = torch.tensor(inputs.z_test(N), dtype=torch.float64, device="cuda")
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    ctx.mlsgd_sample_field(0, 0, 0, 0, S, log_a=la)
    ref, out = _buffers(S, N), _buffers(S, N)
    assert ctx.mlsgd_solve_state_adjoint(0, S, la, z, *ref) == 0, ctx.L.mlsgd_last_error(ctx.h)
    for _ in range(2):
        st = _noalloc(ctx, 0, S, la, z, out)
        assert st == 0, ctx.L.mlsgd_last_error(ctx.h)
        torch.cuda.synchronize()
        assert _rel(out[0], ref[0]) <= TOL["mixed"] and _rel(out[1], ref[1]) <= TOL["mixed"]
        assert torch.equal(out[4], ref[4]) and int(out[4].abs().sum()) == 0
    ctx.close()


def test_noalloc_rejects_oversized_batch(lib):
    ctx = lib.Context(**CFG["fp64"])
    N = 32
    S = 64  # ~2.5 MB of scratch per sample on a 32^3 grid: far beyond the static array
    la = torch.zeros(S, N ** 3, dtype=torch.float64, device="cuda")
    z = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    st = _noalloc(ctx, 2, S, la, z, _buffers(S, N))
    assert st == 1  # MLSGD_EINVAL
    assert b"static array" in ctx.L.mlsgd_last_error(ctx.h)
    ctx.close()
