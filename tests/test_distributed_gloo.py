"""Multi-rank path: sample sharding, the all-gather of level records and their
pairwise merge (world size 2, gloo).

On the CPU the host logic is checked with records that are plain tensors and a
merge that records its pairing: every rank gathers all records in rank order and
merges them in the same fixed tree, so all ranks hold the same result.  The GPU
test (two ranks sharing one GPU; their kernels never wait on each other, the
records travel through host memory) merges library records with the library's
own mlsgd_stats_merge and compares them with one single-process call over all
samples."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2606_09291_gb300 import distributed as D


def test_shard_range_covers_exactly():
    for n in (0, 1, 7, 64):
        for world in (1, 2, 3, 8):
            parts = [D.shard_range(n, r, world) for r in range(world)]
            covered = []
            for first, cnt in parts:
                covered.extend(range(first, first + cnt))
            assert covered == list(range(n))


def test_tree_merge_pairing():
    for n in range(1, 9):
        items = [[i] for i in range(n)]
        pairs = []

        def merge(a, b):
            pairs.append((a[0], b[0]))
            a.extend(b)

        out = D.tree_merge(items, merge)
        assert sorted(out) == list(range(n)) and len(pairs) == n - 1
        # distance-doubling pairing: 0+1, 2+3, ..., then 0+2, ..., then 0+4
        d, expect = 1, []
        while d < n:
            expect += [(i, i + d) for i in range(0, n - d, 2 * d)]
            d *= 2
        assert pairs == expect


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _host_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    field = torch.full((5,), float(rank + 1), dtype=torch.float64)
    scalars = torch.arange(8, dtype=torch.float64) + 10 * rank
    fs, ss = D.gather_records(field, scalars)
    items = [[(int(f[0].item()), int(s[0].item()))] for f, s in zip(fs, ss)]
    merged = D.tree_merge(items, lambda a, b: a.extend(b))
    out.put((rank, merged))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_gather_and_tree_on_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_host_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [(1, 0), (2, 10)]


CFG = dict(n_levels=2, n0=8, n_modes=16, corr_len=0.3, sigma=1.0, theta=20.0, alpha=1e-4, seed=1, rtol=1e-12,
           max_iter=400, precision="fp64")
N_SAMPLES = 7


def _gpu_worker(rank, world, port, out):
    import torch.distributed as dist

    import __graft_entry__
    from paper_2606_09291_gb300 import inputs, mlsgd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if rank == 0:
        __graft_entry__.build()
    dist.barrier()
    mlsgd.load()
    torch.cuda.set_device(0)
    ctx = mlsgd.Context(**CFG)
    zt = torch.tensor(inputs.z_test(16), dtype=torch.float64, device="cuda")
    first, cnt = D.shard_range(N_SAMPLES, rank, world)
    st = ctx.new_stats(1)
    ctx.mlsgd_level_gradient(0, 1, first, cnt, zt, st)
    m = D.allgather_merge(ctx, st)
    out.put((rank, m.field.cpu().numpy(), m.scalars.cpu().numpy(), st.host()["count"]))
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.timeout(600)
def test_two_rank_library_merge_equals_single_process():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import inputs, mlsgd
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=500) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = mlsgd.Context(**CFG)
    one = c.new_stats(1)
    c.mlsgd_level_gradient(0, 1, 0, N_SAMPLES, torch.tensor(inputs.z_test(16), dtype=torch.float64, device="cuda"),
                           one)
    f1, s1 = one.field.cpu().numpy(), one.scalars.cpu().numpy()
    c.close()
    theta = CFG["theta"]
    assert sorted(r[3] for r in res) == [3, 4]  # each rank merged its own shard
    for _, f, s, _ in res:
        assert s[0] == N_SAMPLES
        g = np.exp(theta * (s[1] - s1[1]))  # compare in unshifted units
        assert np.abs(f * g - f1).max() <= 1e-12 * np.abs(f1).max()
        assert abs(s[2] * g - s1[2]) <= 1e-12 * abs(s1[2])
        assert abs(s[3] * g * g - s1[3]) <= 1e-10 * s1[3] and abs(s[4] * g * g - s1[4]) <= 1e-10 * s1[4]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
