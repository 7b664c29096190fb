"""Multi-rank path on CPU (gloo, world size 2): sharded samples, all-gather and Chan
merge of the level records equal a single-process run (oracle records)."""
import os
import socket

import numpy as np
import pytest
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


def _record(W, level, samples, z):
    from oracle import mlmc
    r = mlmc.level_batch(W, 0, level, samples, z)
    st = r["stats"]
    sc = np.zeros(8)
    sc[D.COUNT], sc[D.SHIFT], sc[D.MEAN_DY], sc[D.S2_DY], sc[D.S2_DX] = st.n, r["shift"], st.mean_y, st.s2_y, st.s2_x
    return st.mean_x, sc


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle import mlmc
    from paper_2606_09291_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W = mlmc.Workload(n0=4, n_levels=2, n_modes=16, corr_len=0.3, sigma=1.0, theta=20.0, alpha=1e-4, seed=1)
    z = inputs.z_test(8)
    first, cnt = D.shard_range(7, rank, world)
    f, sc = _record(W, 1, range(first, first + cnt), z)
    mf, msc = D.allgather_merge(f, sc, W.theta, W.hc3)
    out.put((rank, mf, msc))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.timeout(300)
def test_two_rank_merge_equals_single_process():
    from oracle import mlmc
    from paper_2606_09291_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    W = mlmc.Workload(n0=4, n_levels=2, n_modes=16, corr_len=0.3, sigma=1.0, theta=20.0, alpha=1e-4, seed=1)
    f1, sc1 = _record(W, 1, range(7), inputs.z_test(8))
    for _, mf, msc in res:
        assert msc[D.COUNT] == 7
        # compare in unshifted units
        g = np.exp(W.theta * msc[D.SHIFT]) / np.exp(W.theta * sc1[D.SHIFT])
        assert np.abs(mf * g - f1).max() <= 1e-12 * np.abs(f1).max()
        assert abs(msc[D.MEAN_DY] * g - sc1[D.MEAN_DY]) <= 1e-12 * abs(sc1[D.MEAN_DY])
        assert abs(msc[D.S2_DX] * g * g - sc1[D.S2_DX]) <= 1e-10 * sc1[D.S2_DX]
        assert abs(msc[D.S2_DY] * g * g - sc1[D.S2_DY]) <= 1e-10 * sc1[D.S2_DY]
