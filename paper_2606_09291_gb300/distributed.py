"""Sample sharding and the cross-rank merge of level statistics.

Samples are independent (Sec. 2.2: the draws xi^(m,l) are iid over m and l), so
a level's batch shards by sample index with no exchange on the data path; each
rank merges its samples into its own level record with mlsgd_level_gradient.
The only exchange is the merge of the records (Algorithm 1, PairwiseUpdate;
Sec. 4.2 b): every rank gathers all records (count, shift, mean of dY~,
second-order sums, mean dX~ field) and merges them pairwise in rank order
with the Chan update after rescaling to the largest shift.  The collective is
an all-gather (NCCL/gloo have no custom reduction operator).  Host-side FP64
arithmetic on gathered records; the per-rank record itself is produced on the
GPU.
"""
import numpy as np
import torch
import torch.distributed as dist

# record layout (matches mlsgd_level_stats scalars)
COUNT, SHIFT, MEAN_DY, S2_DY, S2_DX, PHI_MAX, ITERS, NOCONV = range(8)


def shard_range(n_samples, rank, world):
    """Contiguous [first, first + count) share of n_samples for this rank."""
    base, extra = divmod(n_samples, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def merge_records(a_field, a_sc, b_field, b_sc, theta, hc3):
    """Chan merge of two level records (FP64 numpy); returns (field, scalars)."""
    na, nb = a_sc[COUNT], b_sc[COUNT]
    if nb == 0:
        return a_field.copy(), a_sc.copy()
    if na == 0:
        return b_field.copy(), b_sc.copy()
    shift = max(a_sc[SHIFT], b_sc[SHIFT])
    fa, fb = np.exp(theta * (a_sc[SHIFT] - shift)), np.exp(theta * (b_sc[SHIFT] - shift))
    n = na + nb
    xa, xb = a_field * fa, b_field * fb
    dx = xa - xb
    field = xb + (na / n) * dx
    ya, yb = a_sc[MEAN_DY] * fa, b_sc[MEAN_DY] * fb
    dy = ya - yb
    sc = np.zeros_like(a_sc)
    sc[COUNT] = n
    sc[SHIFT] = shift
    sc[MEAN_DY] = yb + (na / n) * dy
    sc[S2_DY] = a_sc[S2_DY] * fa * fa + b_sc[S2_DY] * fb * fb + dy * dy * na * nb / n
    sc[S2_DX] = a_sc[S2_DX] * fa * fa + b_sc[S2_DX] * fb * fb + hc3 * float(dx @ dx) * na * nb / n
    sc[PHI_MAX] = max(a_sc[PHI_MAX], b_sc[PHI_MAX])
    sc[ITERS] = a_sc[ITERS] + b_sc[ITERS]
    sc[NOCONV] = a_sc[NOCONV] + b_sc[NOCONV]
    return field, sc


def allgather_merge(field, scalars, theta, hc3, group=None):
    """Gather every rank's record (CPU tensors or numpy) and merge pairwise in rank
    order (distance-doubling tree over ranks).  Returns (field, scalars) as numpy."""
    world = dist.get_world_size(group)
    f = torch.as_tensor(np.asarray(field, dtype=np.float64))
    s = torch.as_tensor(np.asarray(scalars, dtype=np.float64))
    fs = [torch.empty_like(f) for _ in range(world)]
    ss = [torch.empty_like(s) for _ in range(world)]
    dist.all_gather(fs, f, group=group)
    dist.all_gather(ss, s, group=group)
    recs = [(fs[r].numpy(), ss[r].numpy()) for r in range(world)]
    d = 1
    while d < world:
        for i in range(0, world - d, 2 * d):
            recs[i] = merge_records(recs[i][0], recs[i][1], recs[i + d][0], recs[i + d][1], theta, hc3)
        d *= 2
    return recs[0]
