"""Sample sharding and the cross-rank merge of level statistics.

Samples are independent (Sec. 2.2: the draws xi^(m,l) are iid over m and l), so
a level's batch shards by sample index with no exchange on the data path; each
rank merges its samples into its own level record with mlsgd_level_gradient.
The only exchange is the merge of the records (Algorithm 1, PairwiseUpdate;
Sec. 4.2 b): every rank all-gathers the records (mean dX~ field and the eight
scalars) and merges them pairwise in a fixed order with mlsgd_stats_merge, the
library's Chan update with rescaling to the larger shift, so every rank ends
with the same record.  The collective is an all-gather (NCCL and gloo have no
custom reduction operator); with gloo the records travel through host memory.
No merge arithmetic lives here: the Chan update exists once, in the library.
"""
import torch
import torch.distributed as dist


def shard_range(n_samples, rank, world):
    """Contiguous [first, first + count) share of n_samples for this rank."""
    base, extra = divmod(n_samples, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def gather_records(field, scalars, group=None):
    """Every rank's (field, scalars) tensors, in rank order.  NCCL gathers device
    tensors; other backends gather host copies."""
    world = dist.get_world_size(group)
    dev = field.device if dist.get_backend(group) == "nccl" else torch.device("cpu")
    f, s = field.to(dev).contiguous(), scalars.to(dev).contiguous()
    fs = [torch.empty_like(f) for _ in range(world)]
    ss = [torch.empty_like(s) for _ in range(world)]
    dist.all_gather(fs, f, group=group)
    dist.all_gather(ss, s, group=group)
    return fs, ss


def tree_merge(items, merge):
    """Merge items pairwise at distances 1, 2, 4, ... (item i takes item i + d for i a
    multiple of 2d, the pairing of Algorithm 1's PairwiseUpdate); merge(dst, src)
    merges src into dst in place.  Returns items[0], the merge of all."""
    n, d = len(items), 1
    while d < n:
        for i in range(0, n - d, 2 * d):
            merge(items[i], items[i + d])
        d *= 2
    return items[0]


def allgather_merge(ctx, stats, group=None):
    """The merge of every rank's level record `stats` (an mlsgd.Stats of ctx's
    workload), formed on this rank's device with ctx.mlsgd_stats_merge.  Returns a
    new mlsgd.Stats; `stats` is left unchanged."""
    from .mlsgd import Stats
    fs, ss = gather_records(stats.field, stats.scalars, group)
    recs = []
    for f, s in zip(fs, ss):
        r = Stats(stats.level, stats.field.numel(), device=stats.field.device)
        r.field.copy_(f)
        r.scalars.copy_(s)
        recs.append(r)
    return tree_merge(recs, ctx.mlsgd_stats_merge)
