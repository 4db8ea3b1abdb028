"""Multi-GPU form of the method: independent replicas, one process per GPU.

Frame pairs are independent problems (the method has no exchange between pairs), so N GPUs
run N replicas of the single-GPU pipeline on disjoint shares of the pairs, with no collective
on the data path.  The only communication is host-side bookkeeping: a barrier around timed
regions and the maximum of the ranks' times, taken with torch.distributed (NCCL between GPUs,
gloo on CPU for the tests).
"""


def env_rank_world():
    """(rank, local_rank, world_size) from the torchrun environment (1 process when unset)."""
    import os
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(n_items, rank, world):
    """Contiguous share [lo, hi) of n_items for `rank` of `world`: the first n_items % world
    ranks take one item more; the shares are disjoint and cover all items."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad shard request: n=%r rank=%r world=%r" % (n_items, rank, world))
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity with one process)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def barrier():
    """Barrier over all ranks (no-op with one process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def aggregate_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    if seconds_max <= 0:
        raise ValueError("non-positive time")
    return world * units_per_rank / seconds_max
