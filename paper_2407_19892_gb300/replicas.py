"""Layout of the benchmark over several GPUs: independent replicas.

The benchmark's N-GPU run fits N datasets, one process per GPU, each on its
own dataset: weak scaling with no collective on the data path.  The only
collectives are the barrier around the timed region and the maximum of the
per-rank step times.  (One dataset's fit split over GPUs by cells, with its
all-reduce, broadcasts and all-gather, is ``sharded.py``.)
"""

import os


def rank_env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(seed, rank):
    """Seed of rank ``rank``'s dataset: every replica fits different data."""
    return seed + rank


def _dist_active():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def barrier(device=None):
    """All ranks meet; with a CUDA device, its queued work is finished first
    and after."""
    import torch
    import torch.distributed as dist
    if device is not None and device.type == "cuda":
        torch.cuda.synchronize(device)
    if _dist_active():
        dist.barrier()
    if device is not None and device.type == "cuda":
        torch.cuda.synchronize(device)


def max_over_ranks(x, device=None):
    """The largest of every rank's ``x`` (a step time, in ms), on every rank."""
    import torch
    import torch.distributed as dist
    if not _dist_active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job rate: the units all ranks processed over the slowest rank's
    time per step (``ms``)."""
    return world * units_per_rank / (ms / 1e3)
