"""Replica bookkeeping for runs on several GPUs of one node.

The refined-wall solve does not shard: each rank (one process per GPU) holds
its own copy of the reference wall and works through its own independent
refinement windows ("replicas only"; no collective on the data path).  The
only cross-rank communication is host-side: a barrier around the timed region
and the maximum of the per-rank timings.
"""
import os


def rank_info():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def schedule_seed(rank, base=17):
    """Seed of rank `rank`'s refinement schedule: distinct per rank."""
    return base + 7919 * rank


def max_over_ranks(values):
    """Element-wise maximum of a list of floats over all ranks (identity when
    torch.distributed is not initialised).  Uses a CPU tensor on gloo and a
    CUDA tensor on NCCL."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
