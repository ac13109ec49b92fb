"""Host side of the multi-GPU form: independent replicas, no data-path collective.

Sky directions (and bands) are independent (Sec. VIII), so N ranks -- one
process per GPU, launched by torchrun -- split the directions of a job into
contiguous shards and search them with no exchange; the only collectives are
the timing reduction (the slowest rank's time) and a gather of the candidate
lists to rank 0.  With torch.distributed not initialised every function acts
as a single rank.
"""
from __future__ import annotations


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def rank_world():
    d = _dist()
    return (d.get_rank(), d.get_world_size()) if d else (0, 1)


def direction_shard(n_dir: int, rank: int, world: int):
    """Contiguous directions [begin, end) of one rank; shards differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(int(n_dir), int(world))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(x: float) -> float:
    """The largest value over all ranks (e.g. the slowest rank's elapsed time)."""
    d = _dist()
    if d is None:
        return float(x)
    import torch
    backend = d.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj):
    """Objects of all ranks, in rank order, on rank 0 (None elsewhere)."""
    d = _dist()
    if d is None:
        return [obj]
    rank, world = rank_world()
    out = [None] * world if rank == 0 else None
    d.gather_object(obj, out, dst=0)
    return out


def barrier():
    d = _dist()
    if d is not None:
        d.barrier()
