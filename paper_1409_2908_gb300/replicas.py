"""Host-side logic of multi-GPU runs.  The product has no exchange step, so N
GPUs run N independent replicas of the same workload (weak scaling); the only
collective is on the host: a barrier before and after the timed region and
the maximum of the per-rank times.  Works with any torch.distributed backend
(NCCL on GPUs, gloo on CPU for tests)."""
import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, device="cpu"):
    """Maximum of a per-rank float over all ranks (x itself when not
    distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(per_rank_units, elapsed_ms, device="cpu"):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time (per second).  Returns (units_per_s, max_ms)."""
    import torch.distributed as dist
    ws = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    t = max_over_ranks(elapsed_ms, device)
    return ws * per_rank_units / (t / 1e3), t


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
