"""Host logic of the multi-GPU mode: one independent box per rank (the boxes
of a replica run share no data, so no collective touches the data path),
whole-job throughput = cells of all ranks over the slowest rank's time.
Only the two scalar reductions below cross ranks."""
from __future__ import annotations


def job_throughput(ms_local, cells_local, device="cpu"):
    """(cell-updates/s of the whole job, the slowest rank's ms) over the ranks
    of the default process group; a single process returns its own."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return cells_local / (ms_local * 1e-3), ms_local
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return c.item() / (t.item() * 1e-3), t.item()

