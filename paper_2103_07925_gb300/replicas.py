"""Replica runs on several GPUs of one node: one process per GPU, each advancing its own
scene (or batch of scenes), with no collective on the data path.  The only communication
is around the timed region: a barrier on both sides, the maximum time over ranks, and the
sum of the units every rank processed (whole-job throughput = total units / slowest rank).
"""
from __future__ import annotations

import os


class Replicas:
    """Timing reductions over the ranks of a process group (any backend), or a single
    process when ``dist`` is None."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device
        self.rank = dist.get_rank() if dist is not None else 0
        self.world = dist.get_world_size() if dist is not None else 1

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)

    def throughput(self, units, seconds):
        """Whole-job rate: units summed over ranks over the slowest rank's time."""
        return self.sum(units) / self.max(seconds)


def from_env(backend="nccl"):
    """Join the process group that torch.distributed.run set up (WORLD_SIZE > 1), else a
    single process.  Returns (Replicas, local rank)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world <= 1:
        return Replicas(None), local
    import torch.distributed as dist
    dist.init_process_group(backend)
    return Replicas(dist, device="cuda" if backend == "nccl" else "cpu"), local
