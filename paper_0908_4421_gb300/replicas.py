"""Replica runs across GPUs: one process per GPU, each solving its own plan.

Plans are independent problems, so a multi-GPU run shares no data: the only
collectives are a barrier around the timed region and a max-reduction of the
per-rank timings (the job is as slow as its slowest replica). Rendezvous comes
from the torchrun environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR/PORT).
"""
from __future__ import annotations

import os
from typing import Optional, Tuple


def env() -> Tuple[int, int, int]:
    """(rank, world_size, local_rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Group:
    """The process group of a replica run, or a no-op stand-in for a single process."""

    def __init__(self, backend: Optional[str] = None):
        self.rank, self.world, self.local_rank = env()
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.dist = dist
            self.backend = backend

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, value: float) -> float:
        """Largest value over all ranks (every rank receives it)."""
        if self.dist is None:
            return float(value)
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, value: float) -> float:
        if self.dist is None:
            return float(value)
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self) -> None:
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None
