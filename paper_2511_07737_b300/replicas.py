"""Host side of the multi-GPU run: independent replicas, one process per GPU.

The solver's step has no cross-GPU exchange: each rank solves its own
instance (a different seed), so the only collectives are the timing barrier
and the max / sum of per-rank scalars for the whole-job figure.  The backend
is NCCL on GPUs and gloo in the CPU tests; rendezvous comes from the usual
torchrun environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR, MASTER_PORT).
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s instance: distinct per rank (weak scaling)."""
    return base_seed + 1000 * rank


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, ms: float) -> float:
    """Units of all ranks per second over the slowest rank's time (max over ranks)."""
    return units_per_rank_step * steps * world / (ms / 1e3)


class Replicas:
    """Barrier and scalar reductions across the ranks (no-ops for one process)."""

    def __init__(self, world: int, backend: str = "nccl", device=None):
        self.world = world
        self.dist = None
        self.device = device
        if world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                if backend == "nccl":
                    dist.init_process_group(backend, device_id=device)
                else:
                    dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x: float, op) -> float:
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return x if self.dist is None else self._reduce(x, self.dist.ReduceOp.MAX)

    def sum(self, x: float) -> float:
        return x if self.dist is None else self._reduce(x, self.dist.ReduceOp.SUM)

    def close(self):
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()
