"""Multi-GPU replicas: one process per GPU, each tracing its own sessions (no data exchange).

The hot path shards into independent units -- every client session (server depth image + its
frames) is traced by one GPU on its own splats and LBVH -- so the multi-GPU layout is replicas
with weak scaling: no collective on the data path.  The only cross-rank operations are the
benchmark's barrier around the timed region and the max-over-ranks of its time.  Launch with
``torchrun`` (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_ADDR / MASTER_PORT from the environment);
any torch.distributed backend works (NCCL on GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import datetime
import os
from dataclasses import dataclass
from typing import Optional

import torch


@dataclass
class Replicas:
    rank: int = 0
    world: int = 1
    local_rank: int = 0
    backend: Optional[str] = None   # None: single process, no process group

    @staticmethod
    def from_env(backend: str = "nccl", timeout_s: float = 600.0) -> "Replicas":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        r = Replicas(rank, world, local, None)
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
            r.backend = backend
        return r

    def _device(self):
        return torch.device("cuda") if self.backend == "nccl" else torch.device("cpu")

    def barrier(self) -> None:
        if self.backend is not None:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        """The largest value of x over all ranks (the slowest rank's time)."""
        if self.backend is None:
            return float(x)
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self._device())
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job_rate(self, units_per_rank: float, seconds_max: float) -> float:
        """Units processed by all ranks per second of the slowest rank (weak scaling)."""
        return self.world * units_per_rank / seconds_max

    def pose_seed_offset(self) -> int:
        """Each rank draws its own client poses and sessions."""
        return 97 * self.rank

    def close(self) -> None:
        if self.backend is not None:
            import torch.distributed as dist
            dist.destroy_process_group()
            self.backend = None
