"""Host logic of multi-GPU runs: one independent replica per rank.

Shots are independent problems, so the probed gradient shards over shots with
no data-path collective: every rank runs its own shots on its own GPU, and the
only communication is timing (a barrier around the timed region and the
maximum of the per-rank times).  The whole-job rate is then all ranks' work
over the slowest rank's time (weak scaling: fixed work per rank).

Rank, world size and local rank come from the torchrun environment
(RANK / WORLD_SIZE / LOCAL_RANK); the rendezvous address is MASTER_ADDR /
MASTER_PORT.  The backend is NCCL for GPU runs; the same code runs with gloo
on CPU tensors, which the tests use with two ranks.
"""
from __future__ import annotations

import os
from typing import Optional


class Replicas:
    def __init__(self, env: Optional[dict] = None):
        env = os.environ if env is None else env
        self.world = int(env.get("WORLD_SIZE", "1"))
        self.rank = int(env.get("RANK", "0"))
        self.local = int(env.get("LOCAL_RANK", "0"))
        if self.world < 1 or not 0 <= self.rank < self.world:
            raise ValueError(f"bad rank {self.rank} for world size {self.world}")
        self.device = None
        self._dist = None

    @property
    def printer(self) -> bool:
        """Rank 0 alone prints the result line."""
        return self.rank == 0

    def seed_offset(self) -> int:
        """Each rank draws its own shots (its own seeded workload)."""
        return self.rank

    def init(self, backend: str, device=None):
        """Joins the process group (world > 1).  `device` is where the timing
        reductions run: the rank's GPU for NCCL, the CPU for gloo."""
        import torch
        import torch.distributed as dist
        self.device = torch.device("cpu") if device is None else torch.device(device)
        if self.world > 1:
            kw = {"device_id": self.device} if backend == "nccl" else {}
            dist.init_process_group(backend, rank=self.rank, world_size=self.world, **kw)
            self._dist = dist
        return self

    def barrier(self):
        if self._dist is not None:
            self._dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        """The largest value of x over all ranks (the slowest rank's time)."""
        if self._dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], device=self.device, dtype=torch.float64)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job_rate(self, units_per_rank: float, ms_max: float) -> float:
        """All ranks' units per second, over the slowest rank's time."""
        return units_per_rank * self.world / (ms_max * 1e-3)

    def close(self):
        if self._dist is not None:
            self._dist.destroy_process_group()
            self._dist = None
