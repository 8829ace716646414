"""Replica runs on several GPUs of one node (one process per GPU).

The benchmark workloads are independent problems (a box, or an ensemble of
boxes), so N GPUs run N replicas with no collective in the data path (weak
scaling).  The only communication is host-level bookkeeping: barriers around
the timed region and the maximum of the per-rank times, from which the
whole-job rate is the units all ranks processed divided by that maximum.
Ranks, world size and the local device come from the launcher's environment
(RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR/PORT).
"""
from __future__ import annotations

import os
from typing import Optional


class Replicas:
    """Process-group bookkeeping of a replica run; a single process needs none."""

    def __init__(self, backend: Optional[str] = None, timeout_s: Optional[float] = None):
        """timeout_s: limit of every collective of the group (barriers, the
        timing reduction), so that the ranks left behind by a rank that failed
        get an error at their next collective instead of waiting for ever."""
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", str(self.rank)))
        self.backend = backend or "nccl"
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            kw = {}
            if timeout_s is not None:
                import datetime

                kw["timeout"] = datetime.timedelta(seconds=float(timeout_s))
            if self.backend == "nccl":
                torch.cuda.set_device(self.local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local), **kw)
            else:
                dist.init_process_group(self.backend, **kw)
            self.dist = dist

    @property
    def root(self) -> bool:
        return self.rank == 0

    def seed(self, b: int = 0, nboxes: int = 1) -> int:
        """Seed of box b of this rank's replica: distinct over all ranks and boxes."""
        return self.rank * nboxes + b

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch

        dev = torch.device("cuda", torch.cuda.current_device()) if self.backend == "nccl" else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job_rate(self, units_per_rank: float, seconds_max: float) -> float:
        """Units processed by all ranks per second of the slowest rank."""
        return units_per_rank * self.world / seconds_max

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None
