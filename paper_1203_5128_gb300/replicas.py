"""Independent replicas, one process per GPU.

The filter's work per image has no exchange step (each image, or band of an
image with a read-only halo, is filtered on its own), so N GPUs run N
replicas with no collective on the data path.  What the job needs across
processes is host-side: the process group from the launcher's environment
(RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR / MASTER_PORT), a barrier around
timed regions, and the maximum over ranks of a host number (a job takes as
long as its slowest rank).
"""
from __future__ import annotations

import os


class Replicas:
    """Process-group helper; with WORLD_SIZE 1 every call is local."""

    def __init__(self, backend: str = "nccl", device=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if backend == "nccl" and device is not None else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    @property
    def root(self) -> bool:
        return self.rank == 0

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        """Maximum of a host float over all ranks (x itself with one rank)."""
        if self.dist is None:
            return float(x)
        import torch
        dev = self.device if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None
