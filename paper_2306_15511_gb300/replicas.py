"""Replica coordination for running independent constrained-realization
chains on several GPUs (one process per GPU).

The sampler's hot path has no exchange step: every rank solves its own
realizations with its own white noise (Eq. mapmakingeq for independent
(w1, w2) draws), so the only cross-rank traffic is timing and counting for
the whole-job throughput: a barrier around the timed region, the maximum of
the ranks' elapsed times and the sum of their iteration counts.

Ranks are read from the torchrun environment (RANK, WORLD_SIZE, LOCAL_RANK,
MASTER_ADDR / MASTER_PORT); NCCL on GPUs, gloo for CPU tests.
"""
from __future__ import annotations

import os

# Philox keys of the white noise (w1 in harmonic space, w2 in pixel space)
# for realization b of rank r: ranks > 0 draw fresh keys for both, so that
# replicas are independent chains; rank 0 keeps the recipe's own keys.
_W1_KEY_BASE = 40000
_W2_KEY_BASE = 50000


def w1_key(rank: int, b: int) -> int | None:
    """Philox key for realization b's harmonic white noise on a rank (None:
    the recipe's default key)."""
    if rank == 0:
        return None
    return _W1_KEY_BASE + 100 * rank + b


def w2_key(rank: int, b: int) -> int | None:
    """Philox key for realization b's pixel white noise on a rank (None: the
    recipe's default key)."""
    if rank == 0:
        return None
    return _W2_KEY_BASE + 100 * rank + b


def free_port() -> int:
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_entry(rank, world, port, fn, args):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    rc = fn(*args)
    if rc:
        raise SystemExit(rc)


def launch_local(nprocs: int, fn, args=()) -> None:
    """Run fn(*args) in nprocs spawned processes, one per local GPU, with the
    torchrun environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR =
    127.0.0.1, MASTER_PORT) set in each; returns when all have exited and
    raises if one failed.  fn must be importable (a module-level function)."""
    import torch.multiprocessing as mp
    mp.start_processes(_rank_entry, args=(nprocs, free_port(), fn, tuple(args)), nprocs=nprocs,
                       join=True, start_method="spawn")


class Replicas:
    """Rank bookkeeping and the three reductions the benchmark needs."""

    def __init__(self, backend: str = "nccl", device=None):
        import torch
        import torch.distributed as dist
        self._dist = dist
        self._torch = torch
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device if device is not None else torch.device("cpu")
        self._own = False
        if self.world > 1 and not dist.is_initialized():
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=self.device)
            else:
                dist.init_process_group(backend)
            self._own = True

    def barrier(self) -> None:
        if self.world > 1:
            self._dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if self.world == 1:
            return float(x)
        t = self._torch.tensor([float(x)], dtype=self._torch.float64, device=self.device)
        self._dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        """Maximum over ranks (the whole job's elapsed time)."""
        return self._reduce(x, self._dist.ReduceOp.MAX)

    def sum(self, x: float) -> float:
        """Sum over ranks (the whole job's work)."""
        return self._reduce(x, self._dist.ReduceOp.SUM)

    def throughput(self, units: float, seconds: float) -> float:
        """Whole-job rate: units summed over ranks / the slowest rank's time."""
        return self.sum(units) / self.max(seconds)

    def close(self) -> None:
        if self._own and self._dist.is_initialized():
            self._dist.destroy_process_group()
            self._own = False
