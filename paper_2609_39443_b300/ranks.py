"""Multi-GPU layout of the benchmark: one process per GPU, each advancing its
own independent instances (the configured workloads are independent
simulations), with no collective on the data path.  The only collectives are
a barrier around the timed region and a MAX over ranks of the timings
(weak scaling: per-rank work is fixed as the rank count grows)."""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def rank_env() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_seed(rank: int, base: int = 0) -> int:
    """Seed of a rank's own synthetic instance(s)."""
    return base + rank


def max_over_ranks(values: Sequence[float], dist=None, device="cpu") -> List[float]:
    """Element-wise MAX of per-rank timings (no-op without a process group)."""
    vals = [float(v) for v in values]
    if dist is None:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]
