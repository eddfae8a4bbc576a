"""Sharding of independent (composition, T, P) rows over ranks (one process per GPU).

The rows of an opacity / ODF table are independent units (the paper splits its ODF
table over temperatures among MPI workers, Sect. 4.6); ranks take disjoint rows and
never exchange data.  The only collectives are for measurement: a barrier and the
max / sum of per-rank timings and counts.
"""
from __future__ import annotations

import numpy as np


def rows_for_rank(n_rows: int, rank: int, world: int, order=None) -> np.ndarray:
    """Disjoint, near-equal share of rows 0..n_rows-1 for `rank` (round-robin over `order`,
    by default the natural order), so that ranks get similar mixes of cheap and costly rows."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    idx = np.arange(n_rows) if order is None else np.asarray(order)
    return idx[rank::world].astype(np.int32)


def reduce_scalar(x: float, op: str = "max") -> float:
    """Max or sum of a per-rank scalar over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
