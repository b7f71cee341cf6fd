"""Ensembles of independent lattices across ranks (one process per GPU).

Every rank advances its own lattices -- the same configurations with its own seeds -- with no
communication on the data path (weak scaling).  The only cross-rank operation is the final
combination of ensemble averages on the host (``ensemble_mean``), over torch.distributed.
"""
from __future__ import annotations

import numpy as np


def seeds_for_rank(rank: int, n_per_rank: int, seed0: int = 1000):
    """Seeds of one rank: a block of n_per_rank consecutive seeds, disjoint across ranks."""
    return range(seed0 + rank * n_per_rank, seed0 + (rank + 1) * n_per_rank)


def ensemble_mean(local_sum, local_count: int, group=None):
    """Mean over all ranks of per-sample values: local_sum is this rank's sum over its samples
    (any shape), local_count their number.  Returns the global mean on every rank."""
    import torch
    import torch.distributed as dist

    s = torch.as_tensor(np.asarray(local_sum, dtype=np.float64)).reshape(-1).clone()
    n = torch.tensor([float(local_count)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(n, op=dist.ReduceOp.SUM, group=group)
    return (s / n).numpy().reshape(np.shape(local_sum))
