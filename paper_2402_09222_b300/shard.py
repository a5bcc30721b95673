"""Splitting one problem's histories over ranks (one GPU per rank).

Histories are independent and every random number is keyed by (seed,
problem, history), so a contiguous split of the history range changes no
history: rank r runs `history_range(r, world, n)` with mcx_run_batch's
`first_history`, and the per-batch tallies of all ranks add up to the
single-GPU tallies (to FP64 summation order).  The only exchange is one sum
of the tallies at the end (`reduce_tallies`); nothing is exchanged while
particles are in flight.  Lookup batches need no exchange at all.
"""
from __future__ import annotations

import numpy as np


def history_range(rank: int, world: int, n_histories: int) -> tuple[int, int]:
    """Contiguous [first, last) of rank `rank`; sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError("rank outside the world")
    base, extra = divmod(n_histories, world)
    first = rank * base + min(rank, extra)
    return first, first + base + (1 if rank < extra else 0)


def reduce_tallies(tallies: dict, group=None) -> dict:
    """Sum every array of `tallies` over the ranks (in place semantics are not
    assumed: a new dict of numpy arrays is returned).  Uses the default process
    group's backend (NCCL between GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    out = {}
    for k in sorted(tallies):
        v = tallies[k]
        if not isinstance(v, np.ndarray) or v.dtype.kind not in "fiu":
            out[k] = v
            continue
        t = torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out[k] = t.cpu().numpy()
    return out


def max_over_ranks(x: float, group=None) -> float:
    """The largest value of `x` over the ranks (timings: the slowest rank)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
