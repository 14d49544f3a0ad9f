"""Independent networks spread over ranks (one process per GPU).

Each network's Kirchhoff system (Eq. 3) is solved on its own, so a set of
networks shards over GPUs with no exchange on the data path: every rank solves
the networks assigned to it with its own GPU, and the host gathers the results.
The only collectives are host-side bookkeeping: the gather of per-network
results for the caller and the max-over-ranks time of a timed region.

Assignment is longest-processing-time first on an estimate of each network's
work: Jacobi-preconditioned CG on a lattice of side L needs a number of
iterations that grows like L (the condition number grows like L^2), each over
U unknowns, so the work is taken as U * L.  The assignment depends only on the
shapes, so every rank computes the same one without communicating.
"""
from __future__ import annotations

import heapq
from typing import Callable, Sequence

import numpy as np


def work_estimate(dims) -> float:
    """Relative cost of one network's solve: unknowns x lattice side."""
    dims = [int(v) for v in dims]
    return float(np.prod(dims)) * float(max(dims))


def lpt_assign(works: Sequence[float], world: int) -> list[list[int]]:
    """Indices of ``works`` per rank, longest first onto the least-loaded rank
    (ties: lower index first, lower rank first).  Each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(works)), key=lambda i: (-float(works[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(works[i]), r))
    return [sorted(v) for v in out]


def my_share(dims_list: Sequence, rank: int, world: int) -> list[int]:
    """The indices this rank solves."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} not in [0, {world})")
    return lpt_assign([work_estimate(d) for d in dims_list], world)[rank]


def _dist():
    import torch.distributed as dist

    return dist if dist.is_available() and dist.is_initialized() else None


def gather_results(local: dict, count: int, group=None) -> list:
    """All ranks' ``{index: result}`` merged into one list in index order (on
    every rank).  Raises if an index is missing or claimed twice."""
    dist = _dist()
    parts = [local]
    if dist is not None and dist.get_world_size(group) > 1:
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, local, group=group)
    out = [None] * count
    seen = [False] * count
    for part in parts:
        for i, v in part.items():
            if seen[i]:
                raise RuntimeError(f"network {i} solved on two ranks")
            seen[i] = True
            out[i] = v
    missing = [i for i in range(count) if not seen[i]]
    if missing:
        raise RuntimeError(f"networks {missing[:8]} solved on no rank")
    return out


def max_over_ranks(x: float, group=None, device=None) -> float:
    """Largest value of ``x`` over the ranks (``x`` itself without a process
    group).  ``device`` is where the reduction tensor lives (a CUDA device for
    NCCL, the CPU for gloo)."""
    dist = _dist()
    if dist is None or dist.get_world_size(group) == 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def run_sharded(specs: Sequence, solve_fn: Callable[[list], list], rank: int, world: int,
                group=None) -> list:
    """Solve ``specs`` (a list of ``(dims, planes)``) over ``world`` ranks:
    this rank calls ``solve_fn`` on its share (a list of specs, returning one
    result per spec) and every rank gets all results in the order of
    ``specs``."""
    mine = my_share([d for d, _ in specs], rank, world)
    res = solve_fn([specs[i] for i in mine]) if mine else []
    if len(res) != len(mine):
        raise RuntimeError("solve_fn returned a wrong number of results")
    return gather_results(dict(zip(mine, res)), len(specs), group)
