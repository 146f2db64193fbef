"""Host-side logic of the one-process-per-GPU runs.

The limited-convection step has no exchange between independent problems, so
N > 1 GPUs run replicas (one mesh per rank) or split a batch of boxes across
ranks; no collective sits on the data path.  The only collectives are the
timing reduction (max over ranks) and, for diagnostics, a sum.

* ``lpt_partition`` splits boxes by cell count with the longest-processing-
  time rule (largest first onto the least-loaded rank), which keeps the
  heaviest rank within 4/3 of the optimum (Graham's bound).
* ``max_over_ranks`` / ``sum_over_ranks`` reduce one float over the process
  group (any backend: NCCL on GPUs, gloo on the host).
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def lpt_partition(weights: Sequence[int], n_parts: int) -> List[List[int]]:
    """Indices of ``weights`` split into ``n_parts`` lists, largest first onto
    the least-loaded part (ties: lower index first, lower part first).  Each
    list is returned in increasing index order."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-int(weights[i]), i))
    heap = [(0, p) for p in range(n_parts)]
    parts: List[List[int]] = [[] for _ in range(n_parts)]
    for i in order:
        load, p = heapq.heappop(heap)
        parts[p].append(i)
        heapq.heappush(heap, (load + int(weights[i]), p))
    return [sorted(p) for p in parts]


def part_loads(weights: Sequence[int], parts: List[List[int]]) -> List[int]:
    return [sum(int(weights[i]) for i in p) for p in parts]


def _reduce(value: float, op_name: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of ``value`` over the default process group (the value itself
    when no group is initialised)."""
    return _reduce(value, "MAX", device)


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of ``value`` over the default process group."""
    return _reduce(value, "SUM", device)


def whole_job_rate(local_units: float, local_ms: float, device=None) -> tuple:
    """(units of all ranks / max-over-ranks time in s, that time in ms)."""
    ms = max_over_ranks(local_ms, device)
    units = sum_over_ranks(local_units, device)
    return units / (ms * 1e-3), ms
