"""Host-side sharding of independent fragments over ranks (no collective in the data path).

Fragments are independent units (Sec. II.B: E_c = sum_F E^(F), Eq. 7 and Eq. 14), so a multi-GPU run
assigns whole fragments to ranks and only the per-fragment energies are gathered at the end and
summed in fragment order (deterministic regardless of the rank count).
"""
from __future__ import annotations

import heapq


def fragment_cost(nocc: int, nvir: int) -> float:
    """Model flops of one fragment solve: 10 CCSD iterations of 2o^2v^4 + 16o^3v^3 + 2o^4v^2, plus (T)."""
    o, v = float(nocc), float(nvir)
    return 10 * (2 * o**2 * v**4 + 16 * o**3 * v**3 + 2 * o**4 * v**2) + 6 * o**3 * v**4 + 6 * o**4 * v**3


def lpt_assign(costs, world: int):
    """Longest-processing-time-first assignment: returns one list of fragment indices per rank."""
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for f in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(f)
        heapq.heappush(heap, (load + costs[f], r))
    for lst in out:
        lst.sort()
    return out


def gather_energies(local: dict, world: int):
    """All ranks contribute {fragment: energy}; returns the dict of all fragments (every rank)."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local)
    merged = {}
    for p in parts:
        merged.update(p)
    return merged


def ordered_sum(energies: dict) -> float:
    """Sum in fragment order (the same bits for any sharding)."""
    tot = 0.0
    for f in sorted(energies):
        tot += energies[f]
    return tot
