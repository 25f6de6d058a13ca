"""Host-side sharding of independent fragments over ranks (no collective in the data path).

Fragments are independent units (Sec. II.B: E_c = sum_F E^(F), Eq. 7 and Eq. 14), so a multi-GPU run
assigns whole fragments to ranks by longest-processing-time first on a flop cost model, and only the
per-fragment energies are gathered at the end and summed in fragment order (deterministic regardless
of the rank count).

The cost model is the one the batch runtime uses to order fragments on one GPU (lnocc_solve_batch):
CCSD iterations estimated from the HOMO-LUMO gap, min(60, 10 + 1.6 / sqrt(gap)), times the per-iteration
work 2o^2v^4 + 16o^3v^3 + 2o^4v^2, plus (T) 6o^3v^4 + 6o^4v^3 and the integral assembly 2N(o+v)v^3.
"""
from __future__ import annotations

import heapq
import math


def iteration_estimate(gap: float) -> float:
    """CCSD iterations expected for a HOMO-LUMO gap (Eh): small gaps converge more slowly."""
    if not gap > 0:
        return 40.0
    return min(60.0, 10.0 + 1.6 / math.sqrt(gap))


def fragment_cost(nocc: int, nvir: int, naux: int = 0, gap: float = 0.7, triples: bool = True) -> float:
    """Model flops of one fragment solve (see the module docstring)."""
    o, v, N = float(nocc), float(nvir), float(naux)
    it = iteration_estimate(gap) * (2 * o**2 * v**4 + 16 * o**3 * v**3 + 2 * o**4 * v**2)
    t = 6 * o**3 * v**4 + 6 * o**4 * v**3 if triples else 0.0
    return it + t + 2 * N * (o + v) * v**3


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


def assign(shapes, world: int):
    """shapes: one (nocc, nvir, naux, gap) per fragment. Returns the LPT list of fragment indices of
    every rank (the same on every rank: the assignment is a pure function of the shapes)."""
    costs = [fragment_cost(o, v, q, g) for (o, v, q, g) in shapes]
    return lpt_assign(costs, world)


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
