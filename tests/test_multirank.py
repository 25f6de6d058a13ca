"""Sharding of independent fragments over ranks: world-size-2 gloo processes on the CPU.

Each rank takes its share of one fragment list from shard.assign (the LPT split that bench.py's batch
workload uses on the GPU path), solves it (here with the CPU oracle standing in for the GPU solver,
since this pool gives one GPU per box), and the energies gathered with shard.gather_energies and summed
with shard.ordered_sum (the same calls as on the GPU path) must be bit-identical to the single-rank sum.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2407_11258_gb300 import shard, synth  # noqa: E402

NFRAG = 6


def _fragment_energy(f):
    from oracle import ccsd as occ
    fr = synth.batch_fragment(f, scale_shape=lambda o, v: (max(2, o // 4), max(6, v // 20)))
    r = occ.ccsd(fr.eps, fr.B, fr.nocc)
    return r["e_corr"]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes = [(o, v, q, synth.batch_gap(f)) for f, (o, v, q, _) in enumerate(synth.batch_shapes()[:NFRAG])]
    mine = shard.assign(shapes, world)[rank]
    local = {f: _fragment_energy(f) for f in mine}
    allE = shard.gather_energies(local, world)
    if rank == 0:
        out.put((sorted(allE), shard.ordered_sum(allE)))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_cost_model_prefers_small_gaps_and_covers_the_list():
    """The cost grows as the gap closes (more CCSD iterations) and every fragment is assigned once."""
    assert shard.fragment_cost(16, 240, 960, 0.05) > shard.fragment_cost(16, 240, 960, 0.7)
    shapes = [(o, v, q, synth.batch_gap(f)) for f, (o, v, q, _) in enumerate(synth.batch_shapes())]
    parts = shard.assign(shapes, 4)
    assert sorted(sum(parts, [])) == list(range(128))
    costs = [shard.fragment_cost(*s) for s in shapes]
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)  # LPT bound


def test_lpt_assignment_balances_and_covers():
    costs = [5.0, 3.0, 3.0, 2.0, 2.0, 1.0]
    parts = shard.lpt_assign(costs, 2)
    assert sorted(sum(parts, [])) == list(range(6))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= 1.0


def test_two_ranks_match_one_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    frags, total2 = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert frags == list(range(NFRAG))
    total1 = shard.ordered_sum({f: _fragment_energy(f) for f in range(NFRAG)})
    assert total2 == total1
