"""Batched uneven fragments (lnocc_solve_batch) and the graph-replayed CCSD iteration, on the GPU.

Parity: every fragment of the shrunk uneven batch matches the FP64 oracle's stored energies within
1e-6 Eh (tests/golden/oracle_small.json, written from `oracle/` only), and equals the single-fragment
C-ABI calls bit for bit (the batch runs the same kernels; only the schedule differs).
"""
import json
import os

import numpy as np
import pytest

from paper_2407_11258_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-6
KEYS = ("e_mp2", "e_ccsd", "e_mp2_frag", "e_ccsd_frag", "e_t", "e_t_frag")


@pytest.fixture(scope="module")
def lnocc():
    from paper_2407_11258_gb300 import build
    from paper_2407_11258_gb300 import lnocc as m
    build.build()
    m.load()
    return m


def shrunk_batch():
    ref = json.load(open(os.path.join(HERE, "golden", "oracle_small.json")))["batch_shrunk"]
    shrink = lambda o, v: (max(2, o // 3), max(8, v // 10))  # noqa: E731
    frs = [synth.batch_fragment(f, scale_shape=shrink) for f in range(len(ref))]
    return frs, ref


def on_device(fr):
    return (fr.nocc, fr.nvir, fr.naux, torch.tensor(fr.eps, device="cuda"), torch.tensor(fr.B, device="cuda"),
            torch.tensor(fr.U_frag, device="cuda"))


def single(lnocc, item, **opt):
    o, v, q, eps, B, U = item
    f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(**opt))
    try:
        e, it, _ = lnocc.lnocc_ccsd(f)
        ec, em = lnocc.lnocc_fragment_energy(f, U)
        et, etf = lnocc.lnocc_triples(f, U)
        return dict(e_mp2=f.info().e_mp2, e_ccsd=e, e_ccsd_frag=ec, e_mp2_frag=em, e_t=et, e_t_frag=etf, n_iter=it)
    finally:
        f.free()


def as_dict(r):
    return {k: getattr(r, k) for k in KEYS} | {"n_iter": r.n_iter}


def test_batch_matches_oracle_and_single_calls(lnocc):
    frs, ref = shrunk_batch()
    items = [on_device(fr) for fr in frs]
    opts = lnocc.default_opts(precision=1, max_iter=300)
    st, res = lnocc.lnocc_solve_batch(items, opts, lnocc.default_batch_opts(workers=3))
    assert st == lnocc.LNOCC_OK
    for k, (r, want) in enumerate(zip(res, ref)):
        assert r.status == lnocc.LNOCC_OK
        bad = {key: getattr(r, key) - want[key] for key in KEYS if not abs(getattr(r, key) - want[key]) <= TOL}
        assert not bad, f"fragment {k}: {bad}"
    # the schedule changes nothing: same numbers as the one-fragment calls
    for k in (0, 5, len(items) - 1):
        assert as_dict(res[k]) == single(lnocc, items[k], precision=1, max_iter=300), k
    # every fragment ran once, on a valid pipeline, in a complete start order
    assert sorted(r.order for r in res) == list(range(len(res)))
    assert all(0 <= r.worker < 3 and r.t_end_ms >= r.t_start_ms for r in res)


def test_lpt_order_and_memory_budget(lnocc):
    frs, _ = shrunk_batch()
    items = [on_device(fr) for fr in frs[:6]]
    opts = lnocc.default_opts(precision=1, max_iter=300)
    # one pipeline, LPT: fragments start in decreasing order of the cost model
    st, res = lnocc.lnocc_solve_batch(items, opts, lnocc.default_batch_opts(workers=1, triples=0))
    assert st == lnocc.LNOCC_OK
    started = sorted(res, key=lambda r: r.order)
    costs = [r.cost_estimate for r in started]
    assert costs == sorted(costs, reverse=True) and costs[0] > costs[-1] > 0
    # the memory estimate bounds what the handle really held
    assert all(r.bytes_estimate >= r.device_bytes > 0 for r in res)
    # input order
    st, res_in = lnocc.lnocc_solve_batch(items, opts, lnocc.default_batch_opts(workers=1, triples=0, order=1))
    assert [r.order for r in res_in] == list(range(len(items)))
    assert [as_dict(a) for a in res] == [as_dict(b) for b in res_in]
    # a budget below any fragment's footprint: fragments run one at a time even with 4 pipelines
    st, res_b = lnocc.lnocc_solve_batch(items, opts, lnocc.default_batch_opts(workers=4, triples=0, mem_budget_gb=1e-6))
    spans = sorted((r.t_start_ms, r.t_end_ms) for r in res_b)
    assert all(spans[k][1] <= spans[k + 1][0] for k in range(len(spans) - 1))
    assert [as_dict(a) for a in res] == [as_dict(b) for b in res_b]


def test_batch_reports_nonconvergence_per_fragment(lnocc):
    frs, _ = shrunk_batch()
    items = [on_device(fr) for fr in frs[:3]]
    st, res = lnocc.lnocc_solve_batch(items, lnocc.default_opts(precision=1, max_iter=2),
                                      lnocc.default_batch_opts(workers=2, triples=0), allow_noconv=True)
    assert st == lnocc.LNOCC_ENOCONV
    assert all(r.status == lnocc.LNOCC_ENOCONV and r.n_iter == 2 and np.isfinite(r.e_ccsd) for r in res)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_eager(lnocc, prec):
    """CCSD iterations replayed from the captured graph give the eager launches' numbers bit for bit,
    on the default stream and on a side stream."""
    fr = synth.make_fragment(5, 40, 160, 9, decay=20.0, frag=(0, 1))
    item = on_device(fr)
    eager = single(lnocc, item, precision=prec, graph=0)
    graph = single(lnocc, item, precision=prec, graph=1)
    assert eager["n_iter"] >= 3 and eager == graph
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        graph_side = single(lnocc, item, precision=prec, graph=1)
    torch.cuda.synchronize()
    assert graph_side == eager


def test_full_size_batch_fragment_matches_single_call(lnocc):
    """A full-size fragment of the uneven batch (largest nvir among the first 8) through the batch
    runtime with a second fragment alongside: same energies as the single-fragment calls."""
    shapes = synth.batch_shapes()
    k = max(range(8), key=lambda f: shapes[f][1])
    items = [synth.batch_fragment_device(f, "cuda") for f in (k, 1)]
    opts = lnocc.default_opts(precision=1)
    st, res = lnocc.lnocc_solve_batch(items, opts, lnocc.default_batch_opts(workers=2), allow_noconv=True)
    ref = single(lnocc, items[0], precision=1)
    assert as_dict(res[0]) == ref
    assert res[0].status == lnocc.LNOCC_OK


def test_full_size_small_gap_fragment_mixed_matches_fp64(lnocc):
    """Fragment 1 of the uneven batch at full size (nocc=14, nvir=130, naux=520, lithium-like gap 0.054 Eh):
    where the mixed path's residual noise floor and the slow small-gap convergence meet, every mixed
    energy stays within 1e-6 Eh of the plain FP64 GPU path on the same inputs (B drawn on the device as
    for the batch)."""
    item = synth.batch_fragment_device(1, "cuda")
    assert item[:3] == (14, 130, 520)
    mixed = single(lnocc, item, precision=1, max_iter=300)
    fp64 = single(lnocc, item, precision=0, max_iter=300)
    bad = {k: mixed[k] - fp64[k] for k in KEYS if not abs(mixed[k] - fp64[k]) <= TOL}
    assert not bad, bad
