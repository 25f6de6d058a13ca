"""The C-ABI's contracts on the GPU: caller-owned workspace (no device allocation after
lnocc_build_ints), and the bounded device wait that turns a wait that never ends into LNOCC_ETIMEOUT
with the CUDA context still usable."""
import numpy as np
import pytest

from paper_2407_11258_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lnocc():
    from paper_2407_11258_gb300 import build
    from paper_2407_11258_gb300 import lnocc as m
    build.build()
    m.load()
    return m


def test_bounded_wait_runs_out_and_the_context_survives(lnocc):
    """An mbarrier that nothing arrives on: the wait gives up after its budget (here 50 ms) and the call
    reports LNOCC_ETIMEOUT; the next kernels run normally."""
    code, waited = lnocc.lnocc_debug_wait(False, 50_000_000)
    assert code == lnocc.LNOCC_ETIMEOUT
    assert 50_000_000 <= waited < 1_000_000_000, waited
    code, waited = lnocc.lnocc_debug_wait(True, 50_000_000)  # arrived first: no wait at all
    assert code == lnocc.LNOCC_OK and waited < 10_000_000
    A = torch.randn(70, 90, dtype=torch.float64, device="cuda")
    C = torch.zeros(70, 70, dtype=torch.float64, device="cuda")
    lnocc.lnocc_debug_gemm(1, A, A, C)
    assert torch.allclose(C, A @ A.T, rtol=0, atol=1e-4 * float((A.abs() @ A.abs().T).max()))


def test_bounded_wait_rejects_out_of_range_budget(lnocc):
    with pytest.raises(lnocc.LnoccError) as ei:
        lnocc.lnocc_debug_wait(False, 3_000_000_000)
    assert ei.value.code == lnocc.LNOCC_EINVAL


def _solve(lnocc, fr, prec, ws=None, **opt):
    eps = torch.tensor(fr.eps, device="cuda")
    B = torch.tensor(fr.B, device="cuda")
    U = torch.tensor(fr.U_frag, device="cuda")
    opts = lnocc.default_opts(precision=prec, **opt)
    f = lnocc.lnocc_build_ints(fr.nocc, fr.nvir, fr.naux, eps, B, opts)
    try:
        if ws is not None:
            lnocc.lnocc_frag_set_workspace(f, ws)
        torch.cuda.synchronize()
        a0 = f.info().device_allocs
        e, it, _ = lnocc.lnocc_ccsd(f)
        ec, em = lnocc.lnocc_fragment_energy(f, U)
        et, etf = lnocc.lnocc_triples(f, U)
        a1 = f.info().device_allocs
    finally:
        f.free()
    return dict(e_ccsd=e, e_ccsd_frag=ec, e_mp2_frag=em, e_t=et, e_t_frag=etf), a1 - a0


@pytest.mark.parametrize("shape", [(4, 24, 96), (9, 70, 280)])
@pytest.mark.parametrize("prec", [0, 1])
def test_attached_workspace_means_no_allocation_after_build(lnocc, shape, prec):
    o, v, q = shape
    fr = synth.make_fragment(o, v, q, 900 + o, decay=20.0, frag=(0, 1))
    ref, allocs_ref = _solve(lnocc, fr, prec)
    assert allocs_ref > 0  # without a workspace lnocc_triples allocates its temporaries
    nb = lnocc.lnocc_workspace_bytes(o, v, q, lnocc.default_opts(precision=prec))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    got, allocs = _solve(lnocc, fr, prec, ws=ws)
    assert allocs == 0
    assert got == ref  # same kernels, same order: the same bits


def test_workspace_size_follows_the_chunk_option_and_is_checked(lnocc):
    o, v, q = 8, 60, 240  # largest (T) slab ~1.9 MB of FP32 W: a 1 MB chunk bound takes effect
    fr = synth.make_fragment(o, v, q, 950, decay=20.0, frag=(0,))
    big = lnocc.lnocc_workspace_bytes(o, v, q, lnocc.default_opts(precision=1))
    small = lnocc.lnocc_workspace_bytes(o, v, q, lnocc.default_opts(precision=1, triples_chunk_mb=1))
    assert small < big
    ref, _ = _solve(lnocc, fr, 1)
    got, allocs = _solve(lnocc, fr, 1, ws=torch.empty(small, dtype=torch.uint8, device="cuda"), triples_chunk_mb=1)
    assert allocs == 0
    for k in ref:
        assert abs(got[k] - ref[k]) < 1e-12, k
    f = lnocc.lnocc_build_ints(o, v, q, torch.tensor(fr.eps, device="cuda"), torch.tensor(fr.B, device="cuda"),
                               lnocc.default_opts(precision=1))
    try:
        with pytest.raises(lnocc.LnoccError) as ei:
            lnocc.lnocc_frag_set_workspace(f, torch.empty(big - 256, dtype=torch.uint8, device="cuda"))
        assert ei.value.code == lnocc.LNOCC_EINVAL
    finally:
        f.free()
    assert np.isfinite(got["e_t"])


@pytest.mark.parametrize("shape", [(16, 40, 160), (5, 37, 150)])
def test_device_outputs_capture_into_a_cuda_graph(lnocc, shape):
    """lnocc_fragment_energy_device and lnocc_triples_device enqueue without synchronising and write
    device memory: captured into a CUDA graph and replayed they give the synchronous calls' energies
    bit for bit. nocc=16 runs the grouped (T) launches, nocc=5 the per-term ones with device-built
    launch tables."""
    o, v, q = shape
    fr = synth.make_fragment(o, v, q, 1700 + o, decay=20.0, frag=(0, 1))
    eps, B, U = (torch.tensor(x, device="cuda") for x in (fr.eps, fr.B, fr.U_frag))
    opts = lnocc.default_opts(precision=1)
    f = lnocc.lnocc_build_ints(o, v, q, eps, B, opts)
    try:
        lnocc.lnocc_ccsd(f)
        ec, em = lnocc.lnocc_fragment_energy(f, U)
        et, etf = lnocc.lnocc_triples(f, U)
        ws = torch.empty(lnocc.lnocc_workspace_bytes(o, v, q, opts), dtype=torch.uint8, device="cuda")
        lnocc.lnocc_frag_set_workspace(f, ws)
        e1 = torch.zeros(2, dtype=torch.float64, device="cuda")
        e2 = torch.zeros(2, dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        lnocc.lnocc_fragment_energy_device(f, U, e1, stream=s)  # eager enqueue
        lnocc.lnocc_triples_device(f, U, e2, st, stream=s)
        s.synchronize()
        assert e1.tolist() == [ec, em] and e2.tolist() == [et, etf] and int(st.item()) == 0
        e1.zero_()
        e2.zero_()
        st.fill_(-1)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            lnocc.lnocc_fragment_energy_device(f, U, e1, stream=s)
            lnocc.lnocc_triples_device(f, U, e2, st, stream=s)
        assert e2.tolist() == [0.0, 0.0]  # capture records the work, nothing has run yet
        for _ in range(2):
            g.replay()
            torch.cuda.synchronize()
            assert e1.tolist() == [ec, em] and e2.tolist() == [et, etf] and int(st.item()) == 0
        with pytest.raises(lnocc.LnoccError) as ei:  # a workspace is required
            lnocc.lnocc_frag_set_workspace(f, None)
            lnocc.lnocc_triples_device(f, U, e2, st, stream=s)
        assert ei.value.code == lnocc.LNOCC_EINVAL
    finally:
        torch.cuda.synchronize()
        f.free()
