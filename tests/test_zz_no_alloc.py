"""lnocc_gemm_noalloc: the allocation-free contraction entry point, for callers that cannot call
cudaMalloc (a fixed memory budget owned by another allocator, or code that must not synchronize the
device). It must agree with the allocating lnocc_debug_gemm on the same inputs, on consecutive calls
(the shared scratch keeps the previous call's contents), and reject sizes beyond its fixed scratch.

This file is named so that pytest collects it last.
"""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lnocc():
    from paper_2407_11258_gb300 import build
    from paper_2407_11258_gb300 import lnocc as m
    build.build()
    m.load()
    return m


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 3e-5)])
def test_noalloc_matches_allocating_entry_point(lnocc, prec, tol):
    g = torch.Generator(device="cpu").manual_seed(prec)
    shapes = [(300, 77, 131), (129, 200, 1000)]  # two calls in a row, different sizes and contents
    for M, N, K in shapes:
        A = torch.randn(M, K, generator=g, dtype=torch.float64).cuda()
        B = torch.randn(N, K, generator=g, dtype=torch.float64).cuda()
        C_ref = torch.zeros(M, N, dtype=torch.float64, device="cuda")
        C = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        lnocc.lnocc_debug_gemm(prec, A, B, C_ref)
        lnocc.lnocc_gemm_noalloc(prec, A, B, C)
        scale = (A.abs() @ B.abs().T).max()
        assert torch.isfinite(C).all()
        assert ((C - C_ref).abs().max() / scale).item() < tol
        exact = (A.cpu() @ B.cpu().T)
        assert ((C.cpu() - exact).abs().max() / scale.cpu()).item() < tol


@pytest.mark.gpu
def test_noalloc_rejects_oversized_requests(lnocc):
    # (M + N) * roundup(K, 64) * 8 bytes beyond 32 MiB: rejected on the host, before any device work
    A = torch.zeros(4096, 1024, dtype=torch.float64, device="cuda")
    B = torch.zeros(1024, 1024, dtype=torch.float64, device="cuda")
    C = torch.zeros(4096, 1024, dtype=torch.float64, device="cuda")
    with pytest.raises(lnocc.LnoccError) as ei:
        lnocc.lnocc_gemm_noalloc(0, A, B, C)
    assert ei.value.code == lnocc.LNOCC_EINVAL
    assert "32 MiB" in str(ei.value)


@pytest.mark.gpu
def test_noalloc_never_times_tiles_in_tuning_mode(lnocc):
    """With the library-wide tuner in mode 2, a table miss on an ordinary contraction times the tile
    candidates (which allocates a scratch output and synchronizes). The allocation-free entry point must
    only look the table up: no shape tuned, no device memory taken, the same result as before."""
    g = torch.Generator(device="cpu").manual_seed(99)
    M, N, K = 333, 97, 517  # a shape bucket no other test tunes
    A = torch.randn(M, K, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(N, K, generator=g, dtype=torch.float64).cuda()
    C = torch.empty(M, N, dtype=torch.float64, device="cuda")
    C_ref = torch.empty(M, N, dtype=torch.float64, device="cuda")
    lnocc.lnocc_gemm_noalloc(1, A, B, C_ref)  # first call on the device: symbol lookup, module load
    torch.cuda.synchronize()
    prev = lnocc.lnocc_autotune(2)
    try:
        before = lnocc.lnocc_autotune_stats()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(2):
            lnocc.lnocc_gemm_noalloc(1, A, B, C)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        after = lnocc.lnocc_autotune_stats()
    finally:
        lnocc.lnocc_autotune(prev)
    assert after["tuned"] == before["tuned"]
    assert after["misses"] >= before["misses"] + 2  # the lookups did happen
    assert free1 == free0
    assert torch.equal(C, C_ref)
