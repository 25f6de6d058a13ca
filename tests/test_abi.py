"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

from paper_2407_11258_gb300 import build, lnocc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "lnocc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(lnocc_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lnocc.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("lnocc_build_ints", "lnocc_ccsd", "lnocc_triples", "lnocc_fragment_energy"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
    assert set(lnocc.EXPORTS) == set(declared_symbols())


def test_default_options_and_version(lib):
    o = lnocc.default_opts()
    assert o.precision == lnocc.LNOCC_PREC_MIXED and o.max_iter == 100 and o.diis_space == 8
    assert o.conv_rms == 1e-8 and o.conv_energy == 1e-10 and o.graph == 1
    assert b"sm_103a" in lib.lnocc_version()


def test_argument_validation_needs_no_gpu(lib):
    """Bad sizes and null pointers are rejected on the host before any device work."""
    h = ctypes.c_void_p()
    assert lib.lnocc_build_ints(0, 4, 8, None, None, None, None, ctypes.byref(h)) == lnocc.LNOCC_EINVAL
    assert b"bad arguments" in lib.lnocc_last_error()
    opts = lnocc.default_opts(precision=7)
    assert lib.lnocc_build_ints(1, 1, 1, 16, 16, ctypes.byref(opts), None, ctypes.byref(h)) == lnocc.LNOCC_EINVAL
    assert lib.lnocc_ccsd(None, None, None, 0, None, None, None, None, None) == lnocc.LNOCC_EINVAL
    assert lib.lnocc_triples(None, 0, None, None, None, None) == lnocc.LNOCC_EINVAL
    assert lib.lnocc_free_fragment(None) == lnocc.LNOCC_OK


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the header's structs have the C compiler's size and field offsets."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = [("lnocc_opts", lnocc.Opts), ("lnocc_info", lnocc.Info), ("lnocc_batch_item", lnocc.BatchItem),
               ("lnocc_batch_opts", lnocc.BatchOpts), ("lnocc_batch_result", lnocc.BatchResult)]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "lnocc.h"', "int main(void){"]
    for cname, py in mirrors:
        src.append(f'printf("%zu\\n", sizeof({cname}));')
        src += [f'printf("%zu\\n", offsetof({cname}, {f[0]}));' for f in py._fields_]
    src += ["return 0;}"]
    (tmp_path / "t.c").write_text("\n".join(src))
    exe = tmp_path / "t"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(tmp_path / "t.c"), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, py in mirrors:
        want.append(ctypes.sizeof(py))
        want += [getattr(py, f[0]).offset for f in py._fields_]
    assert out == want


def test_batch_argument_validation_needs_no_gpu(lib):
    """lnocc_solve_batch rejects bad items and options on the host before touching the device."""
    b = lnocc.default_batch_opts()
    assert b.workers == 0 and b.triples == 1 and b.order == lnocc.LNOCC_ORDER_LPT and b.mem_budget_gb == 0.0
    res = (lnocc.BatchResult * 1)()
    assert lib.lnocc_solve_batch(0, None, None, None, None, None) == lnocc.LNOCC_OK
    assert lib.lnocc_solve_batch(-1, None, None, None, None, None) == lnocc.LNOCC_EINVAL
    items = (lnocc.BatchItem * 1)()
    items[0] = lnocc.BatchItem(4, 20, 80, 0, 1, 1, None)
    bad = lnocc.default_batch_opts(workers=99)
    assert lib.lnocc_solve_batch(1, items, None, ctypes.byref(bad), res, None) == lnocc.LNOCC_EINVAL
    assert b"batch options" in lib.lnocc_last_error()
    items[0] = lnocc.BatchItem(4, 20, 80, 2, 1, 1, None)  # nlo > 0 without U_frag
    assert lib.lnocc_solve_batch(1, items, None, None, res, None) == lnocc.LNOCC_EINVAL
    assert b"bad item 0" in lib.lnocc_last_error()


def test_autotune_table_io_needs_no_gpu(lib, tmp_path):
    """Mode switch, text table load (merge, invalid lines skipped) and save round trip, host only."""
    prev = lnocc.lnocc_autotune(1)
    try:
        assert lnocc.lnocc_autotune(-1) == 1
        with pytest.raises(lnocc.LnoccError):
            lnocc.lnocc_autotune(3)
        n0 = lnocc.lnocc_autotune_stats()["entries"]
        src = tmp_path / "tiles.txt"
        src.write_text("# comment\n1 20 9 14 128\n2 22 16 10 256\n1 20 9 15 100\nnot a line\n")
        lnocc.lnocc_autotune_load(str(src))
        assert lnocc.lnocc_autotune_stats()["entries"] == n0 + 2  # BN=100 is not a kernel: skipped
        out = tmp_path / "saved.txt"
        lnocc.lnocc_autotune_save(str(out))
        rows = [r for r in out.read_text().splitlines() if not r.startswith("#")]
        assert "1 20 9 14 128" in rows and "2 22 16 10 256" in rows
        with pytest.raises(lnocc.LnoccError):
            lnocc.lnocc_autotune_load(str(tmp_path / "missing.txt"))
    finally:
        lnocc.lnocc_autotune(prev)


def test_binding_rejects_mis_sized_arrays_before_the_call(lib):
    """The binding checks every array's element count against the sizes it passes, before the
    pointer is taken: CPU tensors of the right size get as far as the CUDA-tensor check (TypeError),
    mis-sized ones stop at the size check (ValueError). No device work in either case."""
    import numpy as np
    import torch
    o, v, q = 2, 3, 4
    n = o + v
    eps, B = torch.zeros(n, dtype=torch.float64), torch.zeros(q, n, n, dtype=torch.float64)
    with pytest.raises(TypeError):
        lnocc.lnocc_build_ints(o, v, q, eps, B)
    with pytest.raises(ValueError, match="eps"):
        lnocc.lnocc_build_ints(o, v, q, torch.zeros(n - 1, dtype=torch.float64), B)
    with pytest.raises(ValueError, match="B"):
        lnocc.lnocc_build_ints(o, v, q, eps, torch.zeros(q, n, n - 1, dtype=torch.float64))
    f = lnocc.Fragment(None, (o, v))
    t2 = torch.zeros(o, o, v, v, dtype=torch.float64)
    with pytest.raises(TypeError):
        lnocc.lnocc_ccsd(f, t2_out=t2)
    for kw in ({"t1_in": torch.zeros(o, v + 1, dtype=torch.float64)},
               {"t2_in": torch.zeros(o, o, v, v - 1, dtype=torch.float64)},
               {"t1_out": torch.zeros(o * v - 1, dtype=torch.float64)},
               {"t2_out": torch.zeros(o, v, v, dtype=torch.float64)}):
        with pytest.raises(ValueError, match=next(iter(kw))):
            lnocc.lnocc_ccsd(f, **kw)
    with pytest.raises(ValueError, match="t2_out"):
        lnocc.lnocc_mlp_guess(f, None, torch.zeros(o, o, v, dtype=torch.float64))
    U = torch.zeros(o, 1, dtype=torch.float64)
    with pytest.raises(TypeError):
        lnocc.lnocc_triples(f, U)
    for bad in (torch.zeros(o + 1, 1, dtype=torch.float64), torch.zeros(o, dtype=torch.float64)):
        with pytest.raises(ValueError, match="U_frag"):
            lnocc.lnocc_triples(f, bad)
        with pytest.raises(ValueError, match="U_frag"):
            lnocc.lnocc_fragment_energy(f, bad)
    with pytest.raises(ValueError, match="item 0 B"):
        lnocc.lnocc_solve_batch([(o, v, q, eps, torch.zeros(q, n, dtype=torch.float64), U)])
    with pytest.raises(ValueError, match="item 1 U_frag"):
        lnocc.lnocc_solve_batch([(o, v, q, eps, B, U), (o, v, q, eps, B, torch.zeros(o + 1, 1, dtype=torch.float64))])
    A = torch.zeros(5, 7, dtype=torch.float64)
    with pytest.raises(ValueError, match="C"):
        lnocc.lnocc_debug_gemm(1, A, torch.zeros(3, 7, dtype=torch.float64), torch.zeros(5, 2, dtype=torch.float64))
    with pytest.raises(ValueError, match="B"):
        lnocc.lnocc_gemm_noalloc(1, A, torch.zeros(3, 6, dtype=torch.float64), torch.zeros(5, 3, dtype=torch.float64))
    idx = torch.zeros(6, dtype=torch.int64)
    with pytest.raises(ValueError, match="X"):
        lnocc.lnocc_mlp_samples(f, idx, torch.zeros(6, lnocc.NFEAT - 1, dtype=torch.float32))
    with pytest.raises(ValueError, match="dt"):
        lnocc.lnocc_mlp_samples(f, idx, torch.zeros(6, lnocc.NFEAT, dtype=torch.float32),
                                torch.zeros(5, dtype=torch.float32))
    m = lnocc.Mlp.__new__(lnocc.Mlp)  # no device handle: only the host-side checks run
    m.h = None
    with pytest.raises(ValueError, match="norm"):
        m.set_norm(np.zeros(16))
    with pytest.raises(ValueError, match="dt"):
        m.train_step(torch.zeros(4, lnocc.NFEAT, dtype=torch.float32), torch.zeros(3, dtype=torch.float32), 1e-3)


def test_workspace_queries_need_no_gpu(lib):
    """lnocc_workspace_bytes / lnocc_mp2_workspace_bytes are host arithmetic: bad arguments give
    EINVAL, the (T) scratch grows with the W-chunk bound until the chunk holds the largest b-slab
    ((b + 1)(v - b) nocc^3 elements) and stays constant beyond it, FP32 W needs less than FP64 W, and
    it always holds at least one chunk of W for the largest slab's single c (v nocc^3 elements)."""
    with pytest.raises(lnocc.LnoccError):
        lnocc.lnocc_workspace_bytes(0, 24, 96)
    with pytest.raises(lnocc.LnoccError):
        lnocc.lnocc_workspace_bytes(4, 24, 96, lnocc.default_opts(precision=5))
    with pytest.raises(lnocc.LnoccError):
        lnocc.lnocc_workspace_bytes(4, 24, 96, lnocc.default_opts(triples_chunk_mb=-1))
    with pytest.raises(lnocc.LnoccError):
        lnocc.lnocc_mp2_workspace_bytes(2, 4, 24, 96)
    b = ctypes.c_longlong(0)
    assert lib.lnocc_workspace_bytes(4, 24, 96, None, None) == lnocc.LNOCC_EINVAL
    assert lib.lnocc_workspace_bytes(4, 24, 96, None, ctypes.byref(b)) == lnocc.LNOCC_OK and b.value > 0
    o, v, q = 8, 60, 240
    max_slab = max((bb + 1) * (v - bb) for bb in range(v)) * o ** 3
    for prec, esz in ((lnocc.LNOCC_PREC_FP64, 8), (lnocc.LNOCC_PREC_MIXED, 4)):
        sizes = [lnocc.lnocc_workspace_bytes(o, v, q, lnocc.default_opts(precision=prec, triples_chunk_mb=mb))
                 for mb in (1, 2, 4, 8, 768, 4096)]
        assert all(x <= y for x, y in zip(sizes, sizes[1:]))
        assert sizes[0] >= v * o ** 3 * esz
        assert sizes[-1] == sizes[-2]  # 768 MB already holds the largest slab
        assert sizes[-1] - sizes[0] <= max_slab * esz
    assert (lnocc.lnocc_workspace_bytes(o, v, q, lnocc.default_opts(precision=lnocc.LNOCC_PREC_MIXED))
            < lnocc.lnocc_workspace_bytes(o, v, q, lnocc.default_opts(precision=lnocc.LNOCC_PREC_FP64)))
    for prec in (lnocc.LNOCC_PREC_FP64, lnocc.LNOCC_PREC_MIXED):
        small, large = (lnocc.lnocc_mp2_workspace_bytes(prec, 4, 24, 96),
                        lnocc.lnocc_mp2_workspace_bytes(prec, 16, 240, 960))
        assert 0 < small < large
