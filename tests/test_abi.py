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
    return sorted(set(re.findall(r"\b(lnocc_[a-z_]+)\s*\(", hdr)))


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
    assert o.conv_rms == 1e-8 and o.conv_energy == 1e-10
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
    """ctypes mirrors of lnocc_opts / lnocc_info have the C compiler's size and field offsets."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields_o = [f[0] for f in lnocc.Opts._fields_]
    fields_i = [f[0] for f in lnocc.Info._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "lnocc.h"', "int main(void){",
           'printf("%zu %zu\\n", sizeof(lnocc_opts), sizeof(lnocc_info));']
    src += [f'printf("%zu\\n", offsetof(lnocc_opts, {f}));' for f in fields_o]
    src += [f'printf("%zu\\n", offsetof(lnocc_info, {f}));' for f in fields_i]
    src += ["return 0;}"]
    (tmp_path / "t.c").write_text("\n".join(src))
    exe = tmp_path / "t"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(tmp_path / "t.c"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(lnocc.Opts) and int(out[1]) == ctypes.sizeof(lnocc.Info)
    offs = [int(x) for x in out[2:]]
    assert offs[: len(fields_o)] == [getattr(lnocc.Opts, f).offset for f in fields_o]
    assert offs[len(fields_o):] == [getattr(lnocc.Info, f).offset for f in fields_i]
