"""GPU parity of the projected energies for every single-LO fragment, of the amplitudes element by
element, and of the (T) energy kernels at large nocc and more LOs than the staged kernels hold.

A fragment energy with one LO u reads u^T E u, i.e. every element of the occupied pair matrix, so
running every column U[:, alpha] of the LO matrix covers the off-diagonal elements that the oracle pins
in tests/test_oracle_pairs.py. Tolerances as in test_gpu_parity.py: 1e-6 Eh mixed, 1e-9 Eh FP64.
"""
import functools

import numpy as np
import pytest

from oracle import ccsd as occ
from oracle import fragment as ofr
from oracle import triples as otr
from paper_2407_11258_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6
FP64_TOL = 1e-9


@pytest.fixture(scope="module")
def lnocc():
    from paper_2407_11258_gb300 import build
    from paper_2407_11258_gb300 import lnocc as m
    build.build()
    m.load()
    return m


def _oracle_pairs(fr, do_t=True):
    r = occ.ccsd(fr.eps, fr.B, fr.nocc, tol_t=1e-11, tol_e=1e-13)
    Ec = occ.pair_energy_matrix(r["t1"], r["t2"], fr.B, fr.nocc)
    Em = occ.pair_energy_matrix(np.zeros_like(r["t1"]), occ.mp2_amplitudes(fr.eps, fr.B, fr.nocc), fr.B, fr.nocc)
    Et = otr.pair_matrix(r["t1"], r["t2"], fr.eps, fr.B, fr.nocc) if do_t else None
    return r, Ec, Em, Et


def _build(lnocc, fr, prec, **opt):
    eps = torch.tensor(fr.eps, device="cuda")
    B = torch.tensor(fr.B, device="cuda")
    return lnocc.lnocc_build_ints(fr.nocc, fr.nvir, fr.naux, eps, B, lnocc.default_opts(precision=prec, **opt))


CASES = [("single_fp64", None), ("ragged", (6, 37, 150)), ("ragged", (9, 70, 280)), ("ragged", (3, 131, 140))]


def _case(kind, shape):
    if kind == "single_fp64":
        return synth.single_fp64()
    o, v, q = shape
    return synth.make_fragment(o, v, q, 500 + o + v, decay=20.0, frag=(0, 1) if o > 1 else (0,))


@pytest.mark.parametrize("kind,shape", CASES)
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_every_single_lo_fragment(lnocc, kind, shape, prec, tol):
    """E^(F) for each one-LO fragment U[:, alpha] (CCSD, MP2 and (T)); the GPU's one-LO energies add up
    to its total energies (Eq. 7: the LOs span the occupied space)."""
    fr = _case(kind, shape)
    r, Ec, Em, Et = _oracle_pairs(fr)
    f = _build(lnocc, fr, prec)
    try:
        e_tot, _, _ = lnocc.lnocc_ccsd(f)
        bad, sums = [], {"ccsd": 0.0, "t": 0.0}
        for al in range(fr.nocc):
            u = np.ascontiguousarray(fr.U[:, [al]])
            U = torch.tensor(u, device="cuda")
            ec, em = lnocc.lnocc_fragment_energy(f, U)
            et, etf = lnocc.lnocc_triples(f, U)
            want = {"ccsd": ofr.project(Ec, u), "mp2": ofr.project(Em, u), "t": ofr.project(Et, u),
                    "t_full": float(np.trace(Et))}
            got = {"ccsd": ec, "mp2": em, "t": etf, "t_full": et}
            bad += [(al, k, got[k] - want[k]) for k in want if not abs(got[k] - want[k]) <= tol]
            sums["ccsd"] += ec
            sums["t"] += etf
        assert not bad, bad
        # (the mixed (T) projections form their i-sums in FP32, so the (T) sum rule holds to the tolerance)
        assert abs(sums["ccsd"] - e_tot) <= 1e-12 and abs(sums["t"] - et) <= tol, (sums, e_tot, et)
    finally:
        f.free()


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (1, 2e-6)])
def test_amplitudes_element_by_element(lnocc, prec, tol):
    """t1 and t2 returned through t1_out / t2_out against the oracle's converged amplitudes, element by
    element, at nocc=4 nvir=24 naux=96 (mixed: the BF16x3 residual's noise floor, a few 1e-7 in t)."""
    fr = synth.single_fp64()
    r = occ.ccsd(fr.eps, fr.B, fr.nocc, tol_t=1e-12, tol_e=1e-14)
    f = _build(lnocc, fr, prec)
    try:
        t1 = torch.empty(fr.nocc, fr.nvir, dtype=torch.float64, device="cuda")
        t2 = torch.empty(fr.nocc, fr.nocc, fr.nvir, fr.nvir, dtype=torch.float64, device="cuda")
        lnocc.lnocc_ccsd(f, t1_out=t1, t2_out=t2)
        d1 = np.abs(t1.cpu().numpy() - r["t1"]).max()
        d2 = np.abs(t2.cpu().numpy() - r["t2"]).max()
        assert d1 <= tol and d2 <= tol, (d1, d2)
        assert np.abs(r["t2"]).max() > 1e-3 and np.abs(r["t1"]).max() > 1e-5  # not vacuous
    finally:
        f.free()


def _nocc34(nlo):
    return synth.make_fragment(34, 6, 40, 3409, decay=20.0, frag=tuple(range(nlo)))


@functools.lru_cache(maxsize=1)
def _oracle_nocc34():
    return _oracle_pairs(_nocc34(1))  # the pair matrices do not depend on the fragment's LOs


@pytest.mark.parametrize("prec,tol,nlo", [(0, FP64_TOL, 1), (0, FP64_TOL, 9), (1, MIXED_TOL, 9), (1, MIXED_TOL, 3)])
def test_triples_large_nocc_and_many_los(lnocc, prec, tol, nlo):
    """nocc=34 (beyond 32 occupied orbitals; the FP64 (T) blocks no longer fit shared memory, so the
    generic energy kernel runs) with 1 and 9 LOs (beyond the staged kernels' 8). Small nvir keeps the
    oracle quick."""
    fr = _nocc34(nlo)
    r, Ec, Em, Et = _oracle_nocc34()
    f = _build(lnocc, fr, prec)
    try:
        lnocc.lnocc_ccsd(f)
        U = torch.tensor(fr.U_frag, device="cuda")
        et, etf = lnocc.lnocc_triples(f, U)
        ec, em = lnocc.lnocc_fragment_energy(f, U)
    finally:
        f.free()
    assert abs(et - np.trace(Et)) <= tol, et - np.trace(Et)
    assert abs(etf - ofr.project(Et, fr.U_frag)) <= tol, etf - ofr.project(Et, fr.U_frag)
    assert abs(ec - ofr.project(Ec, fr.U_frag)) <= tol
    assert abs(em - ofr.project(Em, fr.U_frag)) <= tol


@pytest.mark.parametrize("shape", [(16, 30, 120), (32, 12, 48)])
def test_triples_lo_counts_on_the_specialised_kernels(lnocc, shape):
    """The mixed (T) energy kernels are compiled per LO count (0, 1, 2, 4, 8; U zero-padded) and, at
    nocc 16, per nocc; nocc 32 runs the w-only kernel. One solve, then lnocc_triples with no LOs and with
    1, 3, 4, 6 and 8 columns of the LO matrix, each against the oracle's (T) pair matrix projected
    with the same columns; the grouped contraction launches run at both sizes."""
    o, v, q = shape
    fr = synth.make_fragment(o, v, q, 5300 + o, decay=20.0, frag=tuple(range(8)))
    r, Ec, Em, Et = _oracle_pairs(fr)
    f = _build(lnocc, fr, 1)
    try:
        lnocc.lnocc_ccsd(f)
        et0, etf0 = lnocc.lnocc_triples(f, None)
        assert abs(et0 - np.trace(Et)) <= MIXED_TOL and etf0 == 0.0
        for nlo in (1, 3, 4, 6, 8):
            Un = np.ascontiguousarray(fr.U_frag[:, :nlo])
            et, etf = lnocc.lnocc_triples(f, torch.tensor(Un, device="cuda"))
            assert abs(et - et0) < 1e-12  # the canonical sum does not depend on the LOs
            assert abs(etf - ofr.project(Et, Un)) <= MIXED_TOL, (nlo, etf - ofr.project(Et, Un))
    finally:
        f.free()
