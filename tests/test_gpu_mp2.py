"""GPU parity of the MP2 composite correction (Eq. 17): the full-system MP2 energy of lnocc_mp2_energy
and the fragment MP2 energies of lnocc_fragment_energy against oracle/mp2.py.

Fragments here keep every occupied orbital and the lowest k virtuals (C_vir = the first k columns of
the identity, already semicanonical), so their active-space inputs are plain slices of the system's
(eps, B); each fragment is one LO of the system's LO matrix U.
Tolerances: FP64 path 1e-11 Eh (rounding of sums of ~1e5 terms). Mixed path: every (ia|jb) is a sum of
BF16x3 products, whose error is at most about 2^-16 of sum_Q |B_Qia| |B_Qjb| per product split; the
energy moves by at most sum |dE/dx| |dx| with dE/dx_iajb = (4 x_iajb - 2 x_ibja) / D, so the test allows
2^-15 sum_iajb |4 x - 2 x'| / |D| sum_Q |B_Qia| |B_Qjb| (a bound, computed from the oracle's integrals);
the fragment MP2 energies use the same bound in their own active spaces, or 1e-6 Eh, the larger.
"""
import numpy as np
import pytest

from oracle import mp2 as omp2
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


def mixed_bound(eps, Bov, o):
    """2^-15 sum |4x - 2x'| / |D| sum_Q |B_Qia||B_Qjb| (see the module docstring)."""
    e = np.asarray(eps)
    x = np.einsum("Qia,Qjb->iajb", Bov, Bov)
    xa = np.einsum("Qia,Qjb->iajb", np.abs(Bov), np.abs(Bov))
    D = e[:o, None, None, None] - e[None, o:, None, None] + e[None, None, :o, None] - e[None, None, None, o:]
    return 2.0**-15 * float(np.sum(np.abs(4 * x - 2 * x.transpose(0, 3, 2, 1)) / np.abs(D) * xa))


def _system(o, v, q, seed):
    return synth.make_fragment(o, v, q, seed, decay=20.0, frag=tuple(range(o)))


@pytest.mark.parametrize("o,v,q", [(4, 24, 96), (7, 45, 130), (13, 131, 300), (30, 200, 640)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-6)])
def test_full_system_mp2_energy(lnocc, o, v, q, prec, tol):
    fr = _system(o, v, q, 7000 + o)
    Bov = np.ascontiguousarray(fr.B[:, :o, o:])
    want = omp2.full_mp2_energy(fr.eps, Bov, o)
    eps = torch.tensor(fr.eps, device="cuda")
    Bd = torch.tensor(Bov, device="cuda")
    got = lnocc.lnocc_mp2_energy(prec, o, v, q, eps, Bd)
    if prec == 1:
        tol = mixed_bound(fr.eps, Bov, o)
    assert abs(got - want) <= tol, (got, want, tol)
    # the same call on a caller-owned workspace gives the same bits, twice in a row
    nb = lnocc.lnocc_mp2_workspace_bytes(prec, o, v, q)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    assert lnocc.lnocc_mp2_energy(prec, o, v, q, eps, Bd, workspace=ws) == got
    assert lnocc.lnocc_mp2_energy(prec, o, v, q, eps, Bd, workspace=ws) == got


def test_workspace_too_small_is_rejected(lnocc):
    o, v, q = 4, 24, 96
    fr = _system(o, v, q, 7100)
    eps = torch.tensor(fr.eps, device="cuda")
    Bd = torch.tensor(np.ascontiguousarray(fr.B[:, :o, o:]), device="cuda")
    nb = lnocc.lnocc_mp2_workspace_bytes(0, o, v, q)
    ws = torch.empty(nb - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(lnocc.LnoccError) as ei:
        lnocc.lnocc_mp2_energy(0, o, v, q, eps, Bd, workspace=ws)
    assert ei.value.code == lnocc.LNOCC_EINVAL


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_composite_correction(lnocc, prec, tol):
    """Delta E_MP2 = E_MP2(system) - sum_F E_MP2^(F) for one-LO fragments with truncated virtual spaces
    (k_F = 60% .. 100% of the virtuals), and zero when every fragment keeps the whole space."""
    o, v, q = 6, 60, 200
    fr = _system(o, v, q, 7200)
    Bov = np.ascontiguousarray(fr.B[:, :o, o:])
    eps = torch.tensor(fr.eps, device="cuda")
    e_full = lnocc.lnocc_mp2_energy(prec, o, v, q, eps, torch.tensor(Bov, device="cuda"))
    for ks in ([v] * o, [int(v * (0.6 + 0.08 * a)) for a in range(o)]):
        e_frag_gpu, e_frag_ref = [], []
        for a, k in enumerate(ks):
            u = np.ascontiguousarray(fr.U[:, [a]])
            n = o + k
            epsF = torch.tensor(fr.eps[:n], device="cuda")
            BF = torch.tensor(np.ascontiguousarray(fr.B[:, :n, :n]), device="cuda")
            f = lnocc.lnocc_build_ints(o, k, q, epsF, BF, lnocc.default_opts(precision=prec))
            try:
                _, em = lnocc.lnocc_fragment_energy(f, torch.tensor(u, device="cuda"), ccsd=False)
            finally:
                f.free()
            e_frag_gpu.append(em)
            e_frag_ref.append(omp2.fragment_mp2_energy(fr.eps, Bov, o, np.eye(v)[:, :k], u))
        corr_gpu = omp2.composite_correction(e_full, e_frag_gpu)
        corr_ref = omp2.composite_correction(omp2.full_mp2_energy(fr.eps, Bov, o), e_frag_ref)
        if prec == 1:
            tol = max(tol, 2 * mixed_bound(fr.eps, Bov, o))  # the full energy and the fragment sum
        assert abs(corr_gpu - corr_ref) <= tol, (corr_gpu, corr_ref, tol)
        if ks[0] == v:
            assert abs(corr_ref) < 1e-13 and abs(corr_gpu) <= tol
        else:
            assert corr_ref < -1e-5  # truncated virtual spaces leave a negative correction
