"""GPU parity of the k-point integral assembly (lnocc_kpoint_df, Eq. 27a) against oracle/kpoint.py, and a
fragment CCSD solved from the reduced real factors against the oracle's CCSD on the equivalent real
supercell factors (the discrete-Fourier identity pinned in tests/test_oracle_kpoint.py makes their
integrals equal)."""
import numpy as np
import pytest

from oracle import ccsd as occ
from oracle import kpoint as okp
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


@pytest.mark.parametrize("nk,naux,n", [(1, 6, 5), (4, 5, 7), (5, 3, 6), (8, 4, 9)])
def test_reduced_factors_reproduce_the_q_sum(lnocc, nk, naux, n):
    L, qneg, _ = synth.kpoint_factors(nk, naux, n, 50 + nk)
    B, err = lnocc.lnocc_kpoint_df(torch.tensor(L, device="cuda"), list(qneg))
    assert B.shape == (nk * naux, n, n) and err < 1e-14
    Bn = B.cpu().numpy()
    V = np.einsum("Qpq,Qrs->pqrs", Bn, Bn)
    V_ref, imag = okp.eri(L, qneg)
    assert imag < 1e-13
    assert np.abs(V - V_ref).max() < 1e-13 * max(1.0, np.abs(V_ref).max())
    assert np.abs(Bn - Bn.transpose(0, 2, 1)).max() == 0.0  # symmetric in (p, q), as lnocc_build_ints needs


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-6)])
def test_fragment_ccsd_from_kpoint_factors(lnocc, prec, tol):
    nk, naux, o, v = 4, 8, 4, 16
    n = o + v
    L, qneg, Bc = synth.kpoint_factors(nk, naux, n, 77)
    eps = synth.orbital_energies(synth.Stream(77, 1), o, v, (-1.2, -0.4), (0.3, 3.0))
    B, _ = lnocc.lnocc_kpoint_df(torch.tensor(L, device="cuda"), list(qneg))
    f = lnocc.lnocc_build_ints(o, v, nk * naux, torch.tensor(eps, device="cuda"), B, lnocc.default_opts(precision=prec))
    try:
        e, _, _ = lnocc.lnocc_ccsd(f)
        e_t, _ = lnocc.lnocc_triples(f)
    finally:
        f.free()
    from oracle import triples as otr
    r = occ.ccsd(eps, Bc, o, tol_t=1e-11, tol_e=1e-13)
    assert abs(e - r["e_corr"]) <= tol
    assert abs(e_t - otr.energy(r["t1"], r["t2"], eps, Bc, o)) <= tol


def test_factors_without_real_orbital_symmetry_are_rejected(lnocc):
    L, qneg, _ = synth.kpoint_factors(4, 3, 5, 9)
    Lb = L.copy()
    Lb[1, 0, 0, 1] += 1e-3j  # breaks L(-q) = conj L(q)
    with pytest.raises(lnocc.LnoccError) as ei:
        lnocc.lnocc_kpoint_df(torch.tensor(Lb, device="cuda"), list(qneg))
    assert ei.value.code == lnocc.LNOCC_EINVAL
    with pytest.raises(lnocc.LnoccError):
        lnocc.lnocc_kpoint_df(torch.tensor(L, device="cuda"), [0, 2, 1, 1])  # not an involution
