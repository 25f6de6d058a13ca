"""Pins of the k-point integral oracle (oracle/kpoint.py, Eq. 27a).

* Factors built as the discrete Fourier transform of real supercell factors B_R (one block of auxiliary
  functions per cell R) must give, through the q-sum of Eq. 27a, exactly the real supercell integrals
  sum_{P,R} B_R[P][p][q] B_R[P][r][s]: sum_q exp(i q (R - R')) = N_k delta_RR' (an identity of the
  discrete Fourier transform, independent of the oracle's complex sum).
* One k-point (N_k = 1) reduces to the real Gamma-point form the fragment solver uses.
* The result is real and has the 8-fold symmetry of real-orbital integrals.
* A planted mistake (L(q) paired with L(q) instead of L(-q)) breaks both.
"""
import numpy as np
import pytest

from oracle import kpoint
from paper_2407_11258_gb300 import synth


@pytest.mark.parametrize("nk,naux,n", [(1, 6, 5), (3, 4, 6), (4, 5, 5), (6, 3, 4)])
def test_q_sum_reproduces_the_supercell_integrals(nk, naux, n):
    L, qneg, Bc = synth.kpoint_factors(nk, naux, n, 10 + nk)
    V, imag = kpoint.eri(L, qneg)
    Vsc = np.einsum("Qpq,Qrs->pqrs", Bc, Bc)
    assert imag < 1e-13
    assert np.abs(V - Vsc).max() < 1e-13
    assert np.abs(V - V.transpose(1, 0, 2, 3)).max() < 1e-13
    assert np.abs(V - V.transpose(2, 3, 0, 1)).max() < 1e-13


def test_planted_mistake_pairing_q_with_itself_fails():
    L, qneg, Bc = synth.kpoint_factors(4, 5, 5, 3)
    V_bad, imag = kpoint.eri(L, np.arange(4))
    Vsc = np.einsum("Qpq,Qrs->pqrs", Bc, Bc)
    assert np.abs(V_bad - Vsc).max() > 1e-3 or imag > 1e-3
