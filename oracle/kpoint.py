"""ORACLE (test infrastructure only): two-electron integrals of the local Hamiltonian from k-point DF
factors, Eq. 27a, in complex FP64 on the CPU.

    V_pqrs = sum_q^{N_k} sum_P L^P_pq(q) L^P_rs(-q)

with L^P_pq(q) the (complex) DF factors of momentum transfer q in the basis of the active-space orbitals
(Eq. 27b builds them from AO factors; that half-transformation needs an AO basis and is not part of this
oracle). Written as the plain complex sum; for real orbitals the result is real, which `eri` checks.
"""
from __future__ import annotations

import numpy as np


def eri(L, qneg):
    """V[p,q,r,s] (real part) and the largest imaginary part of the q-sum of Eq. 27a."""
    L = np.asarray(L)
    V = np.zeros(L.shape[2:] * 2, dtype=np.complex128)
    for q in range(L.shape[0]):
        V += np.einsum("Ppq,Prs->pqrs", L[q], L[qneg[q]], optimize=True)
    return V.real.copy(), float(np.abs(V.imag).max(initial=0.0))
