"""ORACLE (test infrastructure only): projection of pair matrices onto fragment LOs.

E^(F) = sum_{alpha in F} sum_ii' U_i,alpha E_ii' U_i',alpha (Eq. 12 for CCSD,
Eq. 15 for (T)); with real orbitals the complex conjugate is dropped. When the
columns of U span the occupied space (Eq. 5) the fragment energies of all
fragments add up to the trace of E (Eq. 7).
"""
from __future__ import annotations

import numpy as np


def project(E, U_frag):
    """sum_alpha sum_ii' U[i,alpha] E[i,i'] U[i',alpha] written as explicit loops."""
    E = np.asarray(E, dtype=np.float64)
    U = np.asarray(U_frag, dtype=np.float64)
    if U.ndim == 1:
        U = U[:, None]
    o, nlo = U.shape
    tot = 0.0
    for al in range(nlo):
        for i in range(o):
            for ip in range(o):
                tot += U[i, al] * E[i, ip] * U[ip, al]
    return tot
