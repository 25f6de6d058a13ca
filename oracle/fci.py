"""ORACLE (test infrastructure only): brute-force two-electron singlet FCI.

For two electrons (one doubly occupied orbital, nocc = 1) CCSD is exact, so
E_CCSD = E_FCI - E_HF; this pins the whole closed-shell CCSD oracle,
including the sign of the t1 t1 term in tau (Eq. 7).

The singlet spatial wavefunction is Psi(r1, r2) = sum_pq C_pq phi_p(r1) phi_q(r2)
with C symmetric and sum C_pq^2 = 1. With the Hamiltonian of Eq. 2 its energy is
  E = sum C_pq C_rs [h_pr d_qs + d_pr h_qs + (pr|qs)],
so E_FCI is the lowest eigenvalue of that operator on symmetric C.
The one-electron part h is recovered from the Fock matrix of the closed-shell
determinant: h_pq = f_pq - [2(pq|00) - (p0|0q)].
"""
from __future__ import annotations

import numpy as np


def fci_2e(f, B):
    """Return (E_FCI, E_HF) for one doubly occupied orbital (orbital 0)."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 1:
        f = np.diag(f)
    n = B.shape[1]
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    h = f - 2.0 * eri[:, :, 0, 0] + eri[:, 0, 0, :]
    eye = np.eye(n)
    # H[(p,q),(r,s)] = h_pr d_qs + d_pr h_qs + (pr|qs)
    H = (np.einsum("pr,qs->pqrs", h, eye) + np.einsum("pr,qs->pqrs", eye, h)
         + eri.transpose(0, 2, 1, 3)).reshape(n * n, n * n)
    # symmetric-C subspace: orthonormal basis of symmetric n x n matrices
    basis = []
    for p in range(n):
        for q in range(p, n):
            m = np.zeros((n, n))
            if p == q:
                m[p, p] = 1.0
            else:
                m[p, q] = m[q, p] = 1.0 / np.sqrt(2.0)
            basis.append(m.ravel())
    S = np.array(basis).T
    Hs = S.T @ H @ S
    e_fci = float(np.linalg.eigvalsh(0.5 * (Hs + Hs.T))[0])
    e_hf = float(2.0 * h[0, 0] + eri[0, 0, 0, 0])
    return e_fci, e_hf
