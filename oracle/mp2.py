"""ORACLE (test infrastructure only): full-system MP2 and the MP2 composite correction, FP64 on the CPU.

Eq. 17 corrects the sum of the LNO fragment energies by the error the same truncation makes at the
MP2 level:

    Delta E_c,MP2 = E_c,MP2 - sum_F E_c,MP2^(F),

with E_c,MP2 the canonical MP2 correlation energy of the whole system and E_c,MP2^(F) the MP2 fragment
energy evaluated in the fragment's active space A_F: Eq. 12-13 with the first-order amplitudes of
Eq. 21 (t1 = 0, tau = t2).

Active spaces here keep every occupied orbital and an orthonormal set of virtual combinations (the
columns of C_vir, nvir x nvir(F)), standing in for the truncated LNO virtual space of Sec. II.C. As for
the paper's LNOs, the virtual block of A_F is made semicanonical: the Fock matrix restricted to
span(C_vir) is diagonalised, so the first-order amplitudes of A_F have diagonal denominators. Real
orbitals, Gamma point, chemist's notation (ia|jb) = sum_Q B_Qia B_Qjb.
"""
from __future__ import annotations

import numpy as np

from . import fragment


def _ovov(B_ov):
    return np.einsum("Qia,Qjb->iajb", B_ov, B_ov)


def _denominators(eo, ev):
    """D[i,a,j,b] = e_i + e_j - e_a - e_b."""
    return eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]


def full_mp2_energy(eps, B_ov, nocc):
    """Canonical closed-shell MP2 correlation energy of the whole system from its occupied-virtual DF
    block B_ov[Q][i][a]: sum_ijab (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b)."""
    e = np.asarray(eps, dtype=np.float64)
    ovov = _ovov(np.asarray(B_ov, dtype=np.float64))
    D = _denominators(e[:nocc], e[nocc:])
    return float(np.sum(ovov * (2.0 * ovov - ovov.transpose(0, 3, 2, 1)) / D))


def active_space(eps, B_ov, nocc, C_vir):
    """Semicanonical active space: every occupied orbital plus the virtual combinations C_vir
    (orthonormal columns). Returns (eps_F, B_ov_F): the occupied energies followed by the eigenvalues of
    C_vir^T diag(e_vir) C_vir, and B_ov rotated onto the corresponding eigenvectors C_vir R."""
    e = np.asarray(eps, dtype=np.float64)
    C = np.asarray(C_vir, dtype=np.float64)
    if C.ndim == 1:
        C = C[:, None]
    f_vv = C.T @ np.diag(e[nocc:]) @ C
    ev_F, R = np.linalg.eigh(f_vv)
    return np.concatenate([e[:nocc], ev_F]), np.einsum("Qia,ab->Qib", np.asarray(B_ov, dtype=np.float64), C @ R)


def fragment_pair_matrix(eps, B_ov, nocc, C_vir):
    """MP2 pair matrix of the active space: E_ii' = sum_jab t_ij^ab [2(i'a|jb) - (i'b|ja)] (Eq. 13)
    with t_ij^ab = (ia|jb) / D_ij^ab of the semicanonical active space (Eq. 21)."""
    eF, BF = active_space(eps, B_ov, nocc, C_vir)
    ovov = _ovov(BF)
    t2 = (ovov / _denominators(eF[:nocc], eF[nocc:])).transpose(0, 2, 1, 3)  # t[i,j,a,b]
    L = 2.0 * ovov - ovov.transpose(0, 3, 2, 1)                               # L[i',a,j,b]
    return np.einsum("ijab,kajb->ik", t2, L)


def fragment_mp2_energy(eps, B_ov, nocc, C_vir, U_frag):
    """E_c,MP2^(F) = sum_alpha sum_ii' U_i,alpha E_ii' U_i',alpha (Eq. 12) with the active-space MP2
    pair matrix."""
    return fragment.project(fragment_pair_matrix(eps, B_ov, nocc, C_vir), U_frag)


def composite_correction(e_full, e_frags):
    """Eq. 17: Delta E_c,MP2 = E_c,MP2 - sum_F E_c,MP2^(F)."""
    return float(e_full) - float(np.sum(np.asarray(e_frags, dtype=np.float64)))
