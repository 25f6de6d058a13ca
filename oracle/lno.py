"""ORACLE (test infrastructure only): local active space of a fragment in FP64 on the CPU (Sec. II.C).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` use this module; the
product library never does.

For a fragment F with LO coefficients U_occ^(F) (N_occ x n_LO, rows = canonical occupied orbitals) and,
for LOs that overlap the virtual space, U_vir^(F) (N_vir x n_LO), the steps are those of Sec. II.C:

1. Eq. 18: U = [W W_bar] [Sigma 0] [V V_bar]^T. The left singular vectors with non-zero
   singular values span the internal space (Eq. 19), the others the external space. Reading: a singular
   value counts as zero below `sv_tol` (1e-10 relative to the largest).
2. The internal orbitals are made semi-canonical (the Fock matrix, diagonal eps in the canonical basis,
   is diagonalised inside the internal space; the MP1 amplitudes of Eq. 21 need f_{i_F i_F}).
   Reading: the paper names the amplitudes semi-canonical without printing this step; without it the
   result would depend on the basis chosen inside a degenerate singular subspace (orthonormal LO
   columns give all singular values equal to one), which the tests pin.
3. Eq. 21 with Eq. 22 at the Gamma point and real orbitals:
   t_{i_F a j b} = V_{i_F a j b} / (f_{i_F i_F} + e_j - e_a - e_b),  V_{i_F a j b} = sum_i W_{i i_F} (ia|jb).
   An amplitude with the internal index in the third slot is the same number: t_{j b i_F a}.
4. Eq. 20: the occupied and virtual blocks of the MP2 density with one occupied index
   restricted to the internal space (LNO), or Eq. 28: the cluster-specific bath
   natural orbital (CBNO) densities, where both virtual (occupied block) or both occupied (virtual
   block) indices are internal. Reading of Eq. 28a: the first amplitude's virtual labels are the
   internal a_F, b_F that the sum runs over (the printed t*_{iakb} drops their subscript).
5. Eq. 24-26: diagonalise the density inside the external space, D_bar = W_bar^T D W_bar = X Lambda X^T
   (Eq. 24), LNOs W_bar X (Eq. 25), keep |lambda| >= eta (Eq. 26); eigenvalues in decreasing order.
Real orbitals: complex conjugates are dropped. Plain numpy: SVD and symmetric eigendecomposition are
library routines; the densities are written as in the equations.
"""
from __future__ import annotations

import numpy as np


def internal_space(U, e_block, sv_tol=1e-10):
    """Steps 1-2 for one block (occupied or virtual). U: [n][n_LO]; e_block: canonical energies of the
    block. Returns (W_int [n][n_int] semicanonical, f_int [n_int] ascending, W_ext [n][n - n_int])."""
    U = np.asarray(U, dtype=np.float64)
    if U.ndim == 1:
        U = U[:, None]
    Wfull, s, _ = np.linalg.svd(U, full_matrices=True)
    n_int = int(np.sum(s > sv_tol * max(s.max(initial=0.0), 1e-300))) if s.size else 0
    W, Wbar = Wfull[:, :n_int], Wfull[:, n_int:]
    f = W.T @ np.diag(np.asarray(e_block, dtype=np.float64)) @ W
    f_int, R = np.linalg.eigh(f)
    return W @ R, f_int, Wbar


def _ovov(B_ov):
    return np.einsum("Qia,Qjb->iajb", B_ov, B_ov)


def mp1_internal(eps, B_ov, nocc, W_int, f_int):
    """Step 3: t[iF, a, j, b] = sum_i W[i, iF] (ia|jb) / (f_iF + e_j - e_a - e_b)."""
    e = np.asarray(eps, dtype=np.float64)
    eo, ev = e[:nocc], e[nocc:]
    V = np.einsum("iI,iajb->Iajb", W_int, _ovov(B_ov))
    D = f_int[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return V / D


def lno_densities(eps, B_ov, nocc, U_occ):
    """Step 4, Eq. 20: (D_occ [nocc][nocc], D_vir [nvir][nvir]) of the LNO construction."""
    e = np.asarray(eps, dtype=np.float64)
    W, f, _ = internal_space(U_occ, e[:nocc])
    t = mp1_internal(e, B_ov, nocc, W, f)          # t[kF, b, i, a] = t_{i a kF b}
    # D_ij = 2 sum_kF sum_ab t_{i a kF b} (2 t_{j a kF b} - t_{j b kF a})
    D_occ = 2.0 * (2.0 * np.einsum("Kbia,Kbja->ij", t, t) - np.einsum("Kbia,Kajb->ij", t, t))
    # D_ab = sum_iF sum_jc 2 (t_{iF a j c} t_{iF b j c} + t_{iF c j a} t_{iF c j b})
    #                     - (t_{iF c j a} t_{iF b j c} + t_{iF a j c} t_{iF c j b})
    D_vir = (2.0 * (np.einsum("Iajc,Ibjc->ab", t, t) + np.einsum("Icja,Icjb->ab", t, t))
             - (np.einsum("Icja,Ibjc->ab", t, t) + np.einsum("Iajc,Icjb->ab", t, t)))
    return D_occ, D_vir


def cbno_densities(eps, B_ov, nocc, U_occ, U_vir):
    """Step 4, Eq. 28 (CBNO): D_ij = 2 sum_{aF bF} sum_k t_{i aF k bF} (2 t_{j aF k bF} - t_{j bF k aF}) with
    internal virtuals a_F, b_F; D_ab = 2 sum_{iF jF} sum_c t_{iF a jF c} (2 t_{iF b jF c} - t_{iF c jF b}) with
    internal occupied i_F, j_F. Amplitudes t_{pa qb} = (pa|qb) / (f_p + f_q - f_a - f_b) in the basis where the
    internal orbitals are semi-canonical (canonical energies elsewhere)."""
    e = np.asarray(eps, dtype=np.float64)
    eo, ev = e[:nocc], e[nocc:]
    Wo, fo, _ = internal_space(U_occ, eo)
    Wv, fv, _ = internal_space(U_vir, ev)
    ovov = _ovov(B_ov)
    # occupied block: both virtuals internal
    Vv = np.einsum("iajb,aA,bB->iAjB", ovov, Wv, Wv)
    tv = Vv / (eo[:, None, None, None] - fv[None, :, None, None] + eo[None, None, :, None] - fv[None, None, None, :])
    D_occ = 2.0 * (2.0 * np.einsum("iAkB,jAkB->ij", tv, tv) - np.einsum("iAkB,jBkA->ij", tv, tv))
    # virtual block: both occupieds internal
    Vo = np.einsum("iajb,iI,jJ->IaJb", ovov, Wo, Wo)
    to = Vo / (fo[:, None, None, None] - ev[None, :, None, None] + fo[None, None, :, None] - ev[None, None, None, :])
    D_vir = 2.0 * (2.0 * np.einsum("IaJc,IbJc->ab", to, to) - np.einsum("IaJc,IcJb->ab", to, to))
    return D_occ, D_vir


def select(D, W_ext, eta):
    """Step 5: eigenpairs of W_ext^T D W_ext with |lambda| >= eta, decreasing; returns (lambda, LNO coefficients
    W_ext X [n][n_keep])."""
    Dbar = W_ext.T @ D @ W_ext
    lam, X = np.linalg.eigh(0.5 * (Dbar + Dbar.T))
    order = np.argsort(-lam, kind="stable")
    lam, X = lam[order], X[:, order]
    keep = np.abs(lam) >= eta
    return lam[keep], W_ext @ X[:, keep]


def external_spectrum(D, W_ext):
    """All eigenvalues of the external-space density W_ext^T D W_ext, decreasing."""
    Dbar = W_ext.T @ D @ W_ext
    return np.sort(np.linalg.eigvalsh(0.5 * (Dbar + Dbar.T)))[::-1]


def active_space(eps, B, nocc, C_occ, C_vir):
    """The fragment's active space in semi-canonical form (the input of the fragment CCSD, Sec. II.B):
    the Fock matrix (diagonal eps in the canonical basis) is diagonalised inside span(C_occ) and inside
    span(C_vir); returns (eps_F increasing within each block, B_F[Q] = C_F^T B[Q] C_F, C_F [n][nF] block
    diagonal) with the Gamma-point real DF factors B [naux][n][n] of Eq. 27."""
    e = np.asarray(eps, dtype=np.float64)
    fo, Ro = np.linalg.eigh(C_occ.T @ np.diag(e[:nocc]) @ C_occ)
    fv, Rv = np.linalg.eigh(C_vir.T @ np.diag(e[nocc:]) @ C_vir)
    n = e.size
    no, nv = C_occ.shape[1], C_vir.shape[1]
    CF = np.zeros((n, no + nv))
    CF[:nocc, :no] = C_occ @ Ro
    CF[nocc:, no:] = C_vir @ Rv
    return np.concatenate([fo, fv]), np.einsum("ps,Qpq,qt->Qst", CF, B, CF, optimize=True), CF
