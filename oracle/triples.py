"""ORACLE (test infrastructure only): LNO-(T) pair matrix in FP64 on the CPU.

Follows the supplementary Sec. S1 (intermediates after Nagy & Kallay, J. Chem.
Phys. 146, 214106 (2017)) and Eq. 16 of the main text:

  W_ijk^abc = P_ijk^abc { sum_d (bd|ai) t_kj^cd - sum_l (ck|jl) t_il^ab }
  V_ijk^abc = W_ijk^abc + 1/2 P_ijk^abc { (ai|bj) t_k^c }
  Delta_ijk^abc = f_ii + f_jj + f_kk - f_aa - f_bb - f_cc
  w = W / sqrt(-Delta),  v = V / sqrt(-Delta)
  E_ii',(T) = -1/3 sum_jkabc (4 w_ijk^abc + w_ijk^bca + w_ijk^cab)(v_i'jk^abc - v_i'jk^cba)

where P sums the six simultaneous permutations of (i,a), (j,b), (k,c).
Readings (real orbitals): t_kcjd is t_kj^cd and t_ialb is t_il^ab (the
paper's t_iajb index order); the six terms of 1/2 P{(ai|bj) t_k^c} are
pairwise equal, giving (ai|bj)t_k^c + (ai|ck)t_j^b + (bj|ck)t_i^a; w of row i
uses Delta_ijk and v of row i' uses Delta_i'jk, so -Delta > 0 is required.

No permutational symmetry is used: every (i, j, k) is computed in full, which
costs 12 o^3 v^4 flops. Use small sizes.
"""
from __future__ import annotations

import numpy as np


def _blocks(B, nocc):
    o, v = slice(0, nocc), slice(nocc, None)
    ovvv = np.einsum("Qia,Qbd->iabd", B[:, o, v], B[:, v, v], optimize=True)   # (ia|bd)
    ovoo = np.einsum("Qkc,Qjl->kcjl", B[:, o, v], B[:, o, o], optimize=True)   # (kc|jl)
    ovov = np.einsum("Qia,Qjb->iajb", B[:, o, v], B[:, o, v], optimize=True)   # (ia|jb)
    return ovvv, ovoo, ovov


def _X(i, j, k, t2, ovvv, ovoo):
    """Un-permuted term X[a,b,c] = sum_d (bd|ai) t_kj^cd - sum_l (ck|jl) t_il^ab."""
    return (np.einsum("abd,cd->abc", ovvv[i], t2[k, j], optimize=True)
            - np.einsum("cl,lab->abc", ovoo[k, :, j, :], t2[i], optimize=True))


def W_block(i, j, k, t2, ovvv, ovoo):
    """W_ijk^abc for all a,b,c: the six permutations of the un-permuted term (SI Sec. S1)."""
    return (_X(i, j, k, t2, ovvv, ovoo)
            + np.einsum("acb->abc", _X(i, k, j, t2, ovvv, ovoo))
            + np.einsum("bac->abc", _X(j, i, k, t2, ovvv, ovoo))
            + np.einsum("bca->abc", _X(j, k, i, t2, ovvv, ovoo))
            + np.einsum("cab->abc", _X(k, i, j, t2, ovvv, ovoo))
            + np.einsum("cba->abc", _X(k, j, i, t2, ovvv, ovoo)))


def V_block(i, j, k, W, t1, ovov):
    """V_ijk^abc = W + (ai|bj) t_k^c + (ai|ck) t_j^b + (bj|ck) t_i^a."""
    return (W + np.einsum("ab,c->abc", ovov[i, :, j, :], t1[k])
            + np.einsum("ac,b->abc", ovov[i, :, k, :], t1[j])
            + np.einsum("bc,a->abc", ovov[j, :, k, :], t1[i]))


def pair_matrix(t1, t2, eps, B, nocc):
    """(T) pair matrix E_ii',(T) (Eq. 16). Its trace is the canonical (T) energy."""
    e = np.asarray(eps, dtype=np.float64)
    if e.ndim == 2:
        e = np.diag(e)
    eo, ev = e[:nocc], e[nocc:]
    ovvv, ovoo, ovov = _blocks(B, nocc)
    o = nocc
    E = np.zeros((o, o))
    evsum = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    for j in range(o):
        for k in range(o):
            z = []
            y = []
            for i in range(o):
                W = W_block(i, j, k, t2, ovvv, ovoo)
                V = V_block(i, j, k, W, t1, ovov)
                s = np.sqrt(-(eo[i] + eo[j] + eo[k] - evsum))
                w = W / s
                vv = V / s
                z.append(4.0 * w + np.einsum("bca->abc", w) + np.einsum("cab->abc", w))
                y.append(vv - np.einsum("cba->abc", vv))
            Z = np.stack(z).reshape(o, -1)
            Y = np.stack(y).reshape(o, -1)
            E += -(Z @ Y.T) / 3.0
    return E


def energy(t1, t2, eps, B, nocc):
    """Canonical (T) correlation energy = trace of the pair matrix (full active space, Sec. II.B)."""
    return float(np.trace(pair_matrix(t1, t2, eps, B, nocc)))
