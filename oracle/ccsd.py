"""ORACLE (test infrastructure only): closed-shell fragment CCSD in FP64 on the CPU.

The paper does not print the CCSD amplitude equations; it solves canonical
CCSD with the fragment Hamiltonian (Sec. II.B, Eq. 10-11). The equations here are
the closed-shell spin-adapted CCSD of the T1-transformed Hamiltonian as given
by Koch, Christiansen, Kobayashi, Jorgensen and Helgaker, Chem. Phys. Lett.
228, 233 (1994) and Helgaker, Jorgensen & Olsen, "Molecular
Electronic-Structure Theory" (Wiley 2000), Sec. 13.7: the T1 amplitudes are
folded into the integrals, after which the doubles equations take the CCD-like
form A2 + B2 + P(C2 + D2 + E2).

Conventions (real orbitals, Sec. II):
  * chemist's notation (pq|rs) = sum_Q B_Qpq B_Qrs (Eq. 27a at the Gamma point);
  * occupied orbitals first; t1[i,a] = t_i^a; t2[i,j,a,b] = t_ij^ab, which is
    the paper's t_iajb (a pairs with i, b with j);
  * tau = t2 + t1 t1 (Eq. 7 prints a minus sign; the plus sign is the one for
    which CCSD equals two-electron FCI, and tests pin it that way);
  * f is the fragment Fock matrix: its diagonal is the orbital energies; a
    full f with zero occupied-virtual block is accepted ("general Fock") so
    that invariance under occupied-occupied and virtual-virtual rotations can
    be tested.
"""
from __future__ import annotations

import numpy as np


def _f_matrix(eps_or_f, n):
    f = np.asarray(eps_or_f, dtype=np.float64)
    return np.diag(f) if f.ndim == 1 else f.copy()


def core_hamiltonian(f, B, nocc):
    """h_pq = f_pq - sum_k [2(pq|kk) - (pk|kq)]: the one-electron part whose HF Fock is f (Eq. 11)."""
    o = slice(0, nocc)
    J = np.einsum("Qpq,Qkk->pq", B, B[:, o, o])
    K = np.einsum("Qpk,Qkq->pq", B[:, :, o], B[:, o, :])
    return f - 2.0 * J + K


def hf_energy(f, B, nocc):
    """E_HF = sum_i (h_ii + f_ii) for a closed-shell determinant."""
    h = core_hamiltonian(f, B, nocc)
    return float(np.trace(h[:nocc, :nocc]) + np.trace(f[:nocc, :nocc]))


def t1_transform(B, t1, nocc):
    """B^ = (1 - T) B (1 + T) for every Q, with T[nocc+a, i] = t_i^a (T1-transformed DF factors)."""
    n = B.shape[1]
    T = np.zeros((n, n))
    T[nocc:, :nocc] = t1.T
    X = np.eye(n) - T
    Y = np.eye(n) + T
    return np.einsum("pr,Qrs,sq->Qpq", X, B, Y, optimize=True)


def t1_fock(h, Bh, t1, nocc):
    """F^_pq = h^_pq + sum_k [2 g^_pqkk - g^_pkkq] with T1-transformed h^ and g^."""
    n = h.shape[0]
    o = slice(0, nocc)
    T = np.zeros((n, n))
    T[nocc:, :nocc] = t1.T
    hh = (np.eye(n) - T) @ h @ (np.eye(n) + T)
    J = np.einsum("Qpq,Qkk->pq", Bh, Bh[:, o, o])
    K = np.einsum("Qpk,Qkq->pq", Bh[:, :, o], Bh[:, o, :])
    return hh + 2.0 * J - K


def mp2_amplitudes(eps, B, nocc):
    """First-order doubles t_ij^ab = (ia|jb) / (e_i + e_j - e_a - e_b) (Eq. 21, canonical orbitals)."""
    e = np.asarray(eps, dtype=np.float64)
    o, v = slice(0, nocc), slice(nocc, None)
    ovov = np.einsum("Qia,Qjb->iajb", B[:, o, v], B[:, o, v])
    eo, ev = e[o], e[v]
    D = eo[:, None, None, None] + eo[None, None, :, None] - ev[None, :, None, None] - ev[None, None, None, :]
    return (ovov / D).transpose(0, 2, 1, 3).copy()


def pair_energy_matrix(t1, t2, B, nocc):
    """Fragment pair matrix E_ii' = sum_jab tau_ij^ab [2(i'a|jb) - (i'b|ja)] (Eq. 9 and Eq. 13)."""
    o, v = slice(0, nocc), slice(nocc, None)
    ovov = np.einsum("Qia,Qjb->iajb", B[:, o, v], B[:, o, v])
    L = 2.0 * ovov - ovov.transpose(0, 3, 2, 1)          # L[i',a,j,b] = 2(i'a|jb) - (i'b|ja)
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1)
    return np.einsum("ijab,kajb->ik", tau, L)


def correlation_energy(t1, t2, B, nocc):
    """E_c = sum_ijab tau_ij^ab [2(ia|jb) - (ib|ja)] (Eq. 7) = trace of the pair matrix."""
    return float(np.trace(pair_energy_matrix(t1, t2, B, nocc)))


def residuals(t1, t2, f, B, nocc, h=None):
    """CCSD residuals Omega_ai (singles) and Omega_aibj (doubles, returned as R[i,j,a,b]).

    T1-transformed closed-shell form (Koch et al. 1994; Helgaker, Jorgensen &
    Olsen Sec. 13.7); g^ = integrals of the T1-transformed DF factors, u_ij^ab =
    2 t_ij^ab - t_ji^ab, L_pqrs = 2 g_pqrs - g_psrq, P X_aibj = X_aibj + X_bjai.
    """
    nocc_, n = nocc, B.shape[1]
    o, v = slice(0, nocc_), slice(nocc_, n)
    if h is None:
        h = core_hamiltonian(f, B, nocc)
    Bh = t1_transform(B, t1, nocc)
    F = t1_fock(h, Bh, t1, nocc)
    u = 2.0 * t2 - t2.transpose(1, 0, 2, 3)

    def g(p, q, r, s):
        return np.einsum("Qpq,Qrs->pqrs", Bh[:, p, q], Bh[:, r, s], optimize=True)

    g_ovov = g(o, v, o, v)             # (kc|ld): undressed, B^_ov = B_ov
    g_vvov = g(v, v, o, v)             # (ad|kc)
    g_ooov = g(o, o, o, v)             # (ki|lc)
    g_vovo = g(v, o, v, o)             # (ai|bj)
    g_oooo = g(o, o, o, o)             # (ki|lj)
    g_oovv = g(o, o, v, v)             # (ki|ac)
    g_voov = g(v, o, o, v)             # (ai|kc)
    g_vvoo = g(v, v, o, o)             # (ac|ki)
    L_ovov = 2.0 * g_ovov - g_ovov.transpose(0, 3, 2, 1)

    # ---- singles: Omega_ai = A1 + B1 + C1 + D1
    O1 = (np.einsum("kicd,adkc->ai", u, g_vvov)
          - np.einsum("klac,kilc->ai", u, g_ooov)
          + np.einsum("ikac,kc->ai", u, F[o, v])
          + F[v, o])

    # ---- doubles
    # A2: g^_aibj + sum_cd t_ij^cd g^_acbd   (particle-particle ladder)
    nv = n - nocc_
    ladder = np.zeros((nocc_, nocc_, nv, nv))
    Bvv = Bh[:, v, v]
    for a in range(nv):
        g_a = np.einsum("Qc,Qbd->cbd", Bvv[:, a, :], Bvv, optimize=True)   # g^_acbd for this a
        ladder[:, :, a, :] = np.einsum("ijcd,cbd->ijb", t2, g_a, optimize=True)
    A2 = g_vovo + ladder.transpose(2, 0, 3, 1)
    # B2: sum_kl t_kl^ab [g^_kilj + sum_cd t_ij^cd g^_kcld]   (hole-hole ladder)
    Woooo = g_oooo + np.einsum("ijcd,kcld->kilj", t2, g_ovov, optimize=True)
    B2 = np.einsum("klab,kilj->aibj", t2, Woooo, optimize=True)
    # C2
    X = g_oovv - 0.5 * np.einsum("liad,kdlc->kiac", t2, g_ovov, optimize=True)
    C2 = (-0.5 * np.einsum("kjbc,kiac->aibj", t2, X, optimize=True)
          - np.einsum("kibc,kjac->aibj", t2, X, optimize=True))
    # D2
    L_voov = 2.0 * g_voov - g_vvoo.transpose(0, 3, 2, 1)   # L^_aikc = 2 g^_aikc - g^_acki
    Y = L_voov + 0.5 * np.einsum("ilad,ldkc->aikc", u, L_ovov, optimize=True)
    D2 = 0.5 * np.einsum("jkbc,aikc->aibj", u, Y, optimize=True)
    # E2
    Fvv = F[v, v] - np.einsum("klbd,ldkc->bc", u, g_ovov, optimize=True)
    Foo = F[o, o] + np.einsum("ljcd,kdlc->kj", u, g_ovov, optimize=True)
    E2 = (np.einsum("ijac,bc->aibj", t2, Fvv, optimize=True)
          - np.einsum("ikab,kj->aibj", t2, Foo, optimize=True))
    S = C2 + D2 + E2
    O2 = A2 + B2 + S + S.transpose(2, 3, 0, 1)
    return O1.T.copy(), O2.transpose(1, 3, 0, 2).copy()


class DIIS:
    """Pulay DIIS (Pulay, Chem. Phys. Lett. 73, 393 (1980)) on the flattened (t1, t2)."""

    def __init__(self, nvec=8):
        self.nvec = nvec
        self.vecs, self.errs = [], []

    def update(self, x, err):
        self.vecs.append(x.copy())
        self.errs.append(err.copy())
        if len(self.vecs) > self.nvec:
            self.vecs.pop(0)
            self.errs.pop(0)
        m = len(self.vecs)
        if m < 2:
            return x
        Bm = np.zeros((m + 1, m + 1))
        Bm[:m, :m] = [[float(ei @ ej) for ej in self.errs] for ei in self.errs]
        Bm[m, :m] = Bm[:m, m] = -1.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.lstsq(Bm, rhs, rcond=None)[0][:m]
        return sum(ci * vi for ci, vi in zip(c, self.vecs))


def ccsd(eps_or_f, B, nocc, *, t1=None, t2=None, max_iter=200, tol_t=1e-10, tol_e=1e-12,
         diis=True, diis_nvec=8, callback=None):
    """Solve the closed-shell CCSD equations by Jacobi updates t += Omega / D (optionally DIIS).

    Starts from the MP2 amplitudes (Eq. 21) unless amplitudes are given.
    Returns dict(e_corr, t1, t2, n_iter, converged, e_mp2, history).
    """
    n = B.shape[1]
    f = _f_matrix(eps_or_f, n)
    e = np.diag(f)
    o, v = slice(0, nocc), slice(nocc, n)
    eo, ev = e[o], e[v]
    D1 = eo[:, None] - ev[None, :]
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    h = core_hamiltonian(f, B, nocc)
    nv = n - nocc
    ovov = np.einsum("Qia,Qjb->iajb", B[:, o, v], B[:, o, v])
    if t2 is None:
        t2 = (ovov.transpose(0, 2, 1, 3) / D2).copy()
    if t1 is None:
        t1 = np.zeros((nocc, nv))
    e_mp2 = correlation_energy(np.zeros_like(t1), ovov.transpose(0, 2, 1, 3) / D2, B, nocc)
    e_old = correlation_energy(t1, t2, B, nocc)
    hist = [e_old]
    dii = DIIS(diis_nvec) if diis else None
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        R1, R2 = residuals(t1, t2, f, B, nocc, h=h)
        d1, d2 = R1 / D1, R2 / D2
        t1n, t2n = t1 + d1, t2 + d2
        if dii is not None:
            x = dii.update(np.concatenate([t1n.ravel(), t2n.ravel()]),
                           np.concatenate([d1.ravel(), d2.ravel()]))
            t1n = x[: t1.size].reshape(t1.shape)
            t2n = x[t1.size:].reshape(t2.shape)
        dt = max(np.abs(d1).max(initial=0.0), np.abs(d2).max(initial=0.0))
        t1, t2 = t1n, t2n
        e_new = correlation_energy(t1, t2, B, nocc)
        hist.append(e_new)
        if callback is not None:
            callback(it, e_new, dt)
        if not np.isfinite(e_new):
            break
        if dt < tol_t and abs(e_new - e_old) < tol_e:
            converged = True
            e_old = e_new
            break
        e_old = e_new
    return dict(e_corr=e_old, t1=t1, t2=t2, n_iter=it, converged=converged, e_mp2=e_mp2,
                history=hist)


def mp2_energy_loops(eps, B, nocc):
    """E_MP2 = sum_ijab (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i+e_j-e_a-e_b), written as explicit loops."""
    e = np.asarray(eps, dtype=np.float64)
    n = B.shape[1]
    tot = 0.0
    for i in range(nocc):
        for j in range(nocc):
            for a in range(nocc, n):
                for b in range(nocc, n):
                    iajb = float(B[:, i, a] @ B[:, j, b])
                    ibja = float(B[:, i, b] @ B[:, j, a])
                    tot += iajb * (2.0 * iajb - ibja) / (e[i] + e[j] - e[a] - e[b])
    return tot
