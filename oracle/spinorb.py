"""ORACLE (test infrastructure only): spin-orbital CCSD and (T) for tiny cross-checks.

An independent route to the same energies as `ccsd` / `triples`, used only to
pin the closed-shell spin-adapted forms (which the paper does not print,
Sec. II.B). Written from:
  * CCSD: Stanton, Gauss, Watts & Bartlett, J. Chem. Phys. 94, 4334 (1991),
    the F/W-intermediate spin-orbital formulation;
  * (T): Raghavachari, Trucks, Pople & Head-Gordon, Chem. Phys. Lett. 157, 479
    (1989), in the connected/disconnected spin-orbital form of Crawford &
    Schaefer, Rev. Comp. Chem. 14, 33 (2000).
Spin orbitals are spatial orbitals times {alpha, beta}; antisymmetrised
integrals <pq||rs> = <pq|rs> - <pq|sr> with <pq|rs> = (pr|qs) delta_spin.
Sizes: a handful of spatial orbitals (the arrays are (2n)^4).
"""
from __future__ import annotations

import numpy as np


def spin_integrals(f, B, nocc):
    """Return (fs, g, O) with fs the spin-orbital Fock, g = <pq||rs>, O = number of occupied spin orbitals."""
    n = B.shape[1]
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 1:
        f = np.diag(f)
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)             # (pq|rs)
    ns = 2 * n
    spat = np.arange(ns) // 2
    spin = np.arange(ns) % 2
    fs = f[np.ix_(spat, spat)] * (spin[:, None] == spin[None, :])
    # <pq|rs> = (pr|qs) d(sp,sr) d(sq,ss)
    phys = eri[np.ix_(spat, spat, spat, spat)].transpose(0, 2, 1, 3)
    same_pr = spin[:, None, None, None] == spin[None, None, :, None]
    same_qs = spin[None, :, None, None] == spin[None, None, None, :]
    phys = phys * (same_pr & same_qs)
    g = phys - phys.transpose(0, 1, 3, 2)
    return fs, g, 2 * nocc


def ccsd(f, B, nocc, max_iter=300, tol=1e-12):
    """Spin-orbital CCSD (Stanton et al. 1991). Returns (E_corr, t1, t2, fs, g, O)."""
    fs, g, O = spin_integrals(f, B, nocc)
    ns = fs.shape[0]
    o, v = slice(0, O), slice(O, ns)
    fd = np.diag(fs)
    Dia = fd[o, None] - fd[None, v]
    Dijab = fd[o, None, None, None] + fd[None, o, None, None] - fd[None, None, v, None] - fd[None, None, None, v]
    t1 = np.zeros((O, ns - O))
    t2 = g[o, o, v, v] / Dijab
    fov = fs[o, v]

    def energy(t1, t2):
        return (np.einsum("ia,ia->", fov, t1) + 0.25 * np.einsum("ijab,ijab->", g[o, o, v, v], t2)
                + 0.5 * np.einsum("ijab,ia,jb->", g[o, o, v, v], t1, t1))

    E = energy(t1, t2)
    hist_x, hist_e = [], []
    for _ in range(max_iter):
        r1, r2 = amplitude_rhs(t1, t2, fs, g, O)
        t1n, t2n = r1 / Dia, r2 / Dijab
        d = max(np.abs(t1n - t1).max(initial=0.0), np.abs(t2n - t2).max())
        # Pulay extrapolation over the last 6 iterates (keeps strongly coupled cases convergent)
        hist_x.append(np.concatenate([t1n.ravel(), t2n.ravel()]))
        hist_e.append(np.concatenate([(t1n - t1).ravel(), (t2n - t2).ravel()]))
        hist_x, hist_e = hist_x[-6:], hist_e[-6:]
        m = len(hist_x)
        if m > 1:
            A = np.zeros((m + 1, m + 1))
            A[:m, :m] = np.array(hist_e) @ np.array(hist_e).T
            A[m, :m] = A[:m, m] = -1.0
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.lstsq(A, rhs, rcond=None)[0][:m]
            x = c @ np.array(hist_x)
            t1n, t2n = x[: t1.size].reshape(t1.shape), x[t1.size:].reshape(t2.shape)
        En = energy(t1n, t2n)
        t1, t2 = t1n, t2n
        if d < tol and abs(En - E) < tol:
            E = En
            break
        E = En
    return float(E), t1, t2, fs, g, O


def amplitude_rhs(t1, t2, fs, g, O):
    """Right-hand sides of the Stanton et al. (1991) T1 and T2 equations (t D = rhs)."""
    ns = fs.shape[0]
    o, v = slice(0, O), slice(O, ns)
    fov = fs[o, v]
    foo_off = fs[o, o] - np.diag(np.diag(fs[o, o]))
    fvv_off = fs[v, v] - np.diag(np.diag(fs[v, v]))
    tau_t = t2 + 0.5 * (np.einsum("ia,jb->ijab", t1, t1) - np.einsum("ib,ja->ijab", t1, t1))
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1) - np.einsum("ib,ja->ijab", t1, t1)
    Fae = (fvv_off - 0.5 * np.einsum("me,ma->ae", fov, t1)
           + np.einsum("mf,mafe->ae", t1, g[o, v, v, v])
           - 0.5 * np.einsum("mnaf,mnef->ae", tau_t, g[o, o, v, v]))
    Fmi = (foo_off + 0.5 * np.einsum("ie,me->mi", t1, fov)
           + np.einsum("ne,mnie->mi", t1, g[o, o, o, v])
           + 0.5 * np.einsum("inef,mnef->mi", tau_t, g[o, o, v, v]))
    Fme = fov + np.einsum("nf,mnef->me", t1, g[o, o, v, v])
    X = np.einsum("je,mnie->mnij", t1, g[o, o, o, v])
    Wmnij = g[o, o, o, o] + X - X.transpose(0, 1, 3, 2) + 0.25 * np.einsum("ijef,mnef->mnij", tau, g[o, o, v, v])
    Y = np.einsum("mb,amef->abef", t1, g[v, o, v, v])
    Wabef = g[v, v, v, v] - Y + Y.transpose(1, 0, 2, 3) + 0.25 * np.einsum("mnab,mnef->abef", tau, g[o, o, v, v])
    Wmbej = (g[o, v, v, o] + np.einsum("jf,mbef->mbej", t1, g[o, v, v, v])
             - np.einsum("nb,mnej->mbej", t1, g[o, o, v, o])
             - np.einsum("jnfb,mnef->mbej", 0.5 * t2 + np.einsum("jf,nb->jnfb", t1, t1), g[o, o, v, v]))
    # T1 equation
    r1 = (fov + np.einsum("ie,ae->ia", t1, Fae) - np.einsum("ma,mi->ia", t1, Fmi)
          + np.einsum("imae,me->ia", t2, Fme) - np.einsum("nf,naif->ia", t1, g[o, v, o, v])
          - 0.5 * np.einsum("imef,maef->ia", t2, g[o, v, v, v])
          - 0.5 * np.einsum("mnae,nmei->ia", t2, g[o, o, v, o]))
    # T2 equation
    Fbe = Fae - 0.5 * np.einsum("mb,me->be", t1, Fme)
    Fmj = Fmi + 0.5 * np.einsum("je,me->mj", t1, Fme)
    A = np.einsum("ijae,be->ijab", t2, Fbe)
    Bm = np.einsum("imab,mj->ijab", t2, Fmj)
    C = np.einsum("imae,mbej->ijab", t2, Wmbej) - np.einsum("ie,ma,mbej->ijab", t1, t1, g[o, v, v, o])
    Dt = np.einsum("ie,abej->ijab", t1, g[v, v, v, o])
    Et = np.einsum("ma,mbij->ijab", t1, g[o, v, o, o])
    r2 = (g[o, o, v, v] + A - A.transpose(0, 1, 3, 2) - Bm + Bm.transpose(1, 0, 2, 3)
          + 0.5 * np.einsum("mnab,mnij->ijab", tau, Wmnij)
          + 0.5 * np.einsum("ijef,abef->ijab", tau, Wabef)
          + C - C.transpose(1, 0, 2, 3) - C.transpose(0, 1, 3, 2) + C.transpose(1, 0, 3, 2)
          + Dt - Dt.transpose(1, 0, 2, 3) - Et + Et.transpose(0, 1, 3, 2))
    return r1, r2


def triples(t1, t2, fs, g, O):
    """Spin-orbital (T) energy: E = 1/36 sum t(c) D (t(c) + t(d)) (Raghavachari et al. 1989)."""
    ns = fs.shape[0]
    o, v = slice(0, O), slice(O, ns)
    fd = np.diag(fs)
    eo, ev = fd[o], fd[v]
    D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
         + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
         - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
    # x_ijkabc = sum_e t_jk^ae <ei||bc> - sum_m t_im^bc <ma||jk>
    x = np.einsum("jkae,eibc->ijkabc", t2, g[v, o, v, v]) - np.einsum("imbc,majk->ijkabc", t2, g[o, v, o, o])
    y = np.einsum("ia,jkbc->ijkabc", t1, g[o, o, v, v])

    def Pijk(t):      # P(i/jk) f(ijk) = f(ijk) - f(jik) - f(kji)
        return t - t.transpose(1, 0, 2, 3, 4, 5) - t.transpose(2, 1, 0, 3, 4, 5)

    def Pabc(t):
        return t - t.transpose(0, 1, 2, 4, 3, 5) - t.transpose(0, 1, 2, 5, 4, 3)

    tc = Pijk(Pabc(x)) / D
    td = Pijk(Pabc(y)) / D
    return float(np.einsum("ijkabc,ijkabc->", tc * D, tc + td) / 36.0)


def pair_energy_matrix(t1s, t2s, g, O):
    """Occupied pair matrix of the spin-orbital CCSD energy, summed over spin to spatial indices.

    The spin-orbital correlation energy 1/4 sum_IJAB <IJ||AB> tau_IJ^AB (Stanton et al. 1991, f_ov = 0)
    is split by the occupied index I of tau and the index I' that replaces it on the integral:
    E_II' = 1/4 sum_JAB <I'J||AB> tau_IJ^AB, tau_IJ^AB = t_IJ^AB + t_I^A t_J^B - t_I^B t_J^A. Spin
    orbitals 2p (alpha) and 2p+1 (beta) belong to spatial orbital p; the returned spatial matrix sums
    both spins of i and of i'. Its trace is the spin-orbital CCSD energy. This is an independent route
    (antisymmetrised spin-orbital integrals) to the closed-shell pair matrix of Eq. 9 and Eq. 13.
    """
    o, v = slice(0, O), slice(O, g.shape[0])
    tau = t2s + np.einsum("ia,jb->ijab", t1s, t1s) - np.einsum("ib,ja->ijab", t1s, t1s)
    E = 0.25 * np.einsum("kjab,ijab->ik", g[o, o, v, v], tau)
    return E[0::2, 0::2] + E[0::2, 1::2] + E[1::2, 0::2] + E[1::2, 1::2]


def to_spin_amplitudes(t1, t2):
    """Closed-shell t1[i,a], t2[i,j,a,b] = t_ij^ab to spin-orbital t1s, antisymmetric t2s (spin orbital
    2p + s for spatial p, spin s): t_IJ^AB = t_ij^ab d(s_I,s_A) d(s_J,s_B) - t_ij^ba d(s_I,s_B) d(s_J,s_A)."""
    o, v = t1.shape
    t1s = np.zeros((2 * o, 2 * v))
    t2s = np.zeros((2 * o, 2 * o, 2 * v, 2 * v))
    for s in range(2):
        t1s[s::2, s::2] = t1
    for si in range(2):
        for sj in range(2):
            t2s[si::2, sj::2, si::2, sj::2] += t2
            t2s[si::2, sj::2, sj::2, si::2] -= t2.transpose(0, 1, 3, 2)
    return t1s, t2s


def restricted_mp2_densities(eps, B, nocc, W_occ=None, f_occ=None, W_vir=None, f_vir=None):
    """Spin-orbital first-order amplitudes t_IJ^AB = <IJ||AB> / (f_I + f_J - f_A - f_B) in a basis where
    the occupied (virtual) orbitals are the columns of W_occ (W_vir) followed by the canonical ones, and
    the MP2 density blocks with occupied / virtual indices restricted to those columns:
      D_AB(one internal occupied) = sum_{I int} sum_{J C} t_IJ^AC t_IJ^BC,
      D_IJ(one internal occupied) = sum_{K int} sum_{A B} t_IK^AB t_JK^AB,
      D_AB(both occupied internal) = sum_{I J int} sum_C t_IJ^AC t_IJ^BC,
      D_IJ(both virtuals internal) = sum_K sum_{A B int} t_IK^AB t_JK^AB,
    each summed over spin onto spatial indices (canonical orbitals only; the internal columns act as the
    restricted index). Returns a dict of those four spatial matrices; an independent route to the
    closed-shell densities of the local active space (Sec. II.C and II.E)."""
    e = np.asarray(eps, dtype=np.float64)
    n = B.shape[1]
    nvir = n - nocc
    Bo = np.asarray(B[:, :nocc, nocc:], dtype=np.float64)
    eo, ev = e[:nocc], e[nocc:]
    Wo = np.zeros((nocc, 0)) if W_occ is None else np.asarray(W_occ)
    Wv = np.zeros((nvir, 0)) if W_vir is None else np.asarray(W_vir)
    fo = np.zeros(0) if f_occ is None else np.asarray(f_occ)
    fv = np.zeros(0) if f_vir is None else np.asarray(f_vir)
    no, nv = Wo.shape[1], Wv.shape[1]
    # extended spatial occupied basis [internal | canonical], virtual [internal | canonical]
    Co = np.concatenate([Wo, np.eye(nocc)], axis=1)
    Cv = np.concatenate([Wv, np.eye(nvir)], axis=1)
    Lov = np.einsum("Qia,iI,aA->QIA", Bo, Co, Cv)
    eO = np.concatenate([fo, eo])
    eV = np.concatenate([fv, ev])
    ovov = np.einsum("QIA,QJB->IAJB", Lov, Lov)       # (IA|JB), spatial
    mo, mv = eO.size, eV.size
    # spin orbitals: 2p + s
    spat_o, spin_o = np.arange(2 * mo) // 2, np.arange(2 * mo) % 2
    spat_v, spin_v = np.arange(2 * mv) // 2, np.arange(2 * mv) % 2
    # <IJ|AB> = (IA|JB) d(sI,sA) d(sJ,sB)
    phys = ovov[np.ix_(spat_o, spat_v, spat_o, spat_v)].transpose(0, 2, 1, 3)
    same = ((spin_o[:, None, None, None] == spin_v[None, None, :, None])
            & (spin_o[None, :, None, None] == spin_v[None, None, None, :]))
    g = phys * same
    g = g - g.transpose(0, 1, 3, 2)
    eOs, eVs = eO[spat_o], eV[spat_v]
    t = g / (eOs[:, None, None, None] + eOs[None, :, None, None] - eVs[None, None, :, None] - eVs[None, None, None, :])
    io = np.arange(2 * no)                 # internal occupied spin orbitals
    co = np.arange(2 * no, 2 * mo)         # canonical occupied
    iv = np.arange(2 * nv)
    cv = np.arange(2 * nv, 2 * mv)

    def spatial(M, nrow):
        return M[0::2, 0::2][:nrow, :nrow] + M[1::2, 1::2][:nrow, :nrow]

    out = {}
    if no:
        tt = t[np.ix_(io, co, cv, cv)]
        out["vir_one_int_occ"] = spatial(np.einsum("IJac,IJbc->ab", tt, tt), nvir)
        tt = t[np.ix_(co, io, cv, cv)]
        out["occ_one_int_occ"] = spatial(np.einsum("iKab,jKab->ij", tt, tt), nocc)
        tt = t[np.ix_(io, io, cv, cv)]
        out["vir_two_int_occ"] = spatial(np.einsum("IJac,IJbc->ab", tt, tt), nvir)
    if nv:
        tt = t[np.ix_(co, co, iv, iv)]
        out["occ_two_int_vir"] = spatial(np.einsum("iKAB,jKAB->ij", tt, tt), nocc)
    return out
