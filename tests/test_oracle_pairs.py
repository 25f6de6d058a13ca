"""Pins of the oracle's occupied pair matrices element by element, off-diagonal elements included.

A fragment energy E^(F) = sum_alpha sum_ii' U_i,alpha E_ii' U_i',alpha (Eq. 12, Eq. 15) reads every
element of the pair matrix once U is not the identity, while the total energy (the trace) only reads
the diagonal. The pins here fix the off-diagonal elements:

* CCSD (Eq. 9, Eq. 13): the spin-orbital pair matrix 1/4 sum_JAB <I'J||AB> tau_IJ^AB, summed over spin,
  equals the closed-shell matrix element by element (an independent formulation: antisymmetrised
  spin-orbital integrals and amplitudes), at random amplitudes and at converged ones; and the matrix is
  covariant under an occupied rotation R solved from scratch in the rotated basis (general-Fock mode):
  E -> R E R^T, fragment energies unchanged with U -> R U.
* (T) (Eq. 16 with the intermediates of SI Sec. S1): the closed-shell partition by i is not the
  spin-orbital one (only the traces agree, checked below), so the pins are properties of the definition:
  covariance under rotations inside an exactly degenerate occupied block (the Fock matrix stays
  diagonal and Delta is constant over the block), and the decay of E_ii' when e_i' is pushed down by
  lambda with the amplitudes held fixed: v_i'jk carries 1/sqrt(-Delta_i'jk), so E_ii' (i != i') falls
  as lambda^(-1/2) and E_i'i' as lambda^(-1).
* Each pin is shown to fail on a planted mistake of the kind it guards against.
"""
import numpy as np
import pytest

from oracle import ccsd, fragment, spinorb, triples
from paper_2407_11258_gb300 import synth


def _frag(o, v, seed, naux=24, decay=8.0, scale=1.0):
    fr = synth.make_fragment(o, v, naux, seed, occ_range=(-1.0, -0.5), vir_range=(0.2, 2.0), decay=decay)
    fr.B = fr.B * scale
    return fr


def _random_amplitudes(o, v, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    t1 = scale * rng.normal(size=(o, v))
    t2 = scale * rng.normal(size=(o, o, v, v))
    return t1, 0.5 * (t2 + t2.transpose(1, 0, 3, 2))


def _rotation(n, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def _spin_pair_matrix(t1, t2, eps, B, o):
    fs, g, O = spinorb.spin_integrals(eps, B, o)
    t1s, t2s = spinorb.to_spin_amplitudes(t1, t2)
    return spinorb.pair_energy_matrix(t1s, t2s, g, O)


# ------------------------------------------------------------------------------------- CCSD

@pytest.mark.parametrize("o,v,seed", [(2, 4, 1), (3, 5, 2), (4, 3, 3)])
def test_ccsd_pair_matrix_equals_spin_orbital_at_random_amplitudes(o, v, seed):
    fr = _frag(o, v, 100 + seed)
    t1, t2 = _random_amplitudes(o, v, seed)
    E = ccsd.pair_energy_matrix(t1, t2, fr.B, o)
    Es = _spin_pair_matrix(t1, t2, fr.eps, fr.B, o)
    assert np.abs(E - Es).max() < 1e-15 * max(1.0, np.abs(E).max()) * 10
    assert np.abs(E - np.diag(np.diag(E))).max() > 1e-4  # the off-diagonal elements are not trivially 0


def test_ccsd_pair_matrix_equals_spin_orbital_at_convergence():
    o, v = 3, 5
    fr = _frag(o, v, 7, naux=30, scale=1.5)
    r = ccsd.ccsd(fr.eps, fr.B, o, tol_t=1e-12, tol_e=1e-14)
    E = ccsd.pair_energy_matrix(r["t1"], r["t2"], fr.B, o)
    Es = _spin_pair_matrix(r["t1"], r["t2"], fr.eps, fr.B, o)
    assert np.abs(E - Es).max() < 1e-15
    # and the spin-orbital solve's own amplitudes give the same matrix (independent CCSD as well)
    E_so, t1s, t2s, fs, g, O = spinorb.ccsd(fr.eps, fr.B, o)
    assert np.abs(spinorb.pair_energy_matrix(t1s, t2s, g, O) - E).max() < 1e-10


@pytest.mark.parametrize("mistake", ["exchange_index", "tau_sign", "transpose_t2"])
def test_spin_orbital_pin_catches_planted_ccsd_mistakes(mistake):
    o, v = 3, 4
    fr = _frag(o, v, 11)
    t1, t2 = _random_amplitudes(o, v, 12)
    t2 = t2 + 0.02 * np.random.default_rng(13).normal(size=t2.shape)  # break t_ij^ab = t_ji^ba: guards transposes
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    ovov = np.einsum("Qia,Qjb->iajb", fr.B[:, :o, o:], fr.B[:, :o, o:])
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1)
    if mistake == "exchange_index":       # (ib|ja) taken with the row index i instead of i'
        L2 = 2.0 * ovov
        bad = np.einsum("ijab,kajb->ik", tau, L2) - np.einsum("ijab,ibja->i", tau, ovov)[:, None]
    elif mistake == "tau_sign":
        taum = t2 - np.einsum("ia,jb->ijab", t1, t1)
        bad = np.einsum("ijab,kajb->ik", taum, 2.0 * ovov - ovov.transpose(0, 3, 2, 1))
    else:                                  # t_ij^ab read as t_ij^ba
        taut = t2.transpose(0, 1, 3, 2) + np.einsum("ia,jb->ijab", t1, t1)
        bad = np.einsum("ijab,kajb->ik", taut, 2.0 * ovov - ovov.transpose(0, 3, 2, 1))
    Es = _spin_pair_matrix(t1, t2, fr.eps, fr.B, o)
    assert np.abs(bad - Es).max() > 1e-6


def test_ccsd_pair_matrix_covariant_under_occupied_rotation():
    """Occupied orbitals rotated by a random orthogonal R (f no longer diagonal: general-Fock mode),
    CCSD solved from scratch: the pair matrix becomes R E R^T and every LO's fragment energy is
    unchanged when U becomes R U."""
    o, v = 3, 6
    fr = _frag(o, v, 21, naux=30, scale=1.5)
    ref = ccsd.ccsd(fr.eps, fr.B, o, tol_t=1e-12, tol_e=1e-14)
    E = ccsd.pair_energy_matrix(ref["t1"], ref["t2"], fr.B, o)
    R = np.eye(o + v)
    R[:o, :o] = _rotation(o, 22)
    f = R @ np.diag(fr.eps) @ R.T
    B = np.einsum("pr,Qrs,qs->Qpq", R, fr.B, R)
    rot = ccsd.ccsd(f, B, o, tol_t=1e-12, tol_e=1e-14)
    assert rot["converged"]
    Er = ccsd.pair_energy_matrix(rot["t1"], rot["t2"], B, o)
    Ro = R[:o, :o]
    assert np.abs(Er - Ro @ E @ Ro.T).max() < 1e-10
    for a in range(o):
        assert abs(fragment.project(Er, Ro @ fr.U[:, a]) - fragment.project(E, fr.U[:, a])) < 1e-10


# ------------------------------------------------------------------------------------- (T)

def _solve(eps, B, o):
    r = ccsd.ccsd(eps, B, o, tol_t=1e-12, tol_e=1e-14)
    assert r["converged"]
    return r["t1"], r["t2"]


def test_triples_closed_shell_partition_differs_from_spin_orbital_but_trace_agrees():
    """Why the (T) pins are properties: partitioning the spin-orbital (T) energy by its first occupied
    index gives another matrix with the same trace, so no independent formulation fixes the elements."""
    o, v = 3, 4
    fr = _frag(o, v, 23, naux=20, scale=2.0)
    t1, t2 = _solve(fr.eps, fr.B, o)
    Et = triples.pair_matrix(t1, t2, fr.eps, fr.B, o)
    fs, g, O = spinorb.spin_integrals(fr.eps, fr.B, o)
    t1s, t2s = spinorb.to_spin_amplitudes(t1, t2)
    assert abs(np.trace(Et) - spinorb.triples(t1s, t2s, fs, g, O)) < 1e-12
    assert np.abs(np.diag(Et)).min() > 1e-5


def _degenerate_case(o=3, v=5, seed=31):
    fr = _frag(o, v, seed, naux=24, scale=2.0)
    fr.eps[1] = fr.eps[0]  # occupied orbitals 0 and 1 exactly degenerate
    return fr


def _rotate_block(fr, theta=0.7):
    R = np.eye(fr.nmo)
    c, s = np.cos(theta), np.sin(theta)
    R[:2, :2] = [[c, -s], [s, c]]
    return R, np.einsum("pr,Qrs,qs->Qpq", R, fr.B, R)


def test_triples_pair_matrix_covariant_in_degenerate_occupied_block():
    o = 3
    fr = _degenerate_case(o)
    t1, t2 = _solve(fr.eps, fr.B, o)
    Et = triples.pair_matrix(t1, t2, fr.eps, fr.B, o)
    R, Br = _rotate_block(fr)
    t1r, t2r = _solve(fr.eps, Br, o)  # the Fock matrix stays diagonal: the rotation is inside a degenerate block
    Etr = triples.pair_matrix(t1r, t2r, fr.eps, Br, o)
    Ro = R[:o, :o]
    assert np.abs(Etr - Ro @ Et @ Ro.T).max() < 1e-11
    assert np.abs(Et[0, 1]) > 1e-6 and np.abs(Et[0, 2]) > 1e-6  # off-diagonal elements are exercised
    for a in range(o):
        u = fr.U[:, a]
        assert abs(fragment.project(Etr, Ro @ u) - fragment.project(Et, u)) < 1e-11


def _pair_matrix_v_on_wrong_index(t1, t2, eps, B, nocc):
    """Planted mistake: the disconnected part of V for row i' built from the integrals of row i."""
    e = np.asarray(eps, dtype=np.float64)
    eo, ev = e[:nocc], e[nocc:]
    ovvv, ovoo, ovov = triples._blocks(B, nocc)
    evsum = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    o = nocc
    E = np.zeros((o, o))
    for j in range(o):
        for k in range(o):
            Ws = [triples.W_block(i, j, k, t2, ovvv, ovoo) for i in range(o)]
            for i in range(o):
                s_i = np.sqrt(-(eo[i] + eo[j] + eo[k] - evsum))
                w = Ws[i] / s_i
                z = 4.0 * w + np.einsum("bca->abc", w) + np.einsum("cab->abc", w)
                for ip in range(o):
                    V = (Ws[ip] + np.einsum("ab,c->abc", ovov[i, :, j, :], t1[k])
                         + np.einsum("ac,b->abc", ovov[i, :, k, :], t1[j])
                         + np.einsum("bc,a->abc", ovov[j, :, k, :], t1[ip]))
                    vv = V / np.sqrt(-(eo[ip] + eo[j] + eo[k] - evsum))
                    E[i, ip] += -float(np.sum(z * (vv - np.einsum("cba->abc", vv)))) / 3.0
    return E


def test_degenerate_covariance_catches_planted_integral_index_mistake():
    o = 3
    fr = _degenerate_case(o)
    t1, t2 = _solve(fr.eps, fr.B, o)
    R, Br = _rotate_block(fr)
    t1r, t2r = _solve(fr.eps, Br, o)
    Ro = R[:o, :o]
    bad = _pair_matrix_v_on_wrong_index(t1, t2, fr.eps, fr.B, o)
    badr = _pair_matrix_v_on_wrong_index(t1r, t2r, fr.eps, Br, o)
    assert np.abs(badr - Ro @ bad @ Ro.T).max() > 1e-7
    # the same function with the correct index reproduces the oracle (the planted change is the only one)
    good = triples.pair_matrix(t1, t2, fr.eps, fr.B, o)
    assert np.abs(np.trace(bad) - np.trace(good)) < 1e-14


def _pair_matrix_v_with_row_denominator(t1, t2, eps, B, nocc):
    """Planted mistake: v_i'jk divided by sqrt(-Delta_ijk) (the row's denominator) instead of Delta_i'jk."""
    e = np.asarray(eps, dtype=np.float64)
    eo, ev = e[:nocc], e[nocc:]
    ovvv, ovoo, ovov = triples._blocks(B, nocc)
    evsum = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    o = nocc
    E = np.zeros((o, o))
    for j in range(o):
        for k in range(o):
            Ws = [triples.W_block(i, j, k, t2, ovvv, ovoo) for i in range(o)]
            Vs = [triples.V_block(i, j, k, Ws[i], t1, ovov) for i in range(o)]
            for i in range(o):
                s_i = np.sqrt(-(eo[i] + eo[j] + eo[k] - evsum))
                w = Ws[i] / s_i
                z = 4.0 * w + np.einsum("bca->abc", w) + np.einsum("cab->abc", w)
                for ip in range(o):
                    vv = Vs[ip] / s_i
                    E[i, ip] += -float(np.sum(z * (vv - np.einsum("cba->abc", vv)))) / 3.0
    return E


def _shifted(fr, lam):
    e = fr.eps.copy()
    e[1] -= lam  # occupied orbital 1 pushed down; the amplitudes are held fixed
    return e


@pytest.mark.parametrize("planted", [False, True])
def test_triples_off_diagonal_decay_fixes_the_v_denominator(planted):
    """With t1, t2 and B fixed, E_01 ~ C lambda^(-1/2) and E_11 ~ C' lambda^(-1) as e_1 -> e_1 - lambda
    (Delta_1jk grows like lambda). Dividing v_1jk by the row's Delta_0jk instead leaves E_01 finite."""
    o = 3
    fr = _frag(o, 4, 41, naux=20, scale=2.0)
    t1, t2 = _solve(fr.eps, fr.B, o)
    fn = _pair_matrix_v_with_row_denominator if planted else triples.pair_matrix
    E1 = fn(t1, t2, _shifted(fr, 1e4), fr.B, o)
    E4 = fn(t1, t2, _shifted(fr, 4e4), fr.B, o)
    r01 = E1[0, 1] / E4[0, 1]
    r11 = E1[1, 1] / E4[1, 1]
    if planted:
        assert abs(r01 - 1.0) < 0.05  # the planted form does not decay: the pin below must reject it
        assert not abs(r01 - 2.0) < 0.02
    else:
        assert abs(r01 - 2.0) < 0.02
        assert abs(r11 - 4.0) < 0.05
        # E_10 has z from the shifted row (w_1jk ~ lambda^(-1/2)) and y from row 0: also lambda^(-1/2)
        assert abs(E1[1, 0] / E4[1, 0] - 2.0) < 0.02
