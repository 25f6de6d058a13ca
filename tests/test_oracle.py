"""Pins of the FP64 CPU oracle against results fixed by the paper and the mathematics.

None of these compares the oracle with itself: each check uses an independent
route (brute-force FCI, the spin-orbital formulation, explicit MP2 loops) or an
exact identity (Eq. 5 and 7 sum rule, orbital-rotation invariance, perturbation
orders, permutational symmetry).
"""
import numpy as np
import pytest

from oracle import ccsd, fci, fragment, spinorb, triples
from paper_2407_11258_gb300 import synth


def _frag(o, v, seed, naux=24, decay=8.0, scale=1.0):
    fr = synth.make_fragment(o, v, naux, seed, occ_range=(-1.0, -0.5), vir_range=(0.2, 2.0), decay=decay)
    fr.B = fr.B * scale
    return fr


# ---------------------------------------------------------------- two-electron FCI

@pytest.mark.parametrize("nvir,seed", [(4, 1), (9, 2), (20, 3)])
def test_ccsd_equals_fci_for_two_electrons(nvir, seed):
    fr = _frag(1, nvir, seed, naux=40, scale=2.0)
    r = ccsd.ccsd(fr.eps, fr.B, 1, tol_t=1e-12, tol_e=1e-14)
    assert r["converged"]
    e_fci, e_hf = fci.fci_2e(fr.eps, fr.B)
    assert abs(ccsd.hf_energy(np.diag(fr.eps), fr.B, 1) - e_hf) < 1e-12
    assert abs(r["e_corr"] - (e_fci - e_hf)) < 1e-10


def test_tau_sign_is_plus():
    """Eq. 7 prints tau = t2 - t1 t1; only + t1 t1 reproduces FCI (planted minus sign must fail)."""
    fr = _frag(1, 9, 5, naux=40, scale=3.0)
    r = ccsd.ccsd(fr.eps, fr.B, 1, tol_t=1e-12, tol_e=1e-14)
    e_fci, e_hf = fci.fci_2e(fr.eps, fr.B)
    o, v = slice(0, 1), slice(1, None)
    ovov = np.einsum("Qia,Qjb->iajb", fr.B[:, o, v], fr.B[:, o, v])
    L = 2 * ovov - ovov.transpose(0, 3, 2, 1)
    tau_minus = r["t2"] - np.einsum("ia,jb->ijab", r["t1"], r["t1"])
    e_minus = float(np.einsum("ijab,iajb->", tau_minus, L))
    assert abs(r["e_corr"] - (e_fci - e_hf)) < 1e-10
    assert abs(e_minus - (e_fci - e_hf)) > 1e-8


@pytest.mark.parametrize("nvir", [5, 12])
def test_triples_vanish_for_two_electrons(nvir):
    fr = _frag(1, nvir, 7, naux=30, scale=2.0)
    r = ccsd.ccsd(fr.eps, fr.B, 1)
    E = triples.pair_matrix(r["t1"], r["t2"], fr.eps, fr.B, 1)
    assert abs(E[0, 0]) < 1e-14


# ------------------------------------------------------ spin-orbital cross-checks

def _to_spin(t1, t2):
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


@pytest.mark.parametrize("o,v,seed", [(2, 4, 11), (3, 3, 12), (2, 5, 13)])
def test_residuals_match_spin_orbital(o, v, seed):
    fr = _frag(o, v, seed)
    rng = np.random.default_rng(seed)
    t1 = 0.05 * rng.normal(size=(o, v))
    t2 = 0.05 * rng.normal(size=(o, o, v, v))
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    R1, R2 = ccsd.residuals(t1, t2, np.diag(fr.eps), fr.B, o)
    fs, g, O = spinorb.spin_integrals(fr.eps, fr.B, o)
    t1s, t2s = _to_spin(t1, t2)
    r1, r2 = spinorb.amplitude_rhs(t1s, t2s, fs, g, O)
    fd = np.diag(fs)
    r1 = r1 - (fd[:O, None] - fd[None, O:]) * t1s
    r2 = r2 - (fd[:O, None, None, None] + fd[None, :O, None, None]
               - fd[None, None, O:, None] - fd[None, None, None, O:]) * t2s
    assert np.abs(R1 - r1[0::2, 0::2]).max() < 1e-13
    assert np.abs(R2 - r2[0::2, 1::2, 0::2, 1::2]).max() < 1e-13


@pytest.mark.parametrize("o,v,seed,scale", [(2, 4, 21, 1.0), (2, 5, 22, 2.0), (3, 4, 23, 2.0)])
def test_ccsd_and_triples_match_spin_orbital(o, v, seed, scale):
    fr = _frag(o, v, seed, naux=20, scale=scale)
    r = ccsd.ccsd(fr.eps, fr.B, o, tol_t=1e-12, tol_e=1e-14)
    E, t1s, t2s, fs, g, O = spinorb.ccsd(fr.eps, fr.B, o)
    assert abs(r["e_corr"] - E) < 1e-10
    et_cs = triples.energy(r["t1"], r["t2"], fr.eps, fr.B, o)
    et_so = spinorb.triples(t1s, t2s, fs, g, O)
    assert abs(et_cs - et_so) < 1e-11
    assert abs(et_cs) > 1e-7


# ------------------------------------------------------------- MP2 at iteration 0

def test_iteration_zero_is_mp2():
    fr = synth.single_fp64()
    r = ccsd.ccsd(fr.eps, fr.B, fr.nocc, max_iter=0)
    e_loops = ccsd.mp2_energy_loops(fr.eps, fr.B, fr.nocc)
    assert abs(r["history"][0] - e_loops) < 1e-14
    assert abs(r["e_mp2"] - e_loops) < 1e-14


# ------------------------------------------------------------- invariances

def _rotation(n, seed):
    return synth.orthogonal(synth.Stream(seed, 9), n)


def test_ccsd_invariant_under_oo_and_vv_rotations():
    o, v = 3, 7
    fr = _frag(o, v, 31, naux=30, scale=1.5)
    ref = ccsd.ccsd(fr.eps, fr.B, o, tol_t=1e-12, tol_e=1e-14)
    R = np.zeros((o + v, o + v))
    R[:o, :o] = _rotation(o, 1)
    R[o:, o:] = _rotation(v, 2)
    f = R @ np.diag(fr.eps) @ R.T
    B = np.einsum("pr,Qrs,qs->Qpq", R, fr.B, R)
    rot = ccsd.ccsd(f, B, o, tol_t=1e-12, tol_e=1e-14)
    assert rot["converged"]
    assert abs(rot["e_corr"] - ref["e_corr"]) < 1e-10
    # a plainly non-covariant step (dropping the off-diagonal Fock) must break it
    bad = ccsd.ccsd(np.diag(np.diag(f)), B, o, tol_t=1e-12, tol_e=1e-14)
    assert abs(bad["e_corr"] - ref["e_corr"]) > 1e-6


def test_amplitude_symmetry():
    fr = synth.single_fp64()
    r = ccsd.ccsd(fr.eps, fr.B, fr.nocc, max_iter=4)
    t2 = r["t2"]
    assert np.abs(t2 - t2.transpose(1, 0, 3, 2)).max() < 1e-15


def test_diis_does_not_move_the_fixed_point():
    fr = synth.single_fp64()
    a = ccsd.ccsd(fr.eps, fr.B, fr.nocc, diis=True)
    b = ccsd.ccsd(fr.eps, fr.B, fr.nocc, diis=False)
    assert a["converged"] and b["converged"]
    assert abs(a["e_corr"] - b["e_corr"]) < 1e-10


# ------------------------------------------------------------- projector (Eq. 5-16)

def test_fragment_energies_sum_to_total():
    fr = synth.single_fp64()
    r = ccsd.ccsd(fr.eps, fr.B, fr.nocc)
    Ec = ccsd.pair_energy_matrix(r["t1"], r["t2"], fr.B, fr.nocc)
    Et = triples.pair_matrix(r["t1"], r["t2"], fr.eps, fr.B, fr.nocc)
    U = fr.U
    for E in (Ec, Et):
        parts = [fragment.project(E, U[:, a]) for a in range(fr.nocc)]
        assert abs(sum(parts) - np.trace(E)) < 1e-14
        assert abs(fragment.project(E, np.eye(fr.nocc)[:, 0]) - E[0, 0]) < 1e-16
    assert abs(np.trace(Ec) - r["e_corr"]) < 1e-14
    # rotating the LOs inside a two-LO fragment leaves its energy unchanged
    c, s = np.cos(0.7), np.sin(0.7)
    U2 = U[:, :2] @ np.array([[c, -s], [s, c]])
    assert abs(fragment.project(Et, U2) - fragment.project(Et, U[:, :2])) < 1e-15


def test_projected_triples_with_identity_is_canonical():
    fr = _frag(3, 5, 41, naux=20, scale=2.0)
    r = ccsd.ccsd(fr.eps, fr.B, 3)
    E = triples.pair_matrix(r["t1"], r["t2"], fr.eps, fr.B, 3)
    E_so, t1s, t2s, fs, g, O = spinorb.ccsd(fr.eps, fr.B, 3)
    assert abs(fragment.project(E, np.eye(3)) - spinorb.triples(t1s, t2s, fs, g, O)) < 1e-11


# ------------------------------------------------------------- weak-coupling orders

def test_weak_coupling_orders():
    fr = _frag(2, 5, 51, naux=20)
    res = {}
    for lam in (0.05, 0.1):
        B = fr.B * lam
        r = ccsd.ccsd(fr.eps, B, 2, tol_t=1e-14, tol_e=1e-16)
        res[lam] = (r["e_corr"], r["e_mp2"], triples.energy(r["t1"], r["t2"], fr.eps, B, 2))
    # E_CCSD / E_MP2 -> 1; the first correction is third order in V (~lambda^6 against
    # lambda^4 for MP2), so the relative deviation scales as lambda^2
    d1 = res[0.1][0] / res[0.1][1] - 1.0
    d0 = res[0.05][0] / res[0.05][1] - 1.0
    assert abs(d0) < abs(d1) and 3.6 < d1 / d0 < 4.4
    # E_(T) ~ lambda^8 at leading order
    ratio = res[0.1][2] / res[0.05][2]
    assert 230 < ratio < 270
