"""Pins of the local-active-space oracle (oracle/lno.py, Sec. II.C and II.E, Eq. 18-26 and Eq. 28).

* The closed-shell LNO densities (Eq. 20) and CBNO densities (Eq. 28) equal one half of the spin-orbital
  MP2 density blocks with the same occupied / virtual indices restricted to the internal space, element
  by element (an independent formulation: antisymmetrised spin-orbital amplitudes), for rotated,
  semi-canonical internal orbitals.
* Particle-number conservation of the MP2 density: tr D_occ = tr D_vir for any fragment (Eq. 20).
* Both blocks are positive semidefinite (each is a sum of Gram matrices).
* Basis independence: rotating the LOs inside a fragment (U -> U R) leaves the densities and the LNO
  eigenvalues unchanged; building the amplitudes without the semi-canonical step (a planted mistake)
  breaks it, because orthonormal LO columns make every singular value of Eq. 18 equal to one.
* The LNOs of Eq. 24-26 are orthonormal, orthogonal to the internal space, and their eigen-expansion
  rebuilds the projected density; fewer survive a larger threshold.
"""
import numpy as np
import pytest

from oracle import lno, spinorb
from paper_2407_11258_gb300 import synth


def _system(o, v, seed, naux=30):
    fr = synth.make_fragment(o, v, naux, seed, occ_range=(-1.0, -0.4), vir_range=(0.2, 2.5), decay=8.0)
    return fr, np.ascontiguousarray(fr.B[:, :o, o:])


def _orthonormal_cols(n, k, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return (q * np.sign(np.diag(r)))[:, :k]


@pytest.mark.parametrize("o,v,nlo,seed", [(4, 6, 1, 1), (5, 7, 2, 2), (4, 5, 3, 3)])
def test_lno_densities_are_half_the_spin_orbital_blocks(o, v, nlo, seed):
    fr, Bov = _system(o, v, seed)
    U = fr.U[:, :nlo]
    W, f, _ = lno.internal_space(U, fr.eps[:o])
    D_occ, D_vir = lno.lno_densities(fr.eps, Bov, o, U)
    so = spinorb.restricted_mp2_densities(fr.eps, fr.B, o, W_occ=W, f_occ=f)
    assert np.abs(D_vir - 0.5 * so["vir_one_int_occ"]).max() < 1e-15
    assert np.abs(D_occ - 0.5 * so["occ_one_int_occ"]).max() < 1e-15
    assert np.abs(D_vir).max() > 1e-6 and np.abs(D_occ - np.diag(np.diag(D_occ))).max() > 1e-7


@pytest.mark.parametrize("o,v,nlo,seed", [(4, 6, 2, 4), (5, 7, 3, 5)])
def test_cbno_densities_are_half_the_spin_orbital_blocks(o, v, nlo, seed):
    fr, Bov = _system(o, v, seed)
    Uo = fr.U[:, :nlo]
    Uv = _orthonormal_cols(v, nlo, seed + 100) * 0.6  # LOs with a partial virtual projection (IAO-like)
    Wo, fo, _ = lno.internal_space(Uo, fr.eps[:o])
    Wv, fv, _ = lno.internal_space(Uv, fr.eps[o:])
    D_occ, D_vir = lno.cbno_densities(fr.eps, Bov, o, Uo, Uv)
    so = spinorb.restricted_mp2_densities(fr.eps, fr.B, o, W_occ=Wo, f_occ=fo, W_vir=Wv, f_vir=fv)
    assert np.abs(D_vir - 0.5 * so["vir_two_int_occ"]).max() < 1e-15
    assert np.abs(D_occ - 0.5 * so["occ_two_int_vir"]).max() < 1e-15


@pytest.mark.parametrize("nlo", [1, 2, 4])
def test_lno_density_traces_agree_and_blocks_are_psd(nlo):
    o, v = 4, 7
    fr, Bov = _system(o, v, 10 + nlo)
    D_occ, D_vir = lno.lno_densities(fr.eps, Bov, o, fr.U[:, :nlo])
    assert abs(np.trace(D_occ) - np.trace(D_vir)) < 1e-15
    assert np.linalg.eigvalsh(D_occ).min() > -1e-16 and np.linalg.eigvalsh(D_vir).min() > -1e-16


def _densities_without_semicanonical_step(eps, Bov, o, U):
    """Planted mistake: internal orbitals W = U as given, 'semi-canonical' energies read off the diagonal."""
    e = np.asarray(eps)
    W = U / np.linalg.norm(U, axis=0)
    f = np.diag(W.T @ np.diag(e[:o]) @ W)
    t = lno.mp1_internal(e, Bov, o, W, f)
    D_occ = 2.0 * (2.0 * np.einsum("Kbia,Kbja->ij", t, t) - np.einsum("Kbia,Kajb->ij", t, t))
    D_vir = (2.0 * (np.einsum("Iajc,Ibjc->ab", t, t) + np.einsum("Icja,Icjb->ab", t, t))
             - (np.einsum("Icja,Ibjc->ab", t, t) + np.einsum("Iajc,Icjb->ab", t, t)))
    return D_occ, D_vir


def test_densities_do_not_depend_on_the_lo_basis_of_the_fragment():
    o, v, nlo = 5, 8, 3
    fr, Bov = _system(o, v, 21)
    U = fr.U[:, :nlo]
    R = _orthonormal_cols(nlo, nlo, 22)
    a = lno.lno_densities(fr.eps, Bov, o, U)
    b = lno.lno_densities(fr.eps, Bov, o, U @ R)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-14
    W, _, Wbar = lno.internal_space(U, fr.eps[:o])
    assert np.abs(lno.external_spectrum(a[1], np.eye(v)) - lno.external_spectrum(b[1], np.eye(v))).max() < 1e-14
    # the planted mistake: without the semi-canonical step the same fragment gives other densities
    pa = _densities_without_semicanonical_step(fr.eps, Bov, o, U)
    pb = _densities_without_semicanonical_step(fr.eps, Bov, o, U @ R)
    assert np.abs(pa[1] - pb[1]).max() > 1e-8


def test_complete_fragment_has_no_external_occupied_space():
    o, v = 4, 6
    fr, Bov = _system(o, v, 31)
    W, f, Wbar = lno.internal_space(fr.U, fr.eps[:o])
    assert W.shape == (o, o) and Wbar.shape == (o, 0)
    assert np.abs(np.sort(f) - np.sort(fr.eps[:o])).max() < 1e-14  # semi-canonical = canonical energies


def test_lno_selection_properties():
    o, v, nlo = 6, 10, 2
    fr, Bov = _system(o, v, 41)
    U = fr.U[:, :nlo]
    W, f, Wbar = lno.internal_space(U, fr.eps[:o])
    D_occ, D_vir = lno.lno_densities(fr.eps, Bov, o, U)
    for D, Wi, Wb in ((D_occ, W, Wbar), (D_vir, np.zeros((v, 0)), np.eye(v))):
        lam, C = lno.select(D, Wb, 0.0)
        n = D.shape[0]
        assert C.shape == (n, Wb.shape[1])
        assert np.abs(C.T @ C - np.eye(C.shape[1])).max() < 1e-13
        if Wi.shape[1]:
            assert np.abs(Wi.T @ C).max() < 1e-13
        P = Wb @ Wb.T
        assert np.abs(C @ np.diag(lam) @ C.T - P @ D @ P).max() < 1e-15
        assert np.all(np.diff(lam) <= 0)
        eta = float(np.median(np.abs(lam)))
        lam2, C2 = lno.select(D, Wb, eta)
        assert 0 < lam2.size < lam.size and np.all(np.abs(lam2) >= eta)
