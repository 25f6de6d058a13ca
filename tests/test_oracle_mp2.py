"""Pins of the MP2 composite-correction oracle (oracle/mp2.py, Eq. 17) against results fixed by the
mathematics: explicit four-index loops, the exact sum rule of complete active spaces (Eq. 5 and 7),
invariance of a complete virtual space under rotation (which needs the semicanonical step), a
one-virtual closed form, and the sign and monotonicity that truncating virtuals must give."""
import numpy as np
import pytest

from oracle import ccsd, mp2
from paper_2407_11258_gb300 import synth


def _system(o, v, seed, naux=30):
    fr = synth.make_fragment(o, v, naux, seed, occ_range=(-1.0, -0.5), vir_range=(0.2, 2.0), decay=8.0,
                             frag=tuple(range(o)))
    return fr, fr.B[:, :o, o:].copy()


def _orthogonal(n, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q * np.sign(np.diag(r))


@pytest.mark.parametrize("o,v,seed", [(2, 5, 1), (3, 7, 2)])
def test_full_mp2_matches_explicit_loops(o, v, seed):
    fr, Bov = _system(o, v, seed)
    assert abs(mp2.full_mp2_energy(fr.eps, Bov, o) - ccsd.mp2_energy_loops(fr.eps, fr.B, o)) < 1e-14


@pytest.mark.parametrize("rotate", [False, True])
def test_complete_active_spaces_give_zero_correction(rotate):
    """Every fragment keeps the whole virtual space (as given, or rotated by a random orthogonal
    matrix: the semicanonical step must undo it) and the fragments partition the LOs of an orthogonal
    U: the fragment energies add up to the full MP2 energy, so Eq. 17 gives zero."""
    o, v = 4, 9
    fr, Bov = _system(o, v, 11)
    C = _orthogonal(v, 12) if rotate else np.eye(v)
    U = fr.U
    e_full = mp2.full_mp2_energy(fr.eps, Bov, o)
    parts = [mp2.fragment_mp2_energy(fr.eps, Bov, o, C, U[:, [a]]) for a in range(o)]
    assert abs(mp2.composite_correction(e_full, parts)) < 1e-14
    # two-LO fragments: same sum
    pairs = [mp2.fragment_mp2_energy(fr.eps, Bov, o, C, U[:, [a, a + 1]]) for a in (0, 2)]
    assert abs(mp2.composite_correction(e_full, pairs)) < 1e-14


def test_rotation_without_semicanonical_step_would_fail():
    """Planted mistake: amplitudes built in a rotated, non-semicanonical virtual basis with the
    diagonal of the rotated Fock block as energies do not reproduce the full MP2 energy."""
    o, v = 3, 7
    fr, Bov = _system(o, v, 21)
    C = _orthogonal(v, 22)
    ev_diag = np.diag(C.T @ np.diag(fr.eps[o:]) @ C)
    wrong = mp2.full_mp2_energy(np.concatenate([fr.eps[:o], ev_diag]), np.einsum("Qia,ab->Qib", Bov, C), o)
    assert abs(wrong - mp2.full_mp2_energy(fr.eps, Bov, o)) > 1e-6


def test_one_virtual_combination_closed_form():
    """A_F with one virtual combination c: e_c = c^T diag(e_vir) c and
    E^(F) = sum_ii' U_i U_i' sum_j (ic|jc)(i'c|jc) / (e_i + e_j - 2 e_c) (the exchange term equals the
    Coulomb term when a = b = c)."""
    o, v = 3, 6
    fr, Bov = _system(o, v, 31)
    c = _orthogonal(v, 32)[:, 0]
    u = fr.U[:, 0]
    ec = float(c @ (fr.eps[o:] * c))
    Bc = np.einsum("Qia,a->Qi", Bov, c)
    want = 0.0
    for i in range(o):
        for ip in range(o):
            for j in range(o):
                want += u[i] * u[ip] * float(Bc[:, i] @ Bc[:, j]) * float(Bc[:, ip] @ Bc[:, j]) / (
                    fr.eps[i] + fr.eps[j] - 2.0 * ec)
    assert abs(mp2.fragment_mp2_energy(fr.eps, Bov, o, c, u) - want) < 1e-15


def test_truncated_virtuals_give_a_negative_monotone_correction():
    """With U = I and one-LO fragments the fragment energies add up to the MP2 energy of the truncated
    space, and each pair (a,b),(b,a) contributes 2[x^2 - xy + y^2]/D <= 0 (x = (ia|jb), y = (ib|ja)):
    keeping more virtuals can only lower the sum, so Delta E of Eq. 17 is <= 0 and rises to 0."""
    o, v = 3, 8
    fr, Bov = _system(o, v, 41)
    e_full = mp2.full_mp2_energy(fr.eps, Bov, o)
    I_o = np.eye(o)
    sums = []
    for k in range(1, v + 1):
        C = np.eye(v)[:, :k]
        sums.append(sum(mp2.fragment_mp2_energy(fr.eps, Bov, o, C, I_o[:, [i]]) for i in range(o)))
    corr = [mp2.composite_correction(e_full, [s]) for s in sums]
    assert all(c <= 1e-15 for c in corr)
    assert all(sums[k + 1] <= sums[k] + 1e-15 for k in range(v - 1))
    assert corr[0] < -1e-6 and abs(corr[-1]) < 1e-14
