"""GPU parity of the local active space (Sec. II.C / II.E) against oracle/lno.py, and of a whole LNO fragment
(active space -> fragment CCSD(T) -> projected energies -> MP2 composite correction) against the oracle
doing the same steps.

Every GPU step takes the GPU's own outputs as its inputs (the oracle never feeds the device path).
Orbitals are compared through basis-independent quantities: projectors C C^T, eigenvalues, energies
(semi-canonical orbitals are unique up to sign, LNOs up to sign and rotations inside degenerate sets).
Tolerances: FP64 path 1e-11 relative (densities, projectors) and 1e-9 Eh (energies); mixed path 1e-4 of
the largest density element (two BF16x3 contraction stages, ~2^-16 relative each, on sums of positive
terms) and 1e-6 Eh for fragment energies.
"""
import numpy as np
import pytest

from oracle import ccsd as occ
from oracle import fragment as ofr
from oracle import lno as olno
from oracle import mp2 as omp2
from oracle import triples as otr
from paper_2407_11258_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lnocc():
    from paper_2407_11258_gb300 import build
    from paper_2407_11258_gb300 import lnocc as m
    build.build()
    m.load()
    return m


def _system(o=8, v=40, q=120, seed=8100):
    fr = synth.make_fragment(o, v, q, seed, occ_range=(-1.2, -0.4), vir_range=(0.3, 3.0), decay=12.0)
    return fr, np.ascontiguousarray(fr.B[:, :o, o:])


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def _proj(C):
    C = C.cpu().numpy() if hasattr(C, "cpu") else C
    return C @ C.T


def test_jacobi_eigensolver_through_selection(lnocc):
    """lnocc_lno_select with no internal space and eta = 0 is a plain symmetric eigendecomposition:
    eigenvalues against numpy, A C = C diag(lambda), C orthonormal, for sizes that exercise the byes of
    an odd dimension and several sweeps."""
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 64, 129):
        M = rng.standard_normal((n, n))
        A = M @ M.T / n + np.diag(np.linspace(0.0, 1.0, n))
        C, lam, k = lnocc.lnocc_lno_select(_dev(A), None, 0.0)
        assert k == n
        C, lam = C.cpu().numpy(), lam.cpu().numpy()
        ref = np.sort(np.linalg.eigvalsh(A))[::-1]
        assert np.abs(lam - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
        assert np.abs(C.T @ C - np.eye(n)).max() < 1e-12
        assert np.abs(A @ C - C * lam).max() < 1e-11


@pytest.mark.parametrize("nlo", [1, 2, 3])
def test_internal_space(lnocc, nlo):
    fr, _ = _system()
    U = fr.U[:, :nlo]
    W, f, k = lnocc.lnocc_lno_internal(_dev(U), _dev(fr.eps[:fr.nocc]))
    Wr, fr_, _ = olno.internal_space(U, fr.eps[:fr.nocc])
    assert k == Wr.shape[1] == nlo
    assert np.abs(_proj(W) - _proj(Wr)).max() < 1e-13
    assert np.abs(f.cpu().numpy() - fr_).max() < 1e-13
    Wn = W.cpu().numpy()
    F = Wn.T @ np.diag(fr.eps[:fr.nocc]) @ Wn
    assert np.abs(F - np.diag(np.diag(F))).max() < 1e-13  # semi-canonical


def test_internal_space_of_a_rank_deficient_lo_set(lnocc):
    fr, _ = _system()
    U = np.stack([fr.U[:, 0], fr.U[:, 0], fr.U[:, 1] + 0.5 * fr.U[:, 0]], axis=1)
    W, f, k = lnocc.lnocc_lno_internal(_dev(U), _dev(fr.eps[:fr.nocc]))
    assert k == 2
    assert np.abs(_proj(W) - _proj(fr.U[:, :2])).max() < 1e-12


@pytest.mark.parametrize("prec,rtol", [(0, 1e-11), (1, 1e-4)])
@pytest.mark.parametrize("nlo", [1, 2])
def test_lno_densities(lnocc, prec, rtol, nlo):
    fr, Bov = _system()
    o, v, q = fr.nocc, fr.nvir, fr.naux
    U = fr.U[:, :nlo]
    W, f, k = lnocc.lnocc_lno_internal(_dev(U), _dev(fr.eps[:o]))
    Do, Dv = lnocc.lnocc_lno_densities(prec, lnocc.LNOCC_LNO_MP2, o, v, q, _dev(fr.eps), _dev(Bov), W, f)
    Do_r, Dv_r = olno.lno_densities(fr.eps, Bov, o, U)
    for got, want in ((Do, Do_r), (Dv, Dv_r)):
        g = got.cpu().numpy()
        assert np.abs(g - want).max() <= rtol * np.abs(want).max(), np.abs(g - want).max() / np.abs(want).max()
        assert np.abs(g - g.T).max() == 0.0


@pytest.mark.parametrize("prec,rtol", [(0, 1e-11), (1, 1e-4)])
def test_cbno_densities(lnocc, prec, rtol):
    fr, Bov = _system(seed=8200)
    o, v, q = fr.nocc, fr.nvir, fr.naux
    rng = np.random.default_rng(3)
    Uo = fr.U[:, :2]
    Uv = 0.5 * np.linalg.qr(rng.standard_normal((v, 3)))[0]  # LOs with a virtual projection (IAO-like)
    Wo, fo, ko = lnocc.lnocc_lno_internal(_dev(Uo), _dev(fr.eps[:o]))
    Wv, fv, kv = lnocc.lnocc_lno_internal(_dev(Uv), _dev(fr.eps[o:]))
    assert (ko, kv) == (2, 3)
    Do, Dv = lnocc.lnocc_lno_densities(prec, lnocc.LNOCC_LNO_CBNO, o, v, q, _dev(fr.eps), _dev(Bov), Wo, fo, Wv, fv)
    Do_r, Dv_r = olno.cbno_densities(fr.eps, Bov, o, Uo, Uv)
    for got, want in ((Do, Do_r), (Dv, Dv_r)):
        g = got.cpu().numpy()
        assert np.abs(g - want).max() <= rtol * np.abs(want).max()


def _gap_threshold(lam):
    """A threshold in the widest relative gap of a decreasing positive spectrum (so both sides keep the
    same LNOs)."""
    lam = np.asarray([x for x in lam if x > 1e-14])
    r = lam[:-1] / lam[1:]
    k = int(np.argmax(r[: max(1, len(r) * 3 // 4)]))
    return float(np.sqrt(lam[k] * lam[k + 1])), k + 1


def test_lno_selection(lnocc):
    fr, Bov = _system()
    o, v, q = fr.nocc, fr.nvir, fr.naux
    U = fr.U[:, :2]
    W, f, _ = lnocc.lnocc_lno_internal(_dev(U), _dev(fr.eps[:o]))
    Do, Dv = lnocc.lnocc_lno_densities(0, lnocc.LNOCC_LNO_MP2, o, v, q, _dev(fr.eps), _dev(Bov), W, f)
    Do_r, Dv_r = olno.lno_densities(fr.eps, Bov, o, U)
    Wr, _, Wbar = olno.internal_space(U, fr.eps[:o])
    for D, D_r, Wi, Wext in ((Do, Do_r, W, Wbar), (Dv, Dv_r, None, np.eye(v))):
        eta, nk = _gap_threshold(olno.external_spectrum(D_r, Wext))
        C, lam, k = lnocc.lnocc_lno_select(D, Wi, eta)
        lam_r, C_r = olno.select(D_r, Wext, eta)
        assert k == len(lam_r) == nk
        assert np.abs(lam.cpu().numpy() - lam_r).max() < 1e-11 * lam_r.max()
        assert np.abs(_proj(C) - _proj(C_r)).max() < 1e-9
        if Wi is not None:
            assert np.abs(Wi.cpu().numpy().T @ C.cpu().numpy()).max() < 1e-12


def _oracle_fragment(fr, Bov, cols, eta_o, eta_v):
    o = fr.nocc
    U = fr.U[:, cols]
    Wr, _, Wbar = olno.internal_space(U, fr.eps[:o])
    Do, Dv = olno.lno_densities(fr.eps, Bov, o, U)
    lo, Co = olno.select(Do, Wbar, eta_o)
    lv, Cv = olno.select(Dv, np.eye(fr.nvir), eta_v)
    C_occ = np.concatenate([Wr, Co], axis=1)
    eF, BF, CF = olno.active_space(fr.eps, fr.B, o, C_occ, Cv)
    noF = C_occ.shape[1]
    UF = CF[:o, :noF].T @ U
    r = occ.ccsd(eF, BF, noF, tol_t=1e-11, tol_e=1e-13)
    Ec = occ.pair_energy_matrix(r["t1"], r["t2"], BF, noF)
    Em = occ.pair_energy_matrix(np.zeros_like(r["t1"]), occ.mp2_amplitudes(eF, BF, noF), BF, noF)
    Et = otr.pair_matrix(r["t1"], r["t2"], eF, BF, noF)
    return dict(sizes=(noF, Cv.shape[1]), e_ccsd_frag=ofr.project(Ec, UF), e_mp2_frag=ofr.project(Em, UF),
                e_t_frag=ofr.project(Et, UF))


def _gpu_fragment(lnocc, fr, Bov, cols, eta_o, eta_v, prec):
    o, v, q = fr.nocc, fr.nvir, fr.naux
    eps, B, Bovd = _dev(fr.eps), _dev(fr.B), _dev(Bov)
    Ud = _dev(fr.U[:, cols])
    W, f, _ = lnocc.lnocc_lno_internal(Ud, eps[:o].contiguous())
    Do, Dv = lnocc.lnocc_lno_densities(prec, lnocc.LNOCC_LNO_MP2, o, v, q, eps, Bovd, W, f)
    Co, lo, ko = lnocc.lnocc_lno_select(Do, W, eta_o)
    Cv, lv, kv = lnocc.lnocc_lno_select(Dv, None, eta_v)
    C_occ = torch.cat([W, Co], dim=1).contiguous()
    eF, BF, CF = lnocc.lnocc_active_space(prec, o, v, q, eps, B, C_occ, Cv)
    noF = C_occ.shape[1]
    UF = _dev(CF[:o, :noF].cpu().numpy().T @ fr.U[:, cols])  # the fragment's LOs in the active occupied basis
    f_ = lnocc.lnocc_build_ints(noF, kv, q, eF, BF, lnocc.default_opts(precision=prec))
    try:
        lnocc.lnocc_ccsd(f_)
        ec, em = lnocc.lnocc_fragment_energy(f_, UF)
        et, etf = lnocc.lnocc_triples(f_, UF)
    finally:
        f_.free()
    return dict(sizes=(noF, kv), e_ccsd_frag=ec, e_mp2_frag=em, e_t_frag=etf)


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-6)])
def test_lno_fragment_end_to_end(lnocc, prec, tol):
    """LNO fragment of two LOs: internal space, LNO densities, thresholds in spectral gaps, semi-canonical
    active space, fragment CCSD(T) and its projected energies (Eq. 12, Eq. 15)."""
    fr, Bov = _system()
    o = fr.nocc
    U = fr.U[:, [0, 1]]
    _, _, Wbar = olno.internal_space(U, fr.eps[:o])
    Do, Dv = olno.lno_densities(fr.eps, Bov, o, U)
    eta_o, _ = _gap_threshold(olno.external_spectrum(Do, Wbar))
    eta_v, _ = _gap_threshold(olno.external_spectrum(Dv, np.eye(fr.nvir)))
    ref = _oracle_fragment(fr, Bov, [0, 1], eta_o, eta_v)
    got = _gpu_fragment(lnocc, fr, Bov, [0, 1], eta_o, eta_v, prec)
    assert got["sizes"] == ref["sizes"]
    assert ref["sizes"][1] < fr.nvir  # a truncated virtual space
    for k in ("e_ccsd_frag", "e_mp2_frag", "e_t_frag"):
        assert abs(got[k] - ref[k]) <= tol, (k, got[k], ref[k])


def test_composite_correction_with_lno_fragments(lnocc):
    """Eq. 17 over four two-LO LNO fragments that partition the LOs (FP64 path): E_MP2 of the system
    from lnocc_mp2_energy minus the fragments' MP2 energies, against the oracle; the correction is
    negative (truncated active spaces miss correlation)."""
    fr, Bov = _system()
    o = fr.nocc
    eta = 1e-5
    parts = [[0, 1], [2, 3], [4, 5], [6, 7]]
    gpu = [_gpu_fragment(lnocc, fr, Bov, p, eta, eta, 0)["e_mp2_frag"] for p in parts]
    ref = [_oracle_fragment(fr, Bov, p, eta, eta)["e_mp2_frag"] for p in parts]
    e_full = lnocc.lnocc_mp2_energy(0, o, fr.nvir, fr.naux, _dev(fr.eps), _dev(Bov))
    corr = omp2.composite_correction(e_full, gpu)
    corr_ref = omp2.composite_correction(omp2.full_mp2_energy(fr.eps, Bov, o), ref)
    assert abs(corr - corr_ref) < 1e-9, (corr, corr_ref)
    assert corr_ref < -1e-7
