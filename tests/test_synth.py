"""The seeded input generator: determinism, structure and the value distributions."""
import numpy as np

from oracle import ccsd
from paper_2407_11258_gb300 import synth


def test_splitmix64_reference_values():
    # splitmix64 from state 0: first outputs published with the algorithm (Steele et al. 2014)
    st = synth.Stream(0)
    st.key = np.uint64(0)
    got = st.u64(3)
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_fragment_structure_and_determinism():
    a = synth.single_fp64()
    b = synth.single_fp64()
    assert np.array_equal(a.B, b.B) and np.array_equal(a.eps, b.eps)
    assert a.B.shape == (96, 28, 28)
    assert np.array_equal(a.B, a.B.transpose(0, 2, 1))
    eo, ev = a.eps[:4], a.eps[4:]
    assert np.all(np.diff(eo) >= 0) and np.all(np.diff(ev) >= 0)
    assert -1.5 <= eo.min() and eo.max() <= -0.3 and 0.2 <= ev.min() and ev.max() <= 3.0
    assert np.allclose(a.U @ a.U.T, np.eye(4), atol=1e-14)
    # entry scale: var(B_Qpq) = 0.09 exp(-2|p-q|/L) / naux
    d0 = a.B[:, np.arange(28), np.arange(28)]
    assert 0.5 < d0.var() * 96 / 0.09 < 1.5


def test_small_gap_energies():
    fr = synth.batch_fragment(1, scale_shape=lambda o, v: (4, 12))
    assert fr.kind == "small-gap"
    gap = fr.eps[4] - fr.eps[3]
    assert 0.04 <= gap <= 0.2 + 1e-12
    shapes = synth.batch_shapes()
    assert len(shapes) == 128
    assert all(8 <= o <= 24 and 120 <= v <= 360 and q == 4 * v for o, v, q, _ in shapes)


def test_literal_generator_is_unphysical():
    """N(0,1) entries (no 1/naux) give an MP2 energy of order -100 Eh at nocc=4, nvir=24."""
    fr = synth.make_fragment(4, 24, 96, 1000, occ_range=(-1.5, -0.3), vir_range=(0.2, 3.0),
                             decay=8.0, literal=True)
    e = np.trace(ccsd.pair_energy_matrix(np.zeros((4, 24)), ccsd.mp2_amplitudes(fr.eps, fr.B, 4), fr.B, 4))
    assert e < -50.0
    ok = synth.single_fp64()
    e_ok = np.trace(ccsd.pair_energy_matrix(np.zeros((4, 24)), ccsd.mp2_amplitudes(ok.eps, ok.B, 4), ok.B, 4))
    assert -0.1 < e_ok < 0.0


def test_device_generator_matches_the_cpu_streams_and_distribution():
    """fragment_device (B drawn with torch's generator, here on the CPU device) takes eps and U from the
    same splitmix64 streams as make_fragment, and draws B symmetric with the same entry variance
    0.09 exp(-2|p-q|/20) / naux."""
    torch = __import__("pytest").importorskip("torch")
    for small in (False, True):
        o, v, q, eps, B, U = synth.fragment_device(6, 30, 400, small, 77, "cpu", frag=(0, 2))
        ref = synth.make_fragment(6, 30, 400, 77, small_gap=small, frag=(0, 2))
        assert (o, v, q) == (6, 30, 400)
        assert np.array_equal(eps.numpy(), ref.eps) and np.array_equal(U.numpy(), ref.U_frag)
        b = B.numpy()
        assert b.shape == (400, 36, 36) and np.array_equal(b, b.transpose(0, 2, 1))
    p = np.arange(36)
    w = np.exp(-2.0 * np.abs(p[:, None] - p[None, :]) / 20.0)
    ratio = (b**2).mean(axis=0) * 400 / (0.09 * w)  # per (p,q): mean of 400 squared normals, ~1 +- 0.07
    assert abs(ratio.mean() - 1.0) < 0.02 and 0.7 < ratio.min() and ratio.max() < 1.3
