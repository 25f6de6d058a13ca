"""Seeded synthetic fragment inputs (orbital energies, DF tensor B[Q,p,q], LO matrix U).

This module only draws random numbers; it holds none of the coupled-cluster
arithmetic, so both the CPU oracle tests and the CUDA path use it.

The paper's workloads are real diamond / lithium fragment Hamiltonians built
with PySCF (Sec. III, Sec. IV); none of them is available here, so these
inputs stand in for them with the shapes and value distributions of those
fragments:

* orbital energies: sorted uniform draws, occupied below virtual (the
  semi-canonical fragment Fock diagonal, Eq. 11 and Eq. 21);
* B[Q,p,q]: real, symmetric in (p,q), entries N(0, 1/naux) scaled by
  0.3*exp(-|p-q|/L) (the Gamma-point real form of the DF factors of Eq. 27a,
  (pq|rs) = sum_Q B_Qpq B_Qrs);
* U: a random orthogonal occupied->LO rotation (Eq. 3, span-occupied
  condition Eq. 5); a fragment is a subset of its columns.

Random numbers come from splitmix64 (Steele, Lea & Flood, OOPSLA 2014), a
counter-based generator whose integer stream is identical on every platform;
normals use the Box-Muller transform.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """splitmix64 counter stream: value k of stream `key` is mix(key + (k+1)*golden)."""

    def __init__(self, seed: int, tag: int = 0):
        with np.errstate(over="ignore"):
            self.key = _mix(np.uint64(seed) * _GOLDEN + np.uint64(tag) + _GOLDEN)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix(self.key + k * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return z[:n]

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] inclusive."""
        return lo + (self.u64(n) % np.uint64(hi - lo + 1)).astype(np.int64)


@dataclasses.dataclass
class Fragment:
    """One fragment's inputs. eps: [n]; B: [naux, n, n]; U: [nocc, nocc]; frag: LO columns."""

    nocc: int
    nvir: int
    naux: int
    eps: np.ndarray
    B: np.ndarray
    U: np.ndarray
    frag: tuple
    seed: int
    kind: str = "gapped"

    @property
    def nmo(self) -> int:
        return self.nocc + self.nvir

    @property
    def U_frag(self) -> np.ndarray:
        return np.ascontiguousarray(self.U[:, list(self.frag)])


def orbital_energies(st: Stream, nocc: int, nvir: int, occ_range, vir_range) -> np.ndarray:
    eo = np.sort(st.uniform(nocc, *occ_range))
    ev = np.sort(st.uniform(nvir, *vir_range))
    return np.concatenate([eo, ev])


def small_gap_energies(st: Stream, nocc: int, nvir: int) -> np.ndarray:
    """Lithium-like energies: virtual minimum vmin ~ U[0.02, 0.1] Eh, gap 2*vmin."""
    vmin = float(st.uniform(1, 0.02, 0.1)[0])
    ev = np.sort(st.uniform(nvir, vmin, 4.0))
    ev[0] = vmin
    eo = np.sort(st.uniform(nocc, -0.8, 0.0)) - vmin
    eo[-1] = -vmin
    return np.concatenate([eo, ev])


def df_tensor(st: Stream, naux: int, n: int, decay: float, scale: float = 0.3,
              literal: bool = False) -> np.ndarray:
    """B[Q,p,q] = g_Qpq * scale*exp(-|p-q|/decay), g ~ N(0, 1/naux), symmetric in p,q.

    literal=True draws g ~ N(0,1) (no 1/sqrt(naux)); that form gives MP2
    energies of -134 Eh already at nocc=4, nvir=24 and is kept only to record
    that it is unphysical.
    """
    iu, ju = np.triu_indices(n)
    g = st.normal(naux * iu.size).reshape(naux, iu.size)
    if not literal:
        g *= 1.0 / np.sqrt(naux)
    g *= scale * np.exp(-np.abs(iu - ju) / decay)[None, :]
    B = np.zeros((naux, n, n))
    B[:, iu, ju] = g
    B[:, ju, iu] = g
    return B


def orthogonal(st: Stream, n: int) -> np.ndarray:
    """Q factor of a Gaussian n x n matrix, columns sign-fixed so diag(R) > 0."""
    a = st.normal(n * n).reshape(n, n)
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


def make_fragment(nocc: int, nvir: int, naux: int, seed: int, *, occ_range=(-1.2, -0.4),
                  vir_range=(0.3, 4.0), decay: float = 20.0, small_gap: bool = False,
                  frag=(0,), literal: bool = False) -> Fragment:
    st_e = Stream(seed, 1)
    st_b = Stream(seed, 2)
    st_u = Stream(seed, 3)
    if small_gap:
        eps = small_gap_energies(st_e, nocc, nvir)
    else:
        eps = orbital_energies(st_e, nocc, nvir, occ_range, vir_range)
    B = df_tensor(st_b, naux, nocc + nvir, decay, literal=literal)
    U = orthogonal(st_u, nocc)
    return Fragment(nocc, nvir, naux, eps, B, U, tuple(frag), seed,
                    "small-gap" if small_gap else "gapped")


# --- the five workloads (sizes and distributions of the fragment solves) ---

def single_fp64(seed: int = 1000) -> Fragment:
    """Small closed-shell fragment: nocc=4, nvir=24, naux=96, L=8, projector = first LMO."""
    return make_fragment(4, 24, 96, seed, occ_range=(-1.5, -0.3), vir_range=(0.2, 3.0),
                         decay=8.0, frag=(0,))


def diamond_like(seed: int = 2000) -> Fragment:
    """Diamond-like gapped fragment: nocc=16, nvir=240, naux=960, L=20, projector onto 2 LMOs."""
    return make_fragment(16, 240, 960, seed, occ_range=(-1.2, -0.4), vir_range=(0.3, 4.0),
                         decay=20.0, frag=(0, 1))


def batch_shapes(nfrag: int = 128, seed: int = 3000):
    """Uneven fragment shapes: nocc U{8..24}, nvir U{120..360}, naux = 4*nvir; odd index = small gap."""
    st = Stream(seed, 7)
    no = st.integers(nfrag, 8, 24)
    nv = st.integers(nfrag, 120, 360)
    return [(int(no[f]), int(nv[f]), int(4 * nv[f]), bool(f % 2)) for f in range(nfrag)]


def batch_fragment(f: int, nfrag: int = 128, seed: int = 3000, scale_shape=None) -> Fragment:
    """Fragment f of the uneven batch; scale_shape(o, v) may shrink it for CPU-sized tests."""
    o, v, q, small = batch_shapes(nfrag, seed)[f]
    if scale_shape is not None:
        o, v = scale_shape(o, v)
        q = 4 * v
    return make_fragment(o, v, q, seed + f, small_gap=small, decay=20.0, frag=(0,))


def triples_large(seed: int = 4000, scaled: bool = False) -> Fragment:
    """(T)-dominated fragment nocc=32, nvir=480, naux=1600; scaled: nocc=12, nvir=96, naux=320."""
    if scaled:
        return make_fragment(12, 96, 320, seed + 1, decay=20.0, frag=(0,))
    return make_fragment(32, 480, 1600, seed, decay=20.0, frag=(0,))


def batch_gap(f: int, nfrag: int = 128, seed: int = 3000) -> float:
    """HOMO-LUMO gap of fragment f of the uneven batch (its energies come from the same stream as
    batch_fragment / batch_fragment_device), without drawing its B."""
    o, v, q, small = batch_shapes(nfrag, seed)[f]
    st_e = Stream(seed + f, 1)
    eps = small_gap_energies(st_e, o, v) if small else orbital_energies(st_e, o, v, (-1.2, -0.4), (0.3, 4.0))
    return float(eps[o] - eps[o - 1])


def batch_fragment_device(f: int, device, nfrag: int = 128, seed: int = 3000):
    """Fragment f of the uneven batch at full size with B drawn on the device (fragment_device): the CPU
    stream needs minutes for the ~88 GB batch. Orbital energies and U come from the same splitmix64
    streams as batch_fragment. Returns (nocc, nvir, naux, eps, B, U_frag), U_frag the first LO."""
    o, v, q, small = batch_shapes(nfrag, seed)[f]
    return fragment_device(o, v, q, small, seed + f, device)


def mlp_shapes(nfrag: int, seed: int = 5000):
    """Learned-guess fragments: nocc U{8..16}, nvir U{96..240}, naux = 4*nvir; odd index = small gap."""
    st = Stream(seed, 7)
    no = st.integers(nfrag, 8, 16)
    nv = st.integers(nfrag, 96, 240)
    return [(int(no[f]), int(nv[f]), int(4 * nv[f]), bool(f % 2)) for f in range(nfrag)]


def fragment_device(o: int, v: int, q: int, small: bool, seed: int, device, frag=(0,)):
    """(nocc, nvir, naux, eps, B, U_frag) with eps / U from splitmix64 streams and B drawn on the device with
    torch's seeded generator (same distribution as df_tensor, decay length 20)."""
    import torch
    n = o + v
    st_e, st_u = Stream(seed, 1), Stream(seed, 3)
    eps = small_gap_energies(st_e, o, v) if small else orbital_energies(st_e, o, v, (-1.2, -0.4), (0.3, 4.0))
    U = orthogonal(st_u, o)[:, list(frag)].copy()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    B = torch.randn(q, n, n, generator=gen, device=device, dtype=torch.float64)
    B = torch.triu(B) + torch.triu(B, 1).transpose(1, 2)
    idx = torch.arange(n, device=device, dtype=torch.float64)
    B *= (0.3 / np.sqrt(q)) * torch.exp(-(idx[:, None] - idx[None, :]).abs() / 20.0)
    return (o, v, q, torch.tensor(eps, device=device), B.contiguous(), torch.tensor(U, device=device))


def mlp_fragment_device(k: int, device, seed: int = 5000, nfrag: int = 2256, scale_shape=None):
    """Fragment k of the learned-guess set (k < 2000: training, the rest held out)."""
    o, v, q, small = mlp_shapes(nfrag, seed)[k]
    if scale_shape is not None:
        o, v = scale_shape(o, v)
        q = 4 * v
    return fragment_device(o, v, q, small, seed + 1 + k, device)


def mlp_init(seed: int = 5100, hidden: int = 128) -> np.ndarray:
    """Initial MLP parameters in the layout W1[H][8], b1[H], W2[H][H], b2[H], w3[H], b3[1]:
    weights N(0, 1/fan_in), biases 0."""
    st = Stream(seed, 15)
    parts = [st.normal(hidden * 8) / np.sqrt(8.0), np.zeros(hidden), st.normal(hidden * hidden) / np.sqrt(hidden),
             np.zeros(hidden), st.normal(hidden) / np.sqrt(hidden), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def kpoint_factors(nk: int, naux: int, n: int, seed: int, decay: float = 20.0):
    """Stand-in for the k-point DF factors of the local Hamiltonian (Eq. 27b) on a 1-D mesh of nk
    momentum transfers q: real supercell factors B_R[P][p][r] (one block per cell R, symmetric in p, r,
    drawn like df_tensor, scaled by nk^(-1/2)) and L^P_pr(q) = nk^(-1/2) sum_R exp(2 pi i q R / nk) B_R[P][p][r], which has the
    symmetries of real orbitals (L_pr(q) = L_rp(q), L(-q) = conj L(q)).
    Returns (L [nk][naux][n][n] complex128, qneg [nk] with qneg[q] = -q mod nk, B_cells [nk * naux][n][n])."""
    st = Stream(seed, 31)
    # each cell's factors drawn like df_tensor and scaled by nk^(-1/2): the supercell integrals then have
    # the magnitude of nk * naux auxiliary functions drawn with N(0, 1 / (nk * naux)) entries
    cells = [df_tensor(st, naux, n, decay) / np.sqrt(nk) for _ in range(nk)]
    Bc = np.stack(cells)                                    # [R][P][p][r]
    R = np.arange(nk)
    ph = np.exp(2j * np.pi * np.outer(R, R) / nk) / np.sqrt(nk)  # [q][R]
    L = np.einsum("qR,Rpab->qpab", ph, Bc)
    qneg = (-R) % nk
    return L, qneg, Bc.reshape(nk * naux, n, n)
