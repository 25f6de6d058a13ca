"""Learned T2 guess on the GPU against the oracle (oracle/mlp.py): features, forward, gradients
(FP64 build within 1e-6 relative, FP32 build within 1e-3), the Adam step, the BF16 tensor-core
inference kernel within its rounding bound, and the end-to-end effect of a trained network on CCSD
iteration counts with unchanged converged energies."""
import numpy as np
import pytest

from oracle import ccsd as occ
from oracle import mlp as omlp
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


def solved(lnocc, fr, prec=0):
    eps, B = torch.tensor(fr.eps, device="cuda"), torch.tensor(fr.B, device="cuda")
    f = lnocc.lnocc_build_ints(fr.nocc, fr.nvir, fr.naux, eps, B, lnocc.default_opts(precision=prec))
    t2 = torch.zeros(fr.nocc, fr.nocc, fr.nvir, fr.nvir, dtype=torch.float64, device="cuda")
    lnocc.lnocc_ccsd(f, t2_out=t2)
    return f, t2


def sample_idx(o, v, n, seed):
    st = synth.Stream(seed, 16)
    return st.integers(n, 0, o * o * v * v - 1).astype(np.int64)


def unflat(idx, o, v):
    b = idx % v
    a = (idx // v) % v
    j = (idx // (v * v)) % o
    i = idx // (v * v * o)
    return i, j, a, b


@pytest.fixture(scope="module")
def small_case(lnocc):
    fr = synth.make_fragment(4, 20, 80, 31, decay=20.0)
    f, t2 = solved(lnocc, fr)
    idx = sample_idx(fr.nocc, fr.nvir, 300, 1)
    i, j, a, b = unflat(idx, fr.nocc, fr.nvir)
    idx = np.concatenate([idx, ((j * fr.nocc + i) * fr.nvir + b) * fr.nvir + a])  # and the partners
    X = torch.zeros(idx.size, 8, dtype=torch.float32, device="cuda")
    dt = torch.zeros(idx.size, dtype=torch.float32, device="cuda")
    lnocc.lnocc_mlp_samples(f, torch.tensor(idx, device="cuda"), X, dt)
    yield fr, f, t2, idx, X, dt
    f.free()


def test_samples_match_oracle_features(lnocc, small_case):
    fr, f, t2, idx, X, dt = small_case
    i, j, a, b = unflat(idx, fr.nocc, fr.nvir)
    ref = omlp.features(fr.eps, fr.B, fr.nocc, i, j, a, b)
    np.testing.assert_allclose(X.cpu().numpy(), ref.astype(np.float32), rtol=2e-6, atol=1e-12)
    t2mp2 = occ.mp2_amplitudes(fr.eps, fr.B, fr.nocc)
    want = t2.cpu().numpy()[i, j, a, b] - t2mp2[i, j, a, b]
    np.testing.assert_allclose(dt.cpu().numpy(), want.astype(np.float32), rtol=1e-5, atol=1e-9)
    n = idx.size // 2
    assert torch.equal(X[:n], X[n:])  # (i,j,a,b) and (j,i,b,a) share features


def model_with_norm(lnocc, X, dt, seed=5101):
    m = lnocc.Mlp(synth.mlp_init(seed))
    m.fit_norm(X, dt)
    return m


def test_fit_norm_matches_oracle(lnocc, small_case):
    _, _, _, _, X, dt = small_case
    m = model_with_norm(lnocc, X, dt)
    _, nrm = m.get()
    mu, sd, s_out = omlp.standardisation(X.cpu().numpy().astype(np.float64), dt.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(nrm[:8], mu, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(nrm[8:16], sd, rtol=1e-7)
    assert abs(nrm[16] - s_out) <= 1e-12 * s_out
    m.free()


@pytest.mark.parametrize("prec,rtol", [(0, 1e-10), (1, 1e-5)])
def test_forward_matches_oracle(lnocc, small_case, prec, rtol):
    _, _, _, _, X, dt = small_case
    m = model_with_norm(lnocc, X, dt)
    p, nrm = m.get()
    y = m.forward(X, precision=prec).cpu().numpy()
    yo, _ = omlp.forward(p.astype(np.float64), X.cpu().numpy().astype(np.float64), nrm[:8], nrm[8:16])
    assert np.max(np.abs(y - yo)) <= rtol * np.max(np.abs(yo))
    m.free()


@pytest.mark.parametrize("prec,rtol", [(0, 1e-6), (1, 1e-3)])
def test_gradient_matches_oracle(lnocc, small_case, prec, rtol):
    """Hand-written backward (FP64 build: 1e-6, FP32 build: 1e-3 relative) against the oracle's FP64
    analytic gradient, which itself is pinned by finite differences."""
    _, _, _, _, X, dt = small_case
    m = model_with_norm(lnocc, X, dt)
    p, nrm = m.get()
    loss, g = m.grad(X, dt, precision=prec)
    t = dt.cpu().numpy().astype(np.float64) / nrm[16]
    lo, go = omlp.backward(p.astype(np.float64), X.cpu().numpy().astype(np.float64), t, nrm[:8], nrm[8:16])
    g = g.cpu().numpy()
    assert abs(loss - lo) <= rtol * lo
    for name, _ in omlp.layout():  # every block, relative to its own scale
        sl = slice(*block_range(name))
        assert np.max(np.abs(g[sl] - go[sl])) <= rtol * np.max(np.abs(go[sl])), name
    m.free()


def block_range(name):
    k = 0
    for nm, shape in omlp.layout():
        size = int(np.prod(shape))
        if nm == name:
            return k, k + size
        k += size
    raise KeyError(name)


def test_adam_step_matches_oracle(lnocc, small_case):
    _, _, _, _, X, dt = small_case
    m = model_with_norm(lnocc, X, dt)
    p0, nrm = m.get()
    lr = 1e-3
    t = dt.cpu().numpy().astype(np.float64) / nrm[16]
    _, go = omlp.backward(p0.astype(np.float64), X.cpu().numpy().astype(np.float64), t, nrm[:8], nrm[8:16])
    loss = m.train_step(X, dt, lr)
    p1, _ = m.get()
    pw, _, _ = omlp.adam(p0.astype(np.float64), go, np.zeros_like(go), np.zeros_like(go), 1, lr=lr)
    # FP32 state: the step is lr * g / (|g| + eps) to about 1e-3 relative where |g| >> eps
    big = np.abs(go) > 1e-5
    assert np.max(np.abs(p1[big] - pw[big])) <= 2e-3 * lr + 1e-6 * np.max(np.abs(p0))
    assert np.isfinite(loss) and loss > 0
    m.free()


def test_bf16_inference_within_rounding_bound(lnocc):
    """lnocc_mlp_guess (BF16 tcgen05 layer 2, FP32 accumulation) against the oracle's FP64 guess.
    Bound: h1 and W2 rounded to BF16 (relative 2^-9 each) give |dz2_k| <= 2^-8 sum_l |W2_kl||h1_l|;
    |silu'| <= 1.1 carries it to |dy| <= 1.1 sum_k |w3_k| |dz2_k|; times 1.5 for FP32 sums."""
    fr = synth.make_fragment(5, 28, 112, 41, decay=20.0)  # 19600 amplitudes: 154 tiles with a ragged tail
    f, _ = solved(lnocc, fr)
    o, v = fr.nocc, fr.nvir
    n = o * o * v * v
    m = lnocc.Mlp(synth.mlp_init(5102))
    nrm = np.concatenate([np.full(8, 0.01), np.full(8, 0.5), [3e-3]])
    nrm[1:5] = [-0.8, -0.8, 1.5, 1.5]
    m.set_norm(nrm)
    t2g = torch.zeros(o, o, v, v, dtype=torch.float64, device="cuda")
    lnocc.lnocc_mlp_guess(f, m, t2g)
    g = t2g.cpu().numpy()
    p, _ = m.get()
    P = omlp.unpack(p.astype(np.float64))
    i, j, a, b = (x.ravel() for x in np.meshgrid(np.arange(o), np.arange(o), np.arange(v), np.arange(v),
                                                 indexing="ij"))
    X = omlp.features(fr.eps, fr.B, o, i, j, a, b)
    y, (x, z1, h1, z2, h2) = omlp.forward(p.astype(np.float64), X, nrm[:8], nrm[8:16])
    t2mp2 = occ.mp2_amplitudes(fr.eps, fr.B, o).ravel()
    y_gpu = (g.ravel() - t2mp2) / nrm[16]
    dz2 = 2.0**-8 * (np.abs(h1) @ np.abs(P["W2"]).T)
    bound = 1.5 * 1.1 * (dz2 @ np.abs(P["w3"])) + 1e-4 * (1 + np.abs(y))
    err = np.abs(y_gpu - y)
    assert err.size == n and np.all(err <= bound), (err.max(), bound[np.argmax(err - bound)])
    assert np.max(err) > 0  # BF16 really is used (an FP32 layer 2 would be far inside the bound)
    np.testing.assert_allclose(g, g.transpose(1, 0, 3, 2), rtol=0, atol=1e-15)
    m.free()
    f.free()


def test_trained_guess_cuts_iterations_same_energies(lnocc):
    """Train on GPU solves of shrunk learned-guess fragments, then compare CCSD from the learned guess
    with CCSD from the MP2 guess on held-out fragments (FP64 path, so energies compare at 1e-8)."""
    shrink = lambda o, v: (max(3, o // 2), max(16, v // 6))  # noqa: E731
    dev = "cuda"
    Xs, dts = [], []
    for k in range(24):
        o, v, q, eps, B, U = synth.mlp_fragment_device(k, dev, scale_shape=shrink)
        f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(precision=0))
        lnocc.lnocc_ccsd(f)
        n = min(2048, o * o * v * v)
        idx = torch.tensor(sample_idx(o, v, n, 100 + k), device=dev)
        X = torch.zeros(n, 8, dtype=torch.float32, device=dev)
        dt = torch.zeros(n, dtype=torch.float32, device=dev)
        lnocc.lnocc_mlp_samples(f, idx, X, dt)
        Xs.append(X)
        dts.append(dt)
        f.free()
    X, dt = torch.cat(Xs), torch.cat(dts)
    m = lnocc.Mlp(synth.mlp_init(5103))
    m.fit_norm(X, dt)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    losses = []
    for step in range(400):
        sel = torch.randint(0, X.shape[0], (8192,), generator=gen, device=dev)
        losses.append(m.train_step(X[sel].contiguous(), dt[sel].contiguous(), 3e-3 if step < 300 else 1e-3))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    it_mp2, it_mlp = [], []
    for k in range(2000, 2008):
        o, v, q, eps, B, U = synth.mlp_fragment_device(k, dev, scale_shape=shrink)
        f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(precision=0))
        e0, n0, _ = lnocc.lnocc_ccsd(f)
        lnocc.lnocc_frag_set_mlp(f, m)
        e1, n1, _ = lnocc.lnocc_ccsd(f, guess_mode=lnocc.LNOCC_GUESS_MLP)
        assert abs(e1 - e0) <= 1e-8
        it_mp2.append(n0)
        it_mlp.append(n1)
        f.free()
    assert np.mean(it_mlp) < np.mean(it_mp2), (it_mlp, it_mp2)
    m.free()
