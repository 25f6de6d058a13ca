"""Pins of the learned-guess oracle (oracle/mlp.py) against facts that do not come from its own code:
central finite differences, the small-weight limit of the network, library values of the logistic
function, Adam's first-step property, the MP2 closed form and the t2 permutation symmetry."""
import numpy as np
import pytest
from scipy.special import expit

from oracle import ccsd as occ
from oracle import mlp
from paper_2407_11258_gb300 import synth


def rand_params(H, seed, scale=0.5):
    st = synth.Stream(seed, 11)
    return st.normal(mlp.n_params(H)) * scale


def rand_data(n, seed):
    st = synth.Stream(seed, 12)
    X = st.normal(n * mlp.NFEAT).reshape(n, mlp.NFEAT)
    t = st.normal(n)
    return X, t


def test_layout_size():
    assert mlp.n_params(128) == 128 * 8 + 128 + 128 * 128 + 128 + 128 + 1 == 17793
    P = mlp.unpack(np.arange(mlp.n_params(4), dtype=float), 4)
    assert P["W1"][0, 0] == 0 and P["b1"][0] == 32 and P["W2"][0, 0] == 36 and P["b3"][0] == mlp.n_params(4) - 1


def test_silu_against_library_logistic():
    z = np.linspace(-30, 30, 601)
    assert np.allclose(mlp.silu(z), z * expit(z), rtol=1e-14, atol=1e-300)
    h = 1e-6
    assert np.allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-8)


def test_gradient_tiny_net_all_parameters_finite_differences():
    """Every parameter of a width-4 network: analytic backward vs central differences (FP64)."""
    H = 4
    p = rand_params(H, 1)
    X, t = rand_data(7, 2)
    mu, sd = X.mean(0) * 0.3, X.std(0) * 1.7
    _, g = mlp.backward(p, X, t, mu, sd, H)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (mlp.loss(p + e, X, t, mu, sd, H) - mlp.loss(p - e, X, t, mu, sd, H)) / (2 * h)
    assert np.max(np.abs(g - fd)) / np.max(np.abs(fd)) < 1e-7


def test_gradient_full_width_sampled_finite_differences():
    """Width 128: 200 parameters sampled over every block, relative error below 1e-6."""
    p = rand_params(128, 3, scale=0.1)
    X, t = rand_data(16, 4)
    mu, sd = np.zeros(8), np.ones(8)
    _, g = mlp.backward(p, X, t, mu, sd)
    st = synth.Stream(5, 13)
    idx = np.unique(np.concatenate([st.integers(150, 0, p.size - 1), np.arange(1024, 1024 + 128, 8),
                                    [p.size - 1, p.size - 2]]))
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(p + e, X, t, mu, sd) - mlp.loss(p - e, X, t, mu, sd)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1e-3), k


def test_forward_small_weight_limit_fixes_layer_order():
    """With zero biases and W1, W2 scaled by lam -> 0: silu(z) = z/2 + z^2/4 + O(z^4), so
    y / lam^2 -> w3 . W2 W1 x / 4. A transposed or swapped weight matrix breaks the limit."""
    H = 6
    p = rand_params(H, 6)
    P = mlp.unpack(p, H)
    P["b1"][:] = 0
    P["b2"][:] = 0
    P["b3"][:] = 0
    X, _ = rand_data(5, 7)
    lam = 1e-5
    q = p.copy()
    Q = mlp.unpack(q, H)
    Q["W1"] *= lam
    Q["W2"] *= lam
    y, _ = mlp.forward(q, X, np.zeros(8), np.ones(8), H)
    lin = X @ (P["w3"] @ P["W2"] @ P["W1"]) / 4.0
    assert np.allclose(y / lam**2, lin, rtol=1e-4, atol=1e-8)


def test_forward_zero_weights_gives_output_bias():
    p = np.zeros(mlp.n_params(8))
    mlp.unpack(p, 8)["b3"][0] = 0.37
    y, _ = mlp.forward(p, rand_data(4, 8)[0], np.zeros(8), np.ones(8), 8)
    assert np.all(y == 0.37)


def test_adam_first_step_and_quadratic():
    """Adam's first bias-corrected step is -lr * g / (|g| + eps) (Kingma & Ba, Sec. 2); on f(x) = x^2
    it reaches the minimum."""
    g = np.array([3.0, -0.02, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    x, m, v = np.array([2.0]), np.zeros(1), np.zeros(1)
    for step in range(1, 3001):
        x, m, v = mlp.adam(x, 2 * x, m, v, step, lr=0.01)
    assert abs(x[0]) < 1e-2


def test_features_definitions_and_symmetry():
    fr = synth.make_fragment(3, 7, 30, 17, decay=20.0)
    o, v = fr.nocc, fr.nvir
    st = synth.Stream(9, 14)
    i, j = st.integers(40, 0, o - 1), st.integers(40, 0, o - 1)
    a, b = st.integers(40, 0, v - 1), st.integers(40, 0, v - 1)
    X = mlp.features(fr.eps, fr.B, o, i, j, a, b)
    Xs = mlp.features(fr.eps, fr.B, o, j, i, b, a)
    assert np.array_equal(X, Xs)  # (i,j,a,b) and (j,i,b,a) share features
    t2 = occ.mp2_amplitudes(fr.eps, fr.B, o)
    assert np.allclose(X[:, 0], t2[i, j, a, b], rtol=1e-13, atol=0)
    assert np.all(X[:, 5] < 0)
    eri = np.einsum("Qpq,Qrs->pqrs", fr.B, fr.B)
    ci, cj, ca, cb = mlp.canonical(i, j, a, b)
    assert np.allclose(X[:, 6], eri[ci, o + ca, cj, o + cb], rtol=1e-12)
    assert np.allclose(X[:, 7], eri[ci, o + cb, cj, o + ca], rtol=1e-12)


def test_guess_reduces_to_mp2_and_is_symmetric():
    fr = synth.make_fragment(3, 6, 24, 19, decay=20.0)
    o = fr.nocc
    p = np.zeros(mlp.n_params(8))
    t2 = occ.mp2_amplitudes(fr.eps, fr.B, o)
    g0 = mlp.guess(p, np.zeros(8), np.ones(8), 1.0, fr.eps, fr.B, o, 8)
    assert np.allclose(g0, t2, rtol=1e-13, atol=0)
    g1 = mlp.guess(rand_params(8, 20), np.zeros(8), np.ones(8), 1e-3, fr.eps, fr.B, o, 8)
    assert np.array_equal(g1, g1.transpose(1, 0, 3, 2))
    assert not np.allclose(g1, t2)


@pytest.mark.parametrize("seed", [21, 22])
def test_standardisation(seed):
    X, t = rand_data(50, seed)
    mu, sd, s = mlp.standardisation(X * 3 + 1, t * 0.01)
    assert np.allclose(mu, (X * 3 + 1).mean(0)) and np.allclose(sd, 3 * X.std(0))
    assert np.isclose(s, 0.01 * np.sqrt(np.mean(t**2)))
