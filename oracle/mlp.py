"""ORACLE (test infrastructure only): the learned T2 initial guess in FP64 on the CPU.

The paper starts every fragment's CCSD from first-order (MP2) amplitudes (Eq. 21, canonical form)
and has no learned component. The learned guess is a per-amplitude correction
    t_ij^ab(guess) = t_ij^ab(MP2) + s_out * g(x_ijab),
where g is a small multilayer perceptron and x_ijab holds eight features of the amplitude:
    [t_ij^ab(MP2), e_i, e_j, e_a, e_b, D_ij^ab, (ia|jb), (ib|ja)],  D_ij^ab = e_i + e_j - e_a - e_b,
standardised feature-wise with stored means and standard deviations. The converged amplitudes are
symmetric, t_ij^ab = t_ji^ba, so the features of (i, j, a, b) are taken at the canonical
representative of the pair {(i, j, a, b), (j, i, b, a)} -- the one with i < j, or i == j and a <= b --
which makes the guess symmetric by construction.

Network (width H, 128 in production): z1 = W1 x + b1, h1 = silu(z1), z2 = W2 h1 + b2,
h2 = silu(z2), y = w3 . h2 + b3, with silu(z) = z / (1 + exp(-z)). Training minimises the mean
squared error between y and the standardised target (t_conv - t_MP2) / s_out with Adam
(Kingma & Ba, ICLR 2015: bias-corrected first and second moments).

Parameter vector layout (shared with the GPU kernels, float32 there): W1[H][8], b1[H], W2[H][H],
b2[H], w3[H], b3[1]; matrices row-major with the output index first.
"""
from __future__ import annotations

import numpy as np

NFEAT = 8
HIDDEN = 128


def layout(H: int = HIDDEN):
    """(name, shape) of each parameter block, in storage order."""
    return [("W1", (H, NFEAT)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]


def n_params(H: int = HIDDEN) -> int:
    return sum(int(np.prod(s)) for _, s in layout(H))


def unpack(p: np.ndarray, H: int = HIDDEN) -> dict:
    out, k = {}, 0
    for name, shape in layout(H):
        m = int(np.prod(shape))
        out[name] = p[k:k + m].reshape(shape)
        k += m
    return out


# ------------------------------------------------------------------------------------------ features
def canonical(i, j, a, b):
    """Representative of {(i, j, a, b), (j, i, b, a)}: i < j, or i == j and a <= b."""
    i, j, a, b = (np.asarray(x) for x in (i, j, a, b))
    swap = (i > j) | ((i == j) & (a > b))
    return np.where(swap, j, i), np.where(swap, i, j), np.where(swap, b, a), np.where(swap, a, b)


def features(eps, B, nocc, i, j, a, b):
    """Raw (unstandardised) features [n][8] of amplitudes (i, j, a, b); a, b count virtuals from 0."""
    e = np.asarray(eps, dtype=np.float64)
    ci, cj, ca, cb = canonical(i, j, a, b)
    Bov = B[:, :nocc, nocc:]
    iajb = np.einsum("Qn,Qn->n", Bov[:, ci, ca], Bov[:, cj, cb])  # (ia|jb)
    ibja = np.einsum("Qn,Qn->n", Bov[:, ci, cb], Bov[:, cj, ca])  # (ib|ja)
    ei, ej, ea, eb = e[ci], e[cj], e[nocc + ca], e[nocc + cb]
    D = ei + ej - ea - eb
    return np.stack([iajb / D, ei, ej, ea, eb, D, iajb, ibja], axis=1)


# ------------------------------------------------------------------------------------------ network
def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, X, mu, sd, H: int = HIDDEN):
    """Network output y[n] for raw features X[n][8] (standardised with mu, sd), and the cache."""
    P = unpack(np.asarray(p, dtype=np.float64), H)
    x = (np.asarray(X, dtype=np.float64) - mu) / sd
    z1 = x @ P["W1"].T + P["b1"]
    h1 = silu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = silu(z2)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss(p, X, t, mu, sd, H: int = HIDDEN) -> float:
    y, _ = forward(p, X, mu, sd, H)
    return float(np.mean((y - t) ** 2))


def backward(p, X, t, mu, sd, H: int = HIDDEN):
    """(loss, gradient of the loss with respect to the parameter vector), by the chain rule."""
    P = unpack(np.asarray(p, dtype=np.float64), H)
    y, (x, z1, h1, z2, h2) = forward(p, X, mu, sd, H)
    n = y.shape[0]
    dy = 2.0 * (y - t) / n
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, P["w3"]) * dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * dsilu(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    grad = np.concatenate([g[name].ravel() for name, _ in layout(H)])
    return float(np.mean((y - t) ** 2)), grad


def adam(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ------------------------------------------------------------------------------------------ guess
def standardisation(X, dt):
    """Feature means / standard deviations and the target scale s_out = rms of the corrections dt."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    s_out = float(np.sqrt(np.mean(np.asarray(dt, dtype=np.float64) ** 2)))
    return mu, sd, (s_out if s_out > 0 else 1.0)


def guess(p, mu, sd, s_out, eps, B, nocc, H: int = HIDDEN):
    """Full learned guess t2[i][j][a][b] = t_MP2 + s_out * g(features)."""
    nvir = B.shape[1] - nocc
    i, j, a, b = (x.ravel() for x in np.meshgrid(np.arange(nocc), np.arange(nocc), np.arange(nvir),
                                                 np.arange(nvir), indexing="ij"))
    X = features(eps, B, nocc, i, j, a, b)
    y, _ = forward(p, X, mu, sd, H)
    # t_MP2 of the element itself (equal to that of its canonical representative)
    return (X[:, 0] + s_out * y).reshape(nocc, nocc, nvir, nvir)
