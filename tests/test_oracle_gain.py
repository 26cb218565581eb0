"""Pins for the oracle's gain model M = G R G^H, its loss and gradient.
Expected values: numpy full-matrix algebra and fp64 central differences."""
import numpy as np

import oracle


def _unpack(Vp, N):
    C = Vp.shape[0]
    full = np.zeros((C, N, N), complex)
    i, j = np.tril_indices(N)
    order = np.argsort(i * (i + 1) // 2 + j)
    full[:, i[order], j[order]] = Vp
    full[:, j[order], i[order]] = Vp.conj()
    return full


def _random_hermitian_packed(rng, C, N):
    A = rng.standard_normal((C, N, 5)) + 1j * rng.standard_normal((C, N, 5))
    full = A @ A.conj().transpose(0, 2, 1)
    i, j = np.tril_indices(N)
    order = np.argsort(i * (i + 1) // 2 + j)
    return full[:, i[order], j[order]]


def test_loss_matches_full_matrix():
    rng = np.random.default_rng(31)
    C, N = 3, 7
    R = _random_hermitian_packed(rng, C, N)
    V = _random_hermitian_packed(rng, C, N)
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    L, _ = oracle.gain_loss_grad(R, V, g)
    G = np.diag(g)
    M = G[None] @ _unpack(R, N) @ G.conj().T[None]
    ref = (np.abs(M - _unpack(V, N)) ** 2).sum()
    assert abs(L - ref) <= 1e-12 * ref


def test_gradient_central_differences():
    rng = np.random.default_rng(32)
    C, N = 2, 6
    R = _random_hermitian_packed(rng, C, N)
    V = _random_hermitian_packed(rng, C, N)
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    _, grad = oracle.gain_loss_grad(R, V, g)
    h = 1e-6
    fd = np.zeros(N, complex)
    for k in range(N):
        for part, unit in ((0, 1.0), (1, 1j)):
            gp, gm = g.copy(), g.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            d = (oracle.gain_loss_grad(R, V, gp)[0] - oracle.gain_loss_grad(R, V, gm)[0]) / (2 * h)
            fd[k] += d * unit
    assert np.max(np.abs(grad - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_zero_at_true_gains():
    rng = np.random.default_rng(33)
    C, N = 2, 5
    R = _random_hermitian_packed(rng, C, N)
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    G = np.diag(g)
    Vfull = G[None] @ _unpack(R, N) @ G.conj().T[None]
    i, j = np.tril_indices(N)
    order = np.argsort(i * (i + 1) // 2 + j)
    V = Vfull[:, i[order], j[order]]
    L, grad = oracle.gain_loss_grad(R, V, g)
    assert L < 1e-20 * (np.abs(V) ** 2).sum() + 1e-24
    assert np.max(np.abs(grad)) < 1e-10
