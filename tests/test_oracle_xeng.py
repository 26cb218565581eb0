"""Pins for the oracle's correlation (Sec. 4.2.5) and its whole-stage
composition.  Expected values come from numpy's einsum/eigh, Python integers,
closed forms and invariants -- never from the oracle or the CUDA path."""
import numpy as np
import pytest

import oracle
import synth


def _packed(full):
    N = full.shape[-1]
    i, j = np.tril_indices(N)
    order = np.argsort(i * (i + 1) // 2 + j)
    return full[..., i[order], j[order]]


@pytest.mark.parametrize("N,T", [(1, 1), (2, 3), (3, 7), (5, 4), (4, 1)])
def test_brute_force_tiny(N, T):
    rng = np.random.default_rng(N * 10 + T)
    X = rng.standard_normal((2, N, T)) + 1j * rng.standard_normal((2, N, T))
    V = oracle.correlate(X)
    full = np.einsum("cit,cjt->cij", X, X.conj())
    assert np.allclose(V, _packed(full), atol=1e-12)


def test_packing_order_explicit():
    # N = 3: bl order (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
    X = np.array([[[1.0]], [[2.0j]], [[3.0]]]).reshape(1, 3, 1)
    V = oracle.correlate(X)[0]
    assert np.allclose(V, [1, 2j, 4, 3, -6j, 9])


def test_hermitian_invariants():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((3, 6, 50)) + 1j * rng.standard_normal((3, 6, 50))
    V = oracle.correlate(X)
    for c in range(3):
        full = np.zeros((6, 6), complex)
        k = 0
        for i in range(6):
            for j in range(i + 1):
                full[i, j] = V[c, k]
                k += 1
        auto = np.diag(full)
        assert np.all(np.abs(auto.imag) < 1e-12) and np.all(auto.real >= 0)
        for i in range(6):
            for j in range(i):
                assert abs(full[i, j]) ** 2 <= auto[i].real * auto[j].real * (1 + 1e-12)


def test_int_exact_against_python_ints():
    rng = np.random.default_rng(12)
    N, T = 4, 9
    x = rng.integers(-127, 128, (T, N, 2))
    V = oracle.correlate_int(x)
    k = 0
    for i in range(N):
        for j in range(i + 1):
            re = sum(int(x[t, i, 0]) * int(x[t, j, 0]) + int(x[t, i, 1]) * int(x[t, j, 1]) for t in range(T))
            im = sum(int(x[t, i, 1]) * int(x[t, j, 0]) - int(x[t, i, 0]) * int(x[t, j, 1]) for t in range(T))
            assert V[k, 0] == re and V[k, 1] == im
            k += 1


def test_int_exact_beyond_int32():
    """Full-scale +-127 samples for 140,000 samples: V_ii = 2*127^2*T > 2^31."""
    T = 140000
    x = np.empty((T, 2, 2), np.int16)
    x[:, 0, 0], x[:, 0, 1] = 127, -127
    x[:, 1, 0], x[:, 1, 1] = -127, -127
    V = oracle.correlate_int(x)
    assert V[0, 0] == 2 * 127 * 127 * T > 2 ** 31
    # x1 conj(x0) = (-127 - 127i)(127 + 127i) = -2*127^2 i
    assert V[1, 0] == 0 and V[1, 1] == -2 * 127 * 127 * T


def test_point_source_rank_one_phase():
    """Noise-free single point source through the whole stage: V_c = P_c u u^H,
    phase(V_ij) = phi_i - phi_j, top eigenvalue / trace = 1."""
    N, C, P = 8, 16, 8
    sky = synth.make_sky(N, 1, 1.0, seed=21)
    phi_ant = synth.geometric_phase(sky, 0)[0]
    phi = phi_ant[np.arange(N) // 2]
    rng = np.random.default_rng(22)
    S = C * (P + 40)
    s = rng.standard_normal(S) + 1j * rng.standard_normal(S)
    x = s[:, None] * np.exp(1j * phi)[None, :]
    V = oracle.correlator(x, P, C)[0]                      # [C, NB]
    i, j = np.tril_indices(N)
    order = np.argsort(i * (i + 1) // 2 + j)
    ii, jj = i[order], j[order]
    for c in range(C):
        d = np.angle(V[c] * np.exp(-1j * (phi[ii] - phi[jj])))
        assert np.all(np.abs(d) < 1e-10)
        full = np.zeros((N, N), complex)
        full[ii, jj] = V[c]
        full[jj, ii] = V[c].conj()
        ev = np.linalg.eigvalsh(full)
        assert ev[-1] / ev.sum() > 1 - 1e-12


def test_correlator_raw_int_and_pushes():
    """Raw mode (C = 1): integer input gives int64 sums; pushes and integrations
    partition the stream exactly."""
    rng = np.random.default_rng(23)
    x = rng.integers(-127, 128, (100, 3, 2)).astype(np.int8)
    out = oracle.correlator(x, 1, 1, push_sizes=[30, 30, 40], n_integrate=1)
    assert len(out) == 3
    tot = sum(o for o in out)
    assert np.array_equal(tot, oracle.correlate_int(x))
    out2 = oracle.correlator(x, 1, 1, push_sizes=[30, 30, 40], n_integrate=3)
    assert len(out2) == 1 and np.array_equal(out2[0], tot)


def test_correlator_streaming_equals_single_push():
    rng = np.random.default_rng(24)
    C, P = 16, 4
    x = rng.integers(-127, 128, (C * 30 + 7, 3, 2)).astype(np.int8)
    one = oracle.correlator(x, P, C)[0]
    parts = oracle.correlator(x, P, C, push_sizes=[100, 200, x.shape[0] - 300], n_integrate=3)[0]
    assert np.allclose(one, parts, rtol=1e-13, atol=1e-9)


def test_noise_expectation_loose():
    """E[V_ij] = 2 sigma^2 T delta_ij for white noise (sanity only)."""
    rng = np.random.default_rng(25)
    N, T, sig = 4, 20000, 2.0
    X = sig * (rng.standard_normal((1, N, T)) + 1j * rng.standard_normal((1, N, T)))
    V = oracle.correlate(X)[0] / T
    k = 0
    for i in range(N):
        for j in range(i + 1):
            ref = 2 * sig ** 2 if i == j else 0.0
            assert abs(V[k] - ref) < 0.1 * 2 * sig ** 2
            k += 1
