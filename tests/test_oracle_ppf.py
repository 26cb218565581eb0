"""Pins for the oracle's polyphase filter bank (Sec. 4.2.3) and bandpass
(Sec. 4.2.4).  Each expected value comes from a closed form, a different
library route (numpy FFT) or a statistical identity -- never from the oracle
itself or from the CUDA path."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("P,C", [(16, 64), (16, 16), (16, 256), (4, 8), (1, 1)])
def test_prototype_shape(P, C):
    h = oracle.prototype(P, C)
    L = P * C
    assert h.shape == (L,)
    assert abs(h.sum() - 1.0) < 1e-13                      # unit DC gain
    if L > 1:
        assert np.allclose(h, h[::-1], atol=1e-16)          # symmetric (linear phase)
        assert h[0] == 0.0 and abs(h[-1]) < 1e-18           # Hann end points
        # the sinc's zeros: h vanishes wherever (n - (L-1)/2)/C is a non-zero integer
        # (only when L-1 is even does the centre fall on a sample); peak at centre
        mid = (L - 1) / 2
        assert np.argmax(h) in (int(np.floor(mid)), int(np.ceil(mid)))


def test_prototype_closed_form_values():
    # L = 8, C = 4: u = (n - 3.5)/4, w = 0.5 - 0.5 cos(2 pi n / 7)
    h = oracle.prototype(2, 4)
    n = np.arange(8)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * n / 7)
    u = (n - 3.5) / 4
    ref = w * np.sin(np.pi * u) / (np.pi * u)
    ref /= ref.sum()
    assert np.allclose(h, ref, rtol=0, atol=1e-15)


def _tone(S, C, nu, A=1.0 + 0.5j):
    t = np.arange(S)
    return (A * np.exp(2j * np.pi * nu * t / C))[:, None]


@pytest.mark.parametrize("C,P,c0", [(64, 16, 5), (16, 16, 15), (8, 4, 0)])
def test_pure_tone_on_bin(C, P, c0):
    """A tone on channel c0 lands there with amplitude exactly A (sum h = 1);
    every other channel c sees the filter's response at integer offset
    c0 - c, H(k) = sum_l h[l] exp(2 pi i k l / C), taken from numpy's FFT."""
    A = 1.0 + 0.5j
    S = (P + 6) * C
    h = oracle.prototype(P, C)
    X = oracle.channelise(_tone(S, C, c0, A), h, P, C)       # [C, 1, T]
    T = X.shape[2]
    assert T == oracle.n_spectra(S, P, C) == 7
    assert np.allclose(X[c0, 0], A, atol=1e-12)
    Hf = np.conj(np.fft.fft(h))                              # Hf[q] = sum h e^{+2 pi i q l / L}
    for c in range(C):
        k = (c0 - c) % C
        assert np.allclose(X[c, 0], A * Hf[(k * P) % (P * C)], atol=1e-12)


def test_pure_tone_off_bin_leakage():
    """Tone at c0 + 1/4: X_c[m] = A e^{2 pi i (c0+d) m} H(c0 + d - c), with H
    from a 4x zero-padded numpy FFT of h."""
    C, P, c0, d = 32, 8, 3, 0.25
    A = 2.0 - 1.0j
    S = (P + 5) * C
    h = oracle.prototype(P, C)
    X = oracle.channelise(_tone(S, C, c0 + d, A), h, P, C)
    Z = 4
    Hf = np.conj(np.fft.fft(h, n=P * C * Z))
    m = np.arange(X.shape[2])
    for c in range(C):
        nu = c0 + d - c
        q = int(round(nu * P * Z)) % (P * C * Z)
        ref = A * np.exp(2j * np.pi * (c0 + d) * m) * Hf[q]
        assert np.allclose(X[c, 0], ref, atol=1e-12)


def test_impulse_asymmetric_filter():
    """An impulse at t0 gives X_c[m] = h[t0 - mC] e^{-2 pi i c t0 / C}.  A random,
    non-symmetric filter makes a reversed or shifted tap index fail."""
    rng = np.random.default_rng(7)
    C, P = 16, 4
    h = rng.standard_normal(P * C)
    S = 10 * C
    for t0 in (0, 5, 37, 63, 100):
        x = np.zeros((S, 1), complex)
        x[t0, 0] = 1.0
        X = oracle.channelise(x, h, P, C)
        T = X.shape[2]
        for m in range(T):
            l = t0 - m * C
            for c in range(C):
                ref = h[l] * np.exp(-2j * np.pi * c * t0 / C) if 0 <= l < P * C else 0.0
                assert abs(X[c, 0, m] - ref) < 1e-12


def test_random_input_matches_numpy_fft_route():
    """Same FIR, but the DFT taken by numpy's FFT instead of the naive sum."""
    rng = np.random.default_rng(3)
    C, P, N, S = 64, 16, 3, 64 * 24 + 17
    x = rng.standard_normal((S, N)) + 1j * rng.standard_normal((S, N))
    h = oracle.prototype(P, C)
    X = oracle.channelise(x, h, P, C)
    T = X.shape[2]
    hk = h.reshape(P, C)
    for n in range(N):
        for m in range(T):
            seg = x[m * C:(m + P) * C, n].reshape(P, C)
            y = (hk * seg).sum(axis=0)
            assert np.allclose(X[:, n, m], np.fft.fft(y), atol=1e-11)


def test_channel_subset_and_time_window():
    rng = np.random.default_rng(4)
    C, P, S = 16, 4, 16 * 30
    x = rng.integers(-127, 128, (S, 2, 2)).astype(np.int8)
    h = oracle.prototype(P, C)
    full = oracle.channelise(x, h, P, C)
    part = oracle.channelise(x, h, P, C, m_begin=5, m_end=20, chans=[3, 0, 15])
    assert np.array_equal(part, full[[3, 0, 15]][:, :, 5:20])


def test_bandpass_scales_channel_power():
    rng = np.random.default_rng(5)
    C, P, S = 16, 4, 16 * 40
    x = rng.standard_normal((S, 2)) + 1j * rng.standard_normal((S, 2))
    h = oracle.prototype(P, C)
    w = np.linspace(0.5, 2.0, C)
    a = oracle.channelise(x, h, P, C)
    b = oracle.channelise(x, h, P, C, bandpass=w)
    assert np.allclose(b, a * w[:, None, None], atol=1e-12)


def test_white_noise_channel_power():
    """E|X_c|^2 = 2 sigma^2 sum h^2 for white complex noise (statistical, 5%)."""
    rng = np.random.default_rng(6)
    C, P, sig = 16, 8, 3.0
    S = C * 4000
    x = sig * (rng.standard_normal((S, 1)) + 1j * rng.standard_normal((S, 1)))
    h = oracle.prototype(P, C)
    X = oracle.channelise(x, h, P, C)
    pw = (np.abs(X) ** 2).mean(axis=(1, 2))
    assert np.allclose(pw, 2 * sig ** 2 * (h ** 2).sum(), rtol=0.05)


def test_window_past_end_rejected():
    h = oracle.prototype(4, 8)
    x = np.zeros((40, 1), complex)
    with pytest.raises(ValueError):
        oracle.channelise(x, h, 4, 8, m_begin=0, m_end=3)
    assert oracle.n_spectra(40, 4, 8) == 2
    assert oracle.n_spectra(31, 4, 8) == 0


def test_push_spectra_streaming():
    # 19,532 samples, 16 taps x 64 channels: floor((S - 15*64)/64) = 290 spectra
    assert oracle.push_spectra([19532], 16, 64) == [(0, 290)]
    spans = oracle.push_spectra([1000, 1000, 64, 5], 16, 64)
    assert spans == [(0, 0), (0, 16), (16, 17), (17, 17)]
