"""Pins of the post-correlation oracle (oracle/post.py) against closed forms,
independent formulations and planted cases (no GPU)."""
import numpy as np
import pytest

import oracle
from oracle import post


FS = 195312.5          # subband sample rate (Hz), Sec. 2
F_SB = 300 * FS        # a subband centre in the LBA band


def _tone_inputs(c0, C, delays, S):
    """Inputs carrying one bin-centred tone, each delayed by d_i seconds before
    down-conversion: x_i[t] = e^{2 pi i nu (t/fs - d_i)} e^{-2 pi i f_sb d_i},
    with nu the tone's physical baseband frequency (negative for c0 >= C/2)."""
    nu = (c0 if c0 < C // 2 else c0 - C) * FS / C
    t = np.arange(S) / FS
    x = np.exp(2j * np.pi * nu * (t[:, None] - delays[None, :])) * np.exp(-2j * np.pi * F_SB * delays[None, :])
    return np.stack([x.real, x.imag], axis=-1)


@pytest.mark.parametrize("c0", [3, 13])
def test_delay_compensation_cancels_fractional_delays(c0):
    """End to end through the pinned channeliser and pair sums: a tone whose
    inputs are delayed by fractional samples gives V_ij with phase
    -2 pi f (d_i - d_j) in its channel; compensation leaves it real and equal
    to the autocorrelations.  The fractional delays make the sign, the pair
    orientation and the negative-frequency channel map all matter."""
    C, P, N = 16, 4, 5
    d = np.array([0.0, 0.31, 1.7, 4.05, 9.9]) / FS
    x = _tone_inputs(c0, C, d, S=C * 40)
    h = oracle.prototype(P, C)
    X = oracle.channelise(x, h, P, C)                 # [C, N, T]
    V = oracle.correlate(X)[None]                     # [1, C, NB]
    out = post.delay_compensate(V, d, [F_SB], FS)
    Vc = out[0, c0]
    i, j = post.pairs(N)
    auto = Vc[i == j].real
    assert np.max(np.abs(np.angle(Vc[i != j]))) < 1e-9
    assert np.allclose(np.abs(Vc), auto[0], rtol=1e-9)
    # without compensation the phases are the expected -2 pi f (d_i - d_j)
    f = post.channel_freqs([F_SB], FS, C)[0, c0]
    want = np.exp(-2j * np.pi * f * (d[i] - d[j]))
    assert np.allclose(V[0, c0] / np.abs(V[0, c0]), want, atol=1e-9)


def test_delay_identity_and_roundtrip():
    rng = np.random.default_rng(1)
    N, C = 7, 8
    NB = N * (N + 1) // 2
    V = rng.normal(size=(2, C, NB)) + 1j * rng.normal(size=(2, C, NB))
    d = rng.uniform(-5e-6, 5e-6, N)
    fc = [F_SB, F_SB + FS]
    assert np.array_equal(post.delay_compensate(V, np.zeros(N), fc, FS), V)
    back = post.delay_compensate(post.delay_compensate(V, d, fc, FS), -d, fc, FS)
    assert np.allclose(back, V, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.abs(post.delay_compensate(V, d, fc, FS)), np.abs(V), rtol=1e-12)
    # autocorrelations are untouched
    i, j = post.pairs(N)
    assert np.allclose(post.delay_compensate(V, d, fc, FS)[..., i == j], V[..., i == j], rtol=1e-14)


def test_channel_freqs_natural_order():
    f = post.channel_freqs([F_SB], FS, 8)[0]
    assert f[0] == F_SB
    assert np.allclose(f - F_SB, np.array([0, 1, 2, 3, -4, -3, -2, -1]) * FS / 8)


@pytest.mark.parametrize("nu", [0.0, 0.37 * FS, -0.21 * FS])
def test_raw_subband_delay_compensation_at_subband_centre(nu):
    """A raw subband (one channel, no filter bank) is compensated at the
    subband centre frequency (Sec. 4.2.4).  Inputs delayed by fractional
    samples carry a baseband tone nu: x_i[t] = e^{2 pi i nu (t/fs - d_i)}
    e^{-2 pi i f_sb d_i}, so the raw pair sums carry -2 pi (f_sb + nu)
    (d_i - d_j), and compensation at f_sb must leave exactly -2 pi nu (d_i - d_j)
    (zero for a tone at the centre).  A channel placed one sample rate away
    (f_sb - fs) would leave 2 pi fs (d_i - d_j), which fractional delays make
    visible."""
    N, S = 5, 64
    d = np.array([0.0, 0.31, 1.7, 4.05, 9.9]) / FS
    t = np.arange(S) / FS
    x = np.exp(2j * np.pi * nu * (t[:, None] - d[None, :])) * np.exp(-2j * np.pi * F_SB * d[None, :])
    V = oracle.correlate(x.T[None])[None]                          # [1, 1, NB], raw subband
    assert np.allclose(post.channel_freqs([F_SB], FS, 1), [[F_SB]], rtol=0, atol=0)
    out = post.delay_compensate(V, d, [F_SB], FS)[0, 0]
    i, j = post.pairs(N)
    want = S * np.exp(-2j * np.pi * nu * (d[i] - d[j]))
    assert np.allclose(out, want, rtol=0, atol=1e-9 * S)
    if nu == 0.0:
        assert np.max(np.abs(out.imag)) < 1e-9 * S


def test_integrate_channels_against_reshape_sum():
    rng = np.random.default_rng(2)
    V = rng.normal(size=(3, 16, 10)) + 1j * rng.normal(size=(3, 16, 10))
    for g in (1, 2, 4, 8):
        want = V.reshape(3, 16 // g, g, 10).sum(axis=2)
        assert np.allclose(post.integrate_channels(V, g), want, rtol=1e-14, atol=1e-14)
    assert np.array_equal(post.integrate_channels(V, 1), V)


def test_integrate_channels_groups_are_frequency_contiguous():
    C = 64
    f = post.channel_freqs([0.0], FS, C)[0]
    for g in (2, 4, 8, 16, 32):            # divisors of C/2
        for k in range(C // g):
            fk = np.sort(f[k * g:(k + 1) * g])
            assert np.allclose(np.diff(fk), FS / C)


def test_integrate_channels_int64_exact():
    rng = np.random.default_rng(3)
    V = rng.integers(-2**40, 2**40, size=(2, 8, 6, 2), dtype=np.int64)
    got = post.integrate_channels(V, 4)
    for s in range(2):
        for k in range(2):
            for b in range(6):
                for r in range(2):
                    assert int(got[s, k, b, r]) == sum(int(V[s, 4 * k + g, b, r]) for g in range(4))


def test_weights_brute_force_and_special_cases():
    rng = np.random.default_rng(4)
    nb, N, spb = 9, 6, 16
    m = rng.integers(0, 2, size=(nb, N))
    W = post.lost_sample_weights(m, spb)
    i, j = post.pairs(N)
    for b, (a, c) in enumerate(zip(i, j)):
        assert int(W[b]) == spb * sum(int(m[t, a]) * int(m[t, c]) for t in range(nb))
    assert np.array_equal(W[i == j], spb * m.sum(axis=0))
    full = post.lost_sample_weights(np.ones((nb, N), dtype=np.uint8), spb)
    assert np.all(full == nb * spb)
    m2 = np.ones((nb, N), dtype=np.uint8)
    m2[:, 2] = 0
    W2 = post.lost_sample_weights(m2, spb)
    assert np.all(W2[(i == 2) | (j == 2)] == 0)


def test_reweight():
    V = np.array([[1 + 1j, 2.0, 3j]])
    W = np.array([10, 5, 0])
    out = post.reweight(V, W, 10)
    assert np.allclose(out, [[1 + 1j, 4.0, 0.0]])


def _unit_vis(rng, n_sb, C, N):
    """|V| = 1 everywhere with random phases (deterministic amplitudes)."""
    NB = N * (N + 1) // 2
    return np.exp(2j * np.pi * rng.uniform(size=(n_sb, C, NB)))


def test_sigma_clip_clean_data_has_no_flags():
    rng = np.random.default_rng(5)
    N, C = 12, 16
    NB = N * (N + 1) // 2
    V = rng.normal(size=(2, C, NB)) + 1j * rng.normal(size=(2, C, NB))
    assert post.sigma_clip(V, 50.0, 50.0).sum() == 0


def test_sigma_clip_planted_outliers():
    rng = np.random.default_rng(6)
    N, C = 10, 16
    V = _unit_vis(rng, 1, C, N)
    i, j = post.pairs(N)
    cross = np.nonzero(i != j)[0]
    b1, b2 = cross[3], cross[17]
    V[0, 5, b1] *= 1000.0           # stage 1: far above its channel's RMS
    V[0, 9, b2] *= 3.0              # stage 2 only: 9x power, below k_chan^2 = 25x
    auto = np.nonzero(i == j)[0][4]
    V[0, 2, auto] *= 1e6            # autocorrelations are never flagged
    F = post.sigma_clip(V, 5.0, 2.0)
    want = np.zeros_like(F)
    want[0, 5, b1] = 1
    want[0, 9, b2] = 1
    assert np.array_equal(F, want)


def test_sigma_clip_stage1_flags_leave_stage2_rms():
    """A channel flagged in stage 1 must not inflate the stage-2 RMS of its
    baseline: with it excluded a 3x channel is flagged, with it included
    (k_chan too high to flag it) the 3x channel survives."""
    rng = np.random.default_rng(7)
    N, C = 8, 16
    V = _unit_vis(rng, 1, C, N)
    i, j = post.pairs(N)
    b = np.nonzero(i != j)[0][5]
    V[0, 1, b] *= 1000.0
    V[0, 7, b] *= 3.0
    F = post.sigma_clip(V, 5.0, 2.0)
    assert F[0, 1, b] == 1 and F[0, 7, b] == 1
    F2 = post.sigma_clip(V, 1e9, 2.0)
    assert F2[0, 1, b] == 1 and F2[0, 7, b] == 0
