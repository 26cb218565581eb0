"""CPU oracle for the post-correlation steps of the AARTFAAC correlator stage
(arXiv 1609.04205): delay compensation, channel integration, lost-sample
weighting and sigma-clip flagging of the visibilities V.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s
reference leg; never by the product package.  Plain numpy in float64 /
int64, one step per function, written from the definitions below.  Shares
no code with the CUDA library.

Layouts follow the correlator output: V is [n_subbands, n_channels, NB]
complex with NB = N(N+1)/2 and baseline bl = i(i+1)/2 + j for i >= j
(V_ij = sum_t x_i conj(x_j)).
"""
from __future__ import annotations

import numpy as np


def pairs(N: int):
    """(i, j) of every packed baseline, in bl order."""
    i = np.repeat(np.arange(N), np.arange(1, N + 1))
    j = np.concatenate([np.arange(k + 1) for k in range(N)])
    return i, j


def channel_freqs(f_centre, sample_rate: float, n_channels: int) -> np.ndarray:
    """Sky frequency of every channel (Hz): [n_subbands, n_channels].

    The channeliser computes X_c = sum_n y[n] e^{-2 pi i c n / C} (natural
    order, no shift), so a baseband tone at +c fs / C lands in channel c:
    channel c sits at f_centre + c' fs / C with c' = c for 2c < C and
    c' = c - C otherwise (Sec. 4.2.3 filter bank; frequency order is a
    documented reading).  A single channel (raw subband) sits at f_centre."""
    C = int(n_channels)
    c = np.arange(C)
    off = np.where(2 * c < C, c, c - C) * (float(sample_rate) / C)
    return np.asarray(f_centre, dtype=np.float64)[:, None] + off[None, :]


def delay_compensate(V, delays, f_centre, sample_rate: float) -> np.ndarray:
    """Delay compensation as phase rotations of the visibilities (Sec. 4.2.4).

    An input delayed by d_i (x_i(t) = r(t - d_i)) carries e^{-2 pi i f d_i} at
    sky frequency f, so V_ij carries e^{-2 pi i f (d_i - d_j)}; compensation
    multiplies by the inverse: V_ij <- V_ij e^{+2 pi i f (d_i - d_j)}.
    delays: [N] seconds; f_centre: [n_subbands] Hz."""
    V = np.asarray(V, dtype=np.complex128)
    n_sb, C, NB = V.shape
    N = int(round((np.sqrt(8 * NB + 1) - 1) / 2))
    i, j = pairs(N)
    d = np.asarray(delays, dtype=np.float64)
    f = channel_freqs(f_centre, sample_rate, C)                      # [n_sb, C]
    phase = 2.0 * np.pi * f[:, :, None] * (d[i] - d[j])[None, None, :]
    return V * np.exp(1j * phase)


def integrate_channels(V, group: int) -> np.ndarray:
    """Channel integration to a coarser resolution (Sec. 4.2.4): output channel
    k is the sum of channels k*group ... k*group + group - 1.  With group
    dividing C/2 every group is contiguous in frequency (natural DFT order
    wraps at C/2).  Works for complex and for integer (re, im) int64 V."""
    V = np.asarray(V)
    n_sb, C = V.shape[0], V.shape[1]
    if C % group != 0:
        raise ValueError("group must divide n_channels")
    out_shape = (n_sb, C // group) + V.shape[2:]
    out = np.zeros(out_shape, dtype=V.dtype)
    for k in range(C // group):
        for g in range(group):
            out[:, k] += V[:, k * group + g]
    return out


def lost_sample_weights(mask, samples_per_block: int) -> np.ndarray:
    """Weighting matrix for lost data (Sec. 4.2.1 and the weighting step of
    Sec. 4.3): W_ij = samples_per_block * sum_b m_i[b] m_j[b], where m_i[b] is
    1 when input i's data of time block b arrived.  mask: [n_blocks, N] of
    0/1.  Returns int64 [NB], packed like V (autocorrelations included)."""
    m = np.asarray(mask).astype(np.int64)
    n_blocks, N = m.shape
    i, j = pairs(N)
    W = np.zeros(N * (N + 1) // 2, dtype=np.int64)
    for b in range(n_blocks):
        W += m[b, i] * m[b, j]
    return W * int(samples_per_block)


def reweight(V, W, n_total: int) -> np.ndarray:
    """Re-weighting of the visibilities for lost data: V_ij <- V_ij n_total / W_ij,
    and 0 where no sample pair survived (W_ij = 0).  V: [..., NB]; W: [NB]."""
    V = np.asarray(V, dtype=np.complex128)
    W = np.asarray(W, dtype=np.float64)
    scale = np.where(W > 0, float(n_total) / np.where(W > 0, W, 1.0), 0.0)
    return V * scale


def sigma_clip(V, k_chan: float, k_vis: float) -> np.ndarray:
    """Two-stage sigma-clip flagging of visibility amplitudes (the flagging
    step of Sec. 4.3).

    Stage 1, per spectral channel: RMS over the cross-correlations (i > j)
    of the channel, rms_c = sqrt(mean |V_ij|^2); flag |V_ij| > k_chan rms_c.
    Stage 2, per visibility across channels: RMS over the channels not
    flagged in stage 1, rms_ij = sqrt(mean |V_ij,c|^2); flag channel c when
    |V_ij,c| > k_vis rms_ij.  Autocorrelations are neither used nor flagged.
    Decisions compare squared amplitudes in float64: |V|^2 > k^2 * mean.
    Returns uint8 flags [n_subbands, n_channels, NB] (1 = flagged)."""
    V = np.asarray(V, dtype=np.complex128)
    n_sb, C, NB = V.shape
    N = int(round((np.sqrt(8 * NB + 1) - 1) / 2))
    i, j = pairs(N)
    cross = i != j
    p = V.real ** 2 + V.imag ** 2                                    # |V|^2
    flags = np.zeros(V.shape, dtype=np.uint8)
    n_cross = int(cross.sum())
    for s in range(n_sb):
        for c in range(C):
            ms = float(np.sum(p[s, c, cross])) / max(n_cross, 1)
            flags[s, c] = (cross & (p[s, c] > k_chan * k_chan * ms)).astype(np.uint8)
        for b in np.nonzero(cross)[0]:
            keep = flags[s, :, b] == 0
            n_keep = int(keep.sum())
            if n_keep == 0:
                continue
            ms = float(np.sum(p[s, keep, b])) / n_keep
            flags[s, keep, b] = (p[s, keep, b] > k_vis * k_vis * ms).astype(np.uint8)
    return flags
