"""Seeded synthetic voltage generators shaped like the AARTFAAC arrays.

Shared by the tests, the benchmark and the oracle checks; it holds none of
the correlator's arithmetic (no filter bank, no DFT, no pair sums).  It only
draws the inputs: complex Gaussian noise plus narrow-band point sources seen
by dual-polarisation antennas scattered over a LOFAR station footprint, then
quantised to the station's complex int8 / int16 sample formats.

Signal model (the paper gives shapes, not signals; these are the readings):
  * 48 dual-pol antennas per station (Sec. 2.1), input index = 2*antenna + pol;
  * antenna positions uniform in a disc of diameter 60 m (Sec. 2.1);
  * each point source has direction cosines (l, m) drawn uniformly with
    l^2 + m^2 <= 0.8^2, per-component amplitude std ``flux * sigma`` and
    independent streams per polarisation (unpolarised);
  * geometric phase per antenna phi = -2 pi f (x l + y m) / c at the subband
    centre f (subband 300 + k, 195312.5 Hz wide, Sec. 2.2), applied to the
    complex baseband (narrow-band approximation);
  * receiver noise: per-component std ``sigma``;
  * quantisation: round half away from zero, then clip to +-127 (ci8) or
    +-32767 (ci16); cf32 keeps the floats.

Generation is chunked over subbands and time so full-size inputs (tens of GB)
can be drawn directly on the GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SUBBAND_HZ = 195312.5
C_LIGHT = 299792458.0
FIRST_SUBBAND = 300


@dataclass
class Sky:
    positions: np.ndarray            # [n_ant, 2] metres
    lm: np.ndarray                   # [n_src, 2] direction cosines
    flux: np.ndarray                 # [n_src] in units of sigma
    extra: dict = field(default_factory=dict)


def make_sky(n_inputs: int, n_sources: int, flux, seed: int) -> Sky:
    """Antenna layout and source list, drawn from ``seed``.

    ``flux`` is a scalar (every source) or a (lo, hi) range drawn uniformly.
    """
    rng = np.random.default_rng(seed)
    n_ant = (n_inputs + 1) // 2
    r = 30.0 * np.sqrt(rng.random(n_ant))
    th = 2 * np.pi * rng.random(n_ant)
    pos = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    rs = 0.8 * np.sqrt(rng.random(n_sources))
    ts = 2 * np.pi * rng.random(n_sources)
    lm = np.stack([rs * np.cos(ts), rs * np.sin(ts)], axis=1)
    if np.isscalar(flux):
        fl = np.full(n_sources, float(flux))
    else:
        fl = rng.uniform(float(flux[0]), float(flux[1]), n_sources)
    return Sky(pos, lm, fl)


def geometric_phase(sky: Sky, subband: int) -> np.ndarray:
    """[n_src, n_ant] phase of each source at each antenna (radians)."""
    f = (FIRST_SUBBAND + subband) * SUBBAND_HZ
    return -2 * np.pi * f * (sky.lm @ sky.positions.T) / C_LIGHT


def voltages(n_inputs: int, n_samples: int, n_subbands: int = 1, dtype: str = "ci8",
             sigma: float = 16.0, sky: Sky | None = None, seed: int = 0,
             device="cpu", out: torch.Tensor | None = None,
             chunk: int = 1 << 16) -> torch.Tensor:
    """Draw [n_subbands, n_samples, n_inputs, 2] samples (re, im last).

    dtype: "ci8" (int8), "ci16" (int16) or "cf32" (float32).
    The same (seed, shapes) give the same values on a given device type.
    """
    tdt = {"ci8": torch.int8, "ci16": torch.int16, "cf32": torch.float32}[dtype]
    lim = {"ci8": 127.0, "ci16": 32767.0, "cf32": None}[dtype]
    if out is None:
        out = torch.empty((n_subbands, n_samples, n_inputs, 2), dtype=tdt, device=device)
    dev = out.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    n_ant = (n_inputs + 1) // 2
    ant_of_input = torch.arange(n_inputs, device=dev) // 2
    pol_of_input = torch.arange(n_inputs, device=dev) % 2
    for sb in range(n_subbands):
        if sky is not None and len(sky.flux):
            ph = torch.as_tensor(geometric_phase(sky, sb), dtype=torch.float64, device=dev)
            rot = torch.polar(torch.ones_like(ph), ph).to(torch.complex64)   # [n_src, n_ant]
            rot_in = rot[:, ant_of_input]                                    # [n_src, n_inputs]
            amp = torch.as_tensor(sky.flux, dtype=torch.float32, device=dev) * sigma
        for t0 in range(0, n_samples, chunk):
            t1 = min(n_samples, t0 + chunk)
            nt = t1 - t0
            v = torch.randn((nt, n_inputs, 2), generator=gen, device=dev, dtype=torch.float32)
            v.mul_(sigma)
            if sky is not None and len(sky.flux):
                vc = torch.view_as_complex(v)
                for s in range(len(sky.flux)):
                    sx = torch.randn((nt, 2, 2), generator=gen, device=dev, dtype=torch.float32)
                    sx = torch.view_as_complex(sx.mul_(float(amp[s])))         # [nt, 2 pols]
                    vc += sx[:, pol_of_input] * rot_in[s][None, :]
            if lim is not None:
                v = torch.sign(v) * torch.floor(v.abs() + 0.5)
                v.clamp_(-lim, lim)
            out[sb, t0:t1].copy_(v.to(tdt))
    return out


def unit_gains(n_inputs: int, seed: int, device="cpu") -> torch.Tensor:
    """Per-input complex gains, amplitude U(0.8, 1.2), phase U(-pi, pi)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.8, 1.2, n_inputs)
    p = rng.uniform(-np.pi, np.pi, n_inputs)
    return torch.as_tensor(a * np.exp(1j * p), dtype=torch.complex64, device=device)


def bandpass_ripple(n_channels: int, seed: int) -> np.ndarray:
    """Positive per-channel weights standing in for the station filter's
    deterministic bandpass correction (the real tables are not published)."""
    rng = np.random.default_rng(seed)
    c = np.arange(n_channels)
    return (1.0 + 0.1 * np.cos(2 * np.pi * c / max(n_channels, 1)) + 0.02 * rng.standard_normal(n_channels)).astype(np.float32)


# Workloads shaped like the paper's arrays (Sec. 2.1, 4, Table 1).
WORKLOADS = {
    "tiny": dict(n_inputs=96, n_subbands=1, n_samples=19532, dtype="ci8", sigma=16.0,
                 n_channels=64, n_taps=16, n_sources=1, flux=0.2, seed=1001),
    "a6": dict(n_inputs=576, n_subbands=8, n_samples=195313, dtype="ci8", sigma=16.0,
               n_channels=64, n_taps=16, n_sources=0, flux=0.0, seed=1002),
    "a12": dict(n_inputs=1152, n_subbands=16, n_samples=195313, dtype="ci16", sigma=512.0,
                n_channels=64, n_taps=16, n_sources=3, flux=(0.05, 0.5), seed=1003),
    "gain": dict(n_inputs=576, n_subbands=1, n_samples=97656, dtype="cf32", sigma=1.0,
                 n_channels=64, n_taps=16, n_sources=5, flux=(0.2, 1.0), seed=1005),
}


def ragged_jobs(seed: int = 1004, n_jobs: int = 32):
    """32 independent arrays: antennas from {48, 96, 192, 288, 576} (dual-pol),
    channels from {16, 64, 256}, 0.25 s (48,828 samples) of ci8 each; each job
    is raw-subband (INT8 exact) or channelised (split FP16) with probability 1/2."""
    rng = np.random.default_rng(seed)
    ants = rng.choice([48, 96, 192, 288, 576], size=n_jobs)
    chans = rng.choice([16, 64, 256], size=n_jobs)
    raw = rng.random(n_jobs) < 0.5
    jobs = []
    for k in range(n_jobs):
        jobs.append(dict(n_inputs=int(2 * ants[k]), n_channels=1 if raw[k] else int(chans[k]),
                         n_taps=1 if raw[k] else 16, n_samples=48828, seed=seed * 100 + k,
                         raw=bool(raw[k])))
    return jobs
