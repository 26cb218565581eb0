"""CPU oracle for the AARTFAAC correlator stage (arXiv 1609.04205).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

The arithmetic lives in ``acf_oracle.c`` (fp64 / int64, plain definitions in
the paper's step order: FIR -> DFT -> bandpass -> transpose -> pair sums).
This module only marshals numpy arrays into it and strings the steps
together for whole streams.  It shares no code with the CUDA library.

The post-correlation steps (delay compensation, channel integration,
lost-sample weights, sigma-clip flagging) are plain numpy in ``post.py``.

Every function here has a pin in ``tests/test_oracle_*.py``; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp); returns the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        P = ctypes.c_void_p
        lib.oracle_prototype.argtypes = [i, i, P]
        lib.oracle_prototype.restype = i
        lib.oracle_n_spectra.argtypes = [l, i, i]
        lib.oracle_n_spectra.restype = l
        lib.oracle_channelise.argtypes = [P, l, i, P, i, i, P, l, l, P, i, P]
        lib.oracle_channelise.restype = i
        lib.oracle_correlate_f64.argtypes = [P, i, i, l, P]
        lib.oracle_correlate_f64.restype = None
        lib.oracle_correlate_i64.argtypes = [P, i, l, P]
        lib.oracle_correlate_i64.restype = None
        lib.oracle_gain.argtypes = [P, P, P, i, i, P]
        lib.oracle_gain.restype = d
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return _load().oracle_max_threads()


def prototype(n_taps: int, n_channels: int) -> np.ndarray:
    """Sec. 4.2.3 prototype: Hann-windowed sinc, length P*C, unit sum."""
    h = np.zeros(n_taps * n_channels, dtype=np.float64)
    if _load().oracle_prototype(n_taps, n_channels, _ptr(h)) != 0:
        raise ValueError("bad prototype arguments")
    return h


def n_spectra(length: int, n_taps: int, n_channels: int) -> int:
    """Number of complete FIR windows in ``length`` stream samples."""
    return int(_load().oracle_n_spectra(length, n_taps, n_channels))


def channelise(x, h, n_taps, n_channels, bandpass=None, m_begin=0, m_end=None, chans=None):
    """Direct FIR + naive DFT + bandpass for all inputs of one subband.

    x: [S, N] complex (any numeric dtype) or [S, N, 2] real pairs.
    Returns X: [len(chans), N, m_end - m_begin] complex128.
    """
    xr = _as_pairs_f64(x)
    S, N = xr.shape[0], xr.shape[1]
    C, P = n_channels, n_taps
    if m_end is None:
        m_end = n_spectra(S, P, C)
    chans = np.arange(C, dtype=np.int32) if chans is None else np.asarray(chans, dtype=np.int32)
    h = np.ascontiguousarray(h, dtype=np.float64)
    assert h.size == P * C
    w = None if bandpass is None else np.ascontiguousarray(bandpass, dtype=np.float64)
    T = m_end - m_begin
    X = np.zeros((chans.size, N, T, 2), dtype=np.float64)
    rc = _load().oracle_channelise(
        _ptr(xr), S, N, _ptr(h), P, C, None if w is None else _ptr(w), m_begin, m_end,
        _ptr(chans), chans.size, _ptr(X))
    if rc != 0:
        raise ValueError("window past the end of the stream")
    return X[..., 0] + 1j * X[..., 1]


def correlate(X) -> np.ndarray:
    """Brute-force pair sums. X: [n_ch, N, T] complex -> V: [n_ch, N(N+1)/2] complex128."""
    X = np.asarray(X)
    n_ch, N, T = X.shape
    Xr = np.ascontiguousarray(np.stack([X.real, X.imag], axis=-1), dtype=np.float64)
    V = np.zeros((n_ch, N * (N + 1) // 2, 2), dtype=np.float64)
    _load().oracle_correlate_f64(_ptr(Xr), n_ch, N, T, _ptr(V))
    return V[..., 0] + 1j * V[..., 1]


def correlate_int(x) -> np.ndarray:
    """Exact int64 pair sums of raw integer samples. x: [T, N, 2] integers -> [N(N+1)/2, 2] int64."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    T, N = x.shape[0], x.shape[1]
    V = np.zeros((N * (N + 1) // 2, 2), dtype=np.int64)
    _load().oracle_correlate_i64(_ptr(x), N, T, _ptr(V))
    return V


def gain_loss_grad(R, V, g):
    """Loss and d/dRe + i d/dIm gradient of sum_c ||G R_c G^H - V_c||_F^2.

    R, V: [C, N(N+1)/2] complex (packed lower triangles); g: [N] complex.
    """
    R = np.asarray(R)
    C, NB = R.shape
    N = int(round((np.sqrt(8 * NB + 1) - 1) / 2))
    Rr = np.ascontiguousarray(np.stack([R.real, R.imag], -1), dtype=np.float64)
    Vr = np.ascontiguousarray(np.stack([np.asarray(V).real, np.asarray(V).imag], -1), dtype=np.float64)
    gr = np.ascontiguousarray(np.stack([np.asarray(g).real, np.asarray(g).imag], -1), dtype=np.float64)
    grad = np.zeros((N, 2), dtype=np.float64)
    L = _load().oracle_gain(_ptr(Rr), _ptr(Vr), _ptr(gr), N, C, _ptr(grad))
    return L, grad[:, 0] + 1j * grad[:, 1]


def _as_pairs_f64(x) -> np.ndarray:
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1), dtype=np.float64)
    if x.ndim >= 1 and x.shape[-1] == 2:
        return np.ascontiguousarray(x, dtype=np.float64)
    raise ValueError("expected complex samples or trailing (re, im) axis")


def push_spectra(push_sizes, n_taps, n_channels):
    """Spectra produced by each push of a continuous stream.

    Spectrum m is emitted by the push in which its window [mC, mC + PC)
    becomes complete.  Returns a list of (m_begin, m_end) per push.
    """
    out, total, done = [], 0, 0
    for s in push_sizes:
        total += int(s)
        m_now = n_spectra(total, n_taps, n_channels)
        out.append((done, m_now))
        done = m_now
    return out


def correlator(samples, n_taps, n_channels, push_sizes=None, n_integrate=1, bandpass=None,
               chans=None, inputs=None):
    """Whole correlator stage for one subband stream.

    samples: [S, N, 2] integers or floats (or [S, N] complex), the concatenated
    stream of all pushes.  Channelised mode when n_channels > 1; raw mode
    (no filter bank, exact integer sums for integer input) when n_channels == 1.
    Returns a list, one entry per completed integration, of V arrays
    [len(chans), NB] (complex128, or int64 pairs [NB, 2] in raw integer mode).
    ``inputs`` restricts the correlated inputs to a subset (sampled parity).
    """
    x = np.asarray(samples)
    S = x.shape[0]
    if push_sizes is None:
        push_sizes = [S]
    assert sum(push_sizes) == S
    if inputs is not None:
        x = x[:, inputs]
    raw = n_channels == 1
    integer = raw and np.issubdtype(x.dtype, np.integer)
    spans = push_spectra(push_sizes, n_taps if not raw else 1, n_channels)
    h = prototype(n_taps if not raw else 1, n_channels)
    results, acc, count = [], None, 0
    for (m0, m1) in spans:
        if integer:
            part = correlate_int(x[m0:m1])
        elif raw:
            X = _as_pairs_f64(x[m0:m1])
            Xc = (X[..., 0] + 1j * X[..., 1]).T[None]
            part = correlate(Xc)
        else:
            X = channelise(x, h, n_taps, n_channels, bandpass, m0, m1, chans)
            part = correlate(X)
        acc = part if acc is None else acc + part
        count += 1
        if count == n_integrate:
            results.append(acc)
            acc, count = None, 0
    return results
