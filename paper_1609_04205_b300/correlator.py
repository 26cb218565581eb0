"""Streaming correlator, ragged batch and stateless steps over the C ABI.

PyTorch supplies device memory and streams; the work runs in libacf.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as A


def n_baselines(n_inputs: int) -> int:
    return n_inputs * (n_inputs + 1) // 2


def _vis_dtype(mode: str):
    return torch.int64 if mode == "int8" else torch.float32


class Correlator:
    """One correlator context (Sec. 4.2): push subband blocks, read integrated
    visibilities [n_subbands, n_channels, NB] (complex64, or int64 (re, im)
    pairs in INT8 mode)."""

    def __init__(self, n_inputs, n_subbands=1, n_channels=64, n_taps=16, n_integrate=1,
                 mode="fp32", dtype="ci8", max_samples=1 << 16, variant=None):
        self._L = A.lib()
        self.n_inputs, self.n_subbands, self.n_channels = n_inputs, n_subbands, n_channels
        self.n_taps, self.n_integrate, self.mode, self.dtype = n_taps, n_integrate, mode, dtype
        self.max_samples = max_samples
        h = ctypes.c_void_p()
        st = self._L.acf_create(ctypes.byref(h), n_inputs, n_subbands, n_channels, n_taps, n_integrate,
                                A.MODES[mode], A.DTYPES[dtype], max_samples)
        A.check(st, None)
        self._h = h
        if variant is not None:
            self.set_xengine_variant(variant)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self._L.acf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration
    def set_bandpass(self, w):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        A.check(self._L.acf_set_bandpass(self._h, w.ctypes.data_as(ctypes.c_void_p)), self._h)

    def set_xengine_variant(self, variant: int):
        """0: one SM per tile; 1: SM pairs sharing each 256x256 tile (cta_group::2)."""
        A.check(self._L.acf_set_xengine_variant(self._h, int(variant)), self._h)

    def tune(self):
        """Time every X-engine launch shape on this geometry and keep the
        fastest (acf_tune); only between integrations.  Returns xengine_tuning()."""
        A.check(self._L.acf_tune(self._h), self._h)
        return self.xengine_tuning()

    def xengine_tuning(self) -> dict:
        """The X-engine launch shape in use (acf_query_xengine)."""
        v, nt, ks, tu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        A.check(self._L.acf_query_xengine(self._h, ctypes.byref(v), ctypes.byref(nt), ctypes.byref(ks),
                                          ctypes.byref(tu)), self._h)
        return dict(variant=v.value, n_tile=nt.value, k_split=ks.value, tuned=bool(tu.value))

    def set_delays(self, delays, f_centre, sample_rate: float):
        """Delay-compensate every integration handed out from now on (acf_set_delays);
        delays=None switches it off."""
        import numpy as np
        if delays is None:
            A.check(self._L.acf_set_delays(self._h, None, None, 0.0), self._h)
            return
        d = np.ascontiguousarray(np.asarray(delays, dtype=np.float64))
        f = np.ascontiguousarray(np.asarray(f_centre, dtype=np.float64))
        A.check(self._L.acf_set_delays(self._h, d.ctypes.data_as(ctypes.c_void_p), f.ctypes.data_as(ctypes.c_void_p),
                                       float(sample_rate)), self._h)

    def set_input_scale(self, s: float):
        A.check(self._L.acf_set_input_scale(self._h, float(s)), self._h)

    # -- data path
    def push(self, samples: torch.Tensor, stream=None):
        """samples: [n_subbands, n_samples, n_inputs, 2] of the context dtype, on the
        device (or on the host: copied through the library's staging path)."""
        assert samples.is_contiguous()
        S = samples.shape[1]
        if samples.is_cuda:
            st = self._L.acf_push_block(self._h, A.ptr(samples), S, A.stream_handle(stream))
        else:
            st = self._L.acf_push_block_host(self._h, A.ptr(samples), S, A.stream_handle(stream))
        A.check(st, self._h)

    def empty_visibilities(self, device="cuda"):
        dt = _vis_dtype(self.mode)
        return torch.empty((self.n_subbands, self.n_channels, n_baselines(self.n_inputs), 2), dtype=dt,
                           device=device)

    def visibilities(self, out: torch.Tensor | None = None, stream=None):
        """Completed integration or None.  Float modes return complex64."""
        if out is None:
            out = self.empty_visibilities()
        n = ctypes.c_int(0)
        A.check(self._L.acf_get_visibilities(self._h, A.ptr(out), ctypes.byref(n), A.stream_handle(stream)),
                self._h)
        if n.value == 0:
            return None
        return torch.view_as_complex(out) if out.dtype == torch.float32 else out

    def release(self, stream=None) -> bool:
        """Finish the completed integration in place without copying it
        (acf_release_visibilities); True when one was complete.  Read it with
        device_visibilities() before the next push (in stream order)."""
        n = ctypes.c_int(0)
        A.check(self._L.acf_release_visibilities(self._h, ctypes.byref(n), A.stream_handle(stream)), self._h)
        return n.value == 1

    def device_visibilities(self) -> torch.Tensor:
        """Zero-copy view of the accumulator (acf_visibilities_device): complex64
        [subbands][channels][baselines], or int64 [..][2] in INT8 mode."""
        p = ctypes.c_void_p()
        A.check(self._L.acf_visibilities_device(self._h, ctypes.byref(p)), self._h)
        nb = self.n_inputs * (self.n_inputs + 1) // 2
        int8 = self.mode == "int8"
        view = _DeviceArray(p.value, (self.n_subbands, self.n_channels, nb, 2), "<i8" if int8 else "<f4")
        t = torch.as_tensor(view, device="cuda")
        return t if int8 else torch.view_as_complex(t)

    def enable_timing(self, on=True):
        A.check(self._L.acf_enable_timing(self._h, 1 if on else 0), self._h)

    def last_timing(self):
        """(channeliser ms, X-engine ms) of the last push (CUDA events)."""
        a, b = ctypes.c_float(), ctypes.c_float()
        A.check(self._L.acf_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    def query(self):
        T, ts, sc = ctypes.c_long(), ctypes.c_long(), ctypes.c_float()
        A.check(self._L.acf_query(self._h, ctypes.byref(T), ctypes.byref(ts), ctypes.byref(sc)), self._h)
        return dict(last_spectra=T.value, t_stride=ts.value, scale=sc.value)


def prototype(n_taps: int, n_channels: int):
    import numpy as np
    h = np.zeros(n_taps * n_channels, dtype=np.float32)
    A.check(A.lib().acf_prototype(n_taps, n_channels, h.ctypes.data_as(ctypes.c_void_p)))
    return h


def channelise(samples, n_channels, n_taps, out_kind="f32", bandpass=None, hist=None, scale=1.0,
               stream=None):
    """Stateless channeliser: samples [n_sb, S, N, 2] on the device ->
    (X, X_lo, T) with X [n_sb, C, 2N, t_stride] (float32 or float16)."""
    L = A.lib()
    n_sb, S, N = samples.shape[0], samples.shape[1], samples.shape[2]
    dt = {torch.int8: "ci8", torch.int16: "ci16", torch.float32: "cf32"}[samples.dtype]
    Hn = 0 if hist is None else hist.shape[1]
    total = Hn + S
    PC = n_taps * n_channels
    T = 0 if total < PC else (total - PC) // n_channels + 1
    ts = max(64, (T + 63) // 64 * 64)
    dev = samples.device
    h = torch.as_tensor(prototype(n_taps, n_channels), device=dev)
    bp = torch.ones(n_channels, dtype=torch.float32, device=dev) if bandpass is None else \
        torch.as_tensor(bandpass, dtype=torch.float32, device=dev)
    kind = {"f32": A.OUT_F32, "f16": A.OUT_F16, "f16x3": A.OUT_F16X3}[out_kind]
    xdt = torch.float32 if kind == A.OUT_F32 else torch.float16
    X = torch.zeros((n_sb, n_channels, 2 * N, ts), dtype=xdt, device=dev)
    Xlo = torch.zeros_like(X) if kind == A.OUT_F16X3 else None
    Tout = ctypes.c_long(0)
    st = L.acf_channelise(A.ptr(hist), Hn, A.ptr(samples), S, A.DTYPES[dt], n_sb, N, n_channels, n_taps,
                          A.ptr(h), A.ptr(bp), kind, A.ptr(X), A.ptr(Xlo), ts, float(scale), ctypes.byref(Tout),
                          A.stream_handle(stream))
    A.check(st)
    return X, Xlo, Tout.value


def transpose_raw(samples, out_kind="f16", scale=1.0, stream=None):
    L = A.lib()
    n_sb, S, N = samples.shape[0], samples.shape[1], samples.shape[2]
    dt = {torch.int8: "ci8", torch.int16: "ci16", torch.float32: "cf32"}[samples.dtype]
    ts = (S + 63) // 64 * 64
    kind = {"f32": A.OUT_F32, "f16": A.OUT_F16, "f16x3": A.OUT_F16X3}[out_kind]
    xdt = torch.float32 if kind == A.OUT_F32 else torch.float16
    X = torch.zeros((n_sb, 2 * N, ts), dtype=xdt, device=samples.device)
    Xlo = torch.zeros_like(X) if kind == A.OUT_F16X3 else None
    A.check(L.acf_transpose_raw(A.ptr(samples), S, A.DTYPES[dt], n_sb, N, kind, A.ptr(X), A.ptr(Xlo), ts,
                                float(scale), A.stream_handle(stream)))
    return X, Xlo


def xengine(mode, X, X_lo, n_inputs, n_time, vscale=1.0, V=None, stream=None):
    """Stateless X-engine on an operand [problems..., 2N, t_stride]; accumulates into V."""
    L = A.lib()
    ts = X.shape[-1]
    n_problems = X.numel() // (2 * n_inputs * ts)
    if V is None:
        V = torch.zeros((n_problems, n_baselines(n_inputs), 2), dtype=_vis_dtype(mode), device=X.device)
    A.check(L.acf_xengine(A.MODES[mode], A.ptr(X), A.ptr(X_lo), n_problems, n_inputs, n_time, ts, float(vscale),
                          A.ptr(V), A.stream_handle(stream)))
    return V


class Batch:
    """Ragged batch of independent arrays in one persistent launch (CUDA graph)."""

    def __init__(self, jobs, autotune=False):
        self._L = A.lib()
        arr = (A.Job * len(jobs))()
        for k, j in enumerate(jobs):
            arr[k] = A.Job(j["n_inputs"], j["n_channels"], j["n_taps"], j["n_samples"])
        h = ctypes.c_void_p()
        st = self._L.acf_batch_create(ctypes.byref(h), arr, len(jobs), 1 if autotune else 0)
        A.check(st, batch=None if st != A.OK else h)
        self._h = h
        self.jobs = [dict(j) for j in jobs]

    def outputs(self, device="cuda"):
        outs = []
        for j in self.jobs:
            dt = torch.int64 if j["n_channels"] == 1 else torch.float32
            outs.append(torch.empty((j["n_channels"], n_baselines(j["n_inputs"]), 2), dtype=dt, device=device))
        return outs

    def run(self, inputs, outputs, stream=None):
        n = len(self.jobs)
        ins = (ctypes.c_void_p * n)(*[t.data_ptr() for t in inputs])
        outs = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outputs])
        A.check(self._L.acf_batch_run(self._h, ins, outs, A.stream_handle(stream)), batch=self._h)

    def query(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        A.check(self._L.acf_batch_query(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), batch=self._h)
        pr, od = ctypes.c_int(), ctypes.c_int()
        A.check(self._L.acf_batch_query_plan(self._h, ctypes.byref(pr), ctypes.byref(od)), batch=self._h)
        return dict(n_tile=a.value, k_split=b.value, n_items=c.value, pair=pr.value, order=od.value)

    def set_plan(self, pair, n_tile, k_split, order):
        """Fix the X-engine plan (see acf_batch_set_plan) instead of autotuning."""
        A.check(self._L.acf_batch_set_plan(self._h, int(pair), int(n_tile), int(k_split), int(order)), batch=self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.acf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """__cuda_array_interface__ over a device pointer the library owns (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=tuple(shape), typestr=typestr, data=(int(ptr), False),
                                             version=3, strides=None)


def launch_count() -> int:
    return int(A.lib().acf_launch_count())


def probe_tensor_peak(k_steps: int = 16384) -> dict:
    """Tensor-pipe rate with operands resident in shared memory
    (acf_probe_tensor_peak): kind::f16 MMAs M = 128, N = 256 on every SM."""
    tf, ms = ctypes.c_double(), ctypes.c_float()
    A.check(A.lib().acf_probe_tensor_peak(int(k_steps), ctypes.byref(tf), ctypes.byref(ms)), None)
    return dict(tflops=tf.value, ms=ms.value, k_steps=int(k_steps))


def device_status() -> int:
    return int(A.lib().acf_device_status())
