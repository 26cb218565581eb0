"""ctypes binding of libacf.so (the C ABI in include/acf.h).

Argument marshalling only: every step of the correlator runs in the
library's CUDA kernels.  There is no CPU fallback; when the shared library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libacf.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, EUNSUPPORTED = range(7)
IN_CI8, IN_CI16, IN_CF32 = 0, 1, 2
X_FP32, X_FP16, X_FP16x3, X_INT8 = 0, 1, 2, 3
OUT_F32, OUT_F16, OUT_F16X3 = 0, 1, 2

DTYPES = {"ci8": IN_CI8, "ci16": IN_CI16, "cf32": IN_CF32}
MODES = {"fp32": X_FP32, "fp16": X_FP16, "fp16x3": X_FP16x3, "int8": X_INT8}

# every symbol include/acf.h declares
EXPORTS = [
    "acf_create", "acf_set_bandpass", "acf_set_input_scale", "acf_push_block", "acf_push_block_host",
    "acf_get_visibilities", "acf_visibilities_device", "acf_query", "acf_destroy", "acf_last_error",
    "acf_status_string", "acf_prototype", "acf_channelise", "acf_transpose_raw", "acf_xengine",
    "acf_gain_forward", "acf_gain_backward", "acf_batch_create", "acf_batch_run", "acf_batch_query",
    "acf_batch_query_plan", "acf_batch_set_plan", "acf_batch_destroy", "acf_batch_last_error", "acf_launch_count", "acf_device_status", "acf_version",
    "acf_enable_timing", "acf_last_timing", "acf_gain_forward_noalloc", "acf_set_xengine_variant",
    "acf_delay_compensate", "acf_set_delays", "acf_integrate_channels", "acf_sigma_clip",
    "acf_lost_sample_weights", "acf_reweight", "acf_tune", "acf_query_xengine", "acf_probe_tensor_peak",
    "acf_release_visibilities",
]


class AcfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("acf status %d: %s" % (status, msg))
        self.status = status


class Job(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int), ("n_channels", ctypes.c_int), ("n_taps", ctypes.c_int),
                ("n_samples", ctypes.c_long)]


_lib = None


def build_if_needed():
    from . import build as _build
    return _build.build()


def lib():
    """Load libacf.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        try:
            build_if_needed()
        except Exception as e:  # no nvcc: fail loudly, never fall back
            raise RuntimeError("libacf.so is missing and could not be built: %s" % e) from e
    L = ctypes.CDLL(LIB_PATH)
    P, I, Lg, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_float
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "acf_create": ([ctypes.POINTER(P), I, I, I, I, I, I, I, Lg], I),
        "acf_set_bandpass": ([P, P], I),
        "acf_set_input_scale": ([P, F], I),
        "acf_push_block": ([P, P, Lg, P], I),
        "acf_push_block_host": ([P, P, Lg, P], I),
        "acf_get_visibilities": ([P, P, ctypes.POINTER(I), P], I),
        "acf_visibilities_device": ([P, PP], I),
        "acf_query": ([P, ctypes.POINTER(Lg), ctypes.POINTER(Lg), ctypes.POINTER(F)], I),
        "acf_destroy": ([P], I),
        "acf_last_error": ([P], ctypes.c_char_p),
        "acf_status_string": ([I], ctypes.c_char_p),
        "acf_prototype": ([I, I, P], I),
        "acf_channelise": ([P, Lg, P, Lg, I, I, I, I, I, P, P, I, P, P, Lg, F, ctypes.POINTER(Lg), P], I),
        "acf_transpose_raw": ([P, Lg, I, I, I, I, P, P, Lg, F, P], I),
        "acf_xengine": ([I, P, P, I, I, Lg, Lg, F, P, P], I),
        "acf_gain_forward": ([P, P, P, I, I, P, P, P], I),
        "acf_gain_backward": ([P, P, P, I, I, P, P], I),
        "acf_batch_create": ([ctypes.POINTER(P), ctypes.POINTER(Job), I, I], I),
        "acf_batch_run": ([P, PP, PP, P], I),
        "acf_batch_query": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "acf_batch_query_plan": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "acf_batch_set_plan": ([P, I, I, I, I], I),
        "acf_batch_destroy": ([P], I),
        "acf_batch_last_error": ([P], ctypes.c_char_p),
        "acf_launch_count": ([], ctypes.c_longlong),
        "acf_device_status": ([], I),
        "acf_version": ([], ctypes.c_char_p),
        "acf_enable_timing": ([P, I], I),
        "acf_last_timing": ([P, ctypes.POINTER(F), ctypes.POINTER(F)], I),
        "acf_gain_forward_noalloc": ([P, P, P, I, I, P, P, P], I),
        "acf_set_xengine_variant": ([P, I], I),
        "acf_tune": ([P], I),
        "acf_release_visibilities": ([P, ctypes.POINTER(I), P], I),
        "acf_probe_tensor_peak": ([Lg, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(F)], I),
        "acf_query_xengine": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "acf_delay_compensate": ([P, I, I, I, P, P, ctypes.c_double, P], I),
        "acf_set_delays": ([P, P, P, ctypes.c_double], I),
        "acf_integrate_channels": ([P, P, I, I, I, I, I, P], I),
        "acf_sigma_clip": ([P, P, I, I, I, ctypes.c_double, ctypes.c_double, P], I),
        "acf_lost_sample_weights": ([P, Lg, I, Lg, P, P], I),
        "acf_reweight": ([P, P, Lg, I, I, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def check(status: int, ctx=None, batch=None):
    if status != OK:
        L = lib()
        if batch is not None:
            msg = L.acf_batch_last_error(batch).decode()
        else:
            msg = L.acf_last_error(ctx).decode()
        if not msg:
            msg = L.acf_status_string(status).decode()
        raise AcfError(status, msg)


def stream_handle(stream=None):
    """Raw cudaStream_t of a torch stream (default: the current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None
