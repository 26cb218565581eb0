"""Post-correlation steps on visibilities (delay compensation, channel
integration, lost-data weights, sigma-clip flagging): argument marshalling
for the C ABI in include/acf.h.  V tensors are [n_subbands, n_channels, NB, 2]
(complex float32 as (re, im) pairs, or int64 pairs for INT8 visibilities) on
the current CUDA device; work runs on the current torch stream."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as A


def _n_inputs(NB: int) -> int:
    n = int(round((np.sqrt(8 * NB + 1) - 1) / 2))
    if n * (n + 1) // 2 != NB:
        raise ValueError("last-but-one axis is not a packed triangle")
    return n


def _host_f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def delay_compensate(V, delays, f_centre, sample_rate: float, stream=None):
    """In place: V_ij *= exp(+2 pi i f_c (d_i - d_j)) (acf_delay_compensate)."""
    n_sb, C, NB = V.shape[0], V.shape[1], V.shape[2]
    d, f = _host_f64(delays), _host_f64(f_centre)
    A.check(A.lib().acf_delay_compensate(A.ptr(V), n_sb, C, _n_inputs(NB), d.ctypes.data_as(A.ctypes.c_void_p),
                                         f.ctypes.data_as(A.ctypes.c_void_p), float(sample_rate),
                                         A.stream_handle(stream)))
    return V


def integrate_channels(V, group: int, stream=None):
    """Sums of `group` adjacent channels -> new tensor [n_sb, C/group, NB, 2]."""
    n_sb, C, NB = V.shape[0], V.shape[1], V.shape[2]
    out = torch.empty((n_sb, C // group, NB, 2), dtype=V.dtype, device=V.device)
    A.check(A.lib().acf_integrate_channels(A.ptr(V), A.ptr(out), n_sb, C, _n_inputs(NB), int(group),
                                           1 if V.dtype == torch.int64 else 0, A.stream_handle(stream)))
    return out


def sigma_clip(V, k_chan: float, k_vis: float, stream=None):
    """Two-stage flags, uint8 [n_sb, C, NB] (acf_sigma_clip)."""
    n_sb, C, NB = V.shape[0], V.shape[1], V.shape[2]
    flags = torch.empty((n_sb, C, NB), dtype=torch.uint8, device=V.device)
    A.check(A.lib().acf_sigma_clip(A.ptr(V), A.ptr(flags), n_sb, C, _n_inputs(NB), float(k_chan), float(k_vis),
                                   A.stream_handle(stream)))
    return flags


def lost_sample_weights(mask, samples_per_block: int, stream=None):
    """mask uint8 [n_blocks, N] on the device -> W int64 [NB]."""
    n_blocks, N = mask.shape
    W = torch.empty(N * (N + 1) // 2, dtype=torch.int64, device=mask.device)
    A.check(A.lib().acf_lost_sample_weights(A.ptr(mask), int(n_blocks), int(N), int(samples_per_block), A.ptr(W),
                                            A.stream_handle(stream)))
    return W


def reweight(V, W, n_total: int, stream=None):
    """In place: V_ij *= n_total / W_ij (0 where W_ij == 0), every problem."""
    NB = V.shape[-2]
    n_prob = V.numel() // (NB * 2)
    A.check(A.lib().acf_reweight(A.ptr(V), A.ptr(W), int(n_total), int(n_prob), _n_inputs(NB),
                                 A.stream_handle(stream)))
    return V
