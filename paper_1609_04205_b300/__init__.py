"""acf: B300-native AARTFAAC correlator stage (arXiv 1609.04205, Sec. 4).

Polyphase channeliser (FIR + FFT + bandpass + transpose) and tensor-core
X-engine in hand-written sm_103a CUDA behind the C ABI of include/acf.h;
this package is the thin Python binding.  Nothing here computes: a missing
libacf.so raises instead of falling back.
"""
from ._lib import AcfError, lib  # noqa: F401
from .correlator import (Batch, Correlator, channelise, device_status, launch_count,  # noqa: F401
                         n_baselines, probe_tensor_peak, prototype, transpose_raw, xengine)
from .gain import GainCorr, gain_grad, gain_loss_and_grad  # noqa: F401
from . import postproc  # noqa: F401
