"""The C-ABI library loads, exports every symbol include/acf.h declares, and
rejects bad arguments on the host before touching a device.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1609_04205_b300 import _lib as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "acf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(acf_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert _declared() == sorted(A.EXPORTS)


def test_library_exports_every_symbol():
    L = A.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert b"sm_103a" in L.acf_version()


def test_status_strings():
    L = A.lib()
    for s in range(7):
        assert len(L.acf_status_string(s)) > 0


@pytest.mark.parametrize("args,status", [
    ((0, 1, 64, 16, 1, A.X_FP32, A.IN_CI8, 1000), A.EINVAL),        # no inputs
    ((96, 0, 64, 16, 1, A.X_FP32, A.IN_CI8, 1000), A.EINVAL),       # no subbands
    ((96, 1, 32, 16, 1, A.X_FP32, A.IN_CI8, 1000), A.EINVAL),       # channel count
    ((96, 1, 64, 0, 1, A.X_FP32, A.IN_CI8, 1000), A.EINVAL),        # taps
    ((96, 1, 1, 16, 1, A.X_FP32, A.IN_CI8, 1000), A.EINVAL),        # raw needs 1 tap
    ((96, 1, 64, 16, 0, A.X_FP32, A.IN_CI8, 1000), A.EINVAL),       # n_integrate
    ((96, 1, 64, 16, 1, 7, A.IN_CI8, 1000), A.EINVAL),              # mode
    ((96, 1, 64, 16, 1, A.X_FP32, 9, 1000), A.EINVAL),              # dtype
    ((96, 1, 64, 16, 1, A.X_FP32, A.IN_CI8, 0), A.EINVAL),          # max_samples
    ((96, 1, 64, 16, 1, A.X_INT8, A.IN_CI8, 1000), A.EUNSUPPORTED),  # INT8 needs raw
    ((96, 1, 1, 1, 1, A.X_INT8, A.IN_CI16, 1000), A.EUNSUPPORTED),   # INT8 needs ci8
])
def test_create_rejects_bad_arguments(args, status):
    L = A.lib()
    h = ctypes.c_void_p()
    st = L.acf_create(ctypes.byref(h), *args)
    assert st == status
    assert h.value is None
    assert len(L.acf_last_error(None)) > 0


def test_null_handles():
    L = A.lib()
    assert L.acf_create(None, 96, 1, 64, 16, 1, 0, 0, 100) == A.EINVAL
    assert L.acf_push_block(None, None, 10, None) == A.EINVAL
    assert L.acf_destroy(None) == A.OK
    assert L.acf_batch_destroy(None) == A.OK
    n = ctypes.c_int()
    assert L.acf_get_visibilities(None, None, ctypes.byref(n), None) == A.EINVAL
    assert L.acf_gain_forward(None, None, None, 4, 1, None, None, None) == A.EINVAL
    assert L.acf_xengine(0, None, None, 1, 4, 10, 64, 1.0, None, None) == A.EINVAL


def test_batch_rejects_bad_jobs():
    L = A.lib()
    jobs = (A.Job * 2)(A.Job(96, 64, 16, 1000), A.Job(96, 1, 16, 1000))   # raw job with 16 taps
    h = ctypes.c_void_p()
    assert L.acf_batch_create(ctypes.byref(h), jobs, 2, 0) == A.EINVAL
    assert L.acf_batch_create(ctypes.byref(h), jobs, 0, 0) == A.EINVAL


@pytest.mark.parametrize("P,C", [(16, 64), (16, 256), (4, 16), (1, 1)])
def test_library_prototype_matches_oracle(P, C):
    """Host-side prototype of the library (float) against the fp64 oracle."""
    L = A.lib()
    h = np.zeros(P * C, np.float32)
    assert L.acf_prototype(P, C, h.ctypes.data_as(ctypes.c_void_p)) == A.OK
    ref = oracle.prototype(P, C)
    assert np.max(np.abs(h - ref)) <= 1e-7 * np.max(np.abs(ref)) + 1e-12
    assert L.acf_prototype(0, C, h.ctypes.data_as(ctypes.c_void_p)) == A.EINVAL


@pytest.mark.parametrize("entry", ["acf_gain_forward_noalloc", "acf_gain_forward"])
def test_gain_rejects_sizes_whose_partial_count_overflows_32_bits(entry):
    """2,900,000 inputs over 3 channels need m(m+1)/2 * 4 * ceil(3/8) = 4.1e9
    loss partials (m = ceil(N/64)), past 2^31: the count is kept in 64 bits, so the
    allocation-free entry point rejects it on the host (its fixed scratch holds
    65,536) and the allocating one rejects a channel count past the grid's
    65,535; neither enqueues anything, so dummy pointers are never read."""
    L = A.lib()
    dummy = ctypes.c_void_p(16)
    loss = ctypes.c_void_p(32)
    fn = getattr(L, entry)
    if entry == "acf_gain_forward_noalloc":
        assert fn(dummy, dummy, dummy, 2_900_000, 3, loss, None, None) == A.EINVAL
        assert fn(dummy, dummy, dummy, 64, 65_536, loss, None, None) == A.EINVAL
    else:
        assert fn(dummy, dummy, dummy, 64, 65_536, loss, None, None) == A.EINVAL
