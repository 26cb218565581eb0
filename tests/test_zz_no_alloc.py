"""The allocation-free gain entry point (acf_gain_forward_noalloc) through the
C ABI, against the regular entry point and against the fp64 oracle.

Some callers cannot allocate device memory while they run (processes whose
device memory is reserved up front, real-time loops that must not block in
the allocator, plug-ins of a framework that owns every allocation); this entry
point keeps its loss partials in a fixed array compiled into the library.  The
test makes two calls in a row on different problem sizes (small, then large,
so the second call reads partials past the range the first one wrote) and
checks each result against acf_gain_forward within the gain tests' tolerance
and against oracle.gain_loss_grad; the second call must leave the device's
free memory unchanged.  It sits in its own file so that pytest collects it
last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _problem(N, C, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((C, N, 4)) + 1j * rng.standard_normal((C, N, 4))
    full = A @ A.conj().transpose(0, 2, 1)
    i, j = np.tril_indices(N)
    o = np.argsort(i * (i + 1) // 2 + j)
    R = full[:, i[o], j[o]]
    V = R * (1.0 + 0.05 * rng.standard_normal(R.shape))
    V[:, i[o] == j[o]] = V[:, i[o] == j[o]].real
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    return R, V, g


def test_noalloc_gain_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_04205_b300 import _lib as A
    L = A.lib()
    t = lambda a: torch.as_tensor(a, dtype=torch.complex64, device="cuda").contiguous()
    s = A.stream_handle()
    for call, (N, C) in enumerate([(96, 3), (200, 8)]):        # two calls in a row: 12, then 80 partials
        R, V, g = _problem(N, C, 80 + call)
        Rt, Vt, gt = t(R), t(V), t(g)
        loss_a = torch.empty((), dtype=torch.float32, device="cuda")
        loss_b = torch.empty((), dtype=torch.float32, device="cuda")
        grad_a = torch.empty(N, dtype=torch.complex64, device="cuda")
        grad_b = torch.empty(N, dtype=torch.complex64, device="cuda")
        assert L.acf_gain_forward(A.ptr(Rt), A.ptr(Vt), A.ptr(gt), N, C, A.ptr(loss_a), A.ptr(grad_a), s) == A.OK
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert L.acf_gain_forward_noalloc(A.ptr(Rt), A.ptr(Vt), A.ptr(gt), N, C, A.ptr(loss_b), A.ptr(grad_b),
                                          s) == A.OK
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
        la, lb = loss_a.item(), loss_b.item()
        assert abs(la - lb) <= 1e-5 * abs(la)
        ga, gb = grad_a.cpu().numpy(), grad_b.cpu().numpy()
        assert np.max(np.abs(ga - gb)) <= 1e-4 * np.max(np.abs(ga))
        # against the fp64 oracle, on the fp32 inputs the device saw
        Lr, gref = oracle.gain_loss_grad(Rt.cpu().numpy().astype(np.complex128),
                                         Vt.cpu().numpy().astype(np.complex128),
                                         gt.cpu().numpy().astype(np.complex128))
        assert abs(lb - Lr) <= 1e-4 * Lr
        assert np.linalg.norm(gb - gref) <= 1e-4 * np.linalg.norm(gref)


def test_noalloc_rejects_problems_beyond_the_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_04205_b300 import _lib as A
    L = A.lib()
    # 4096 inputs -> 64 x 65 / 2 = 2080 tiles per channel; 64 channels need 133,120 partials
    dummy = torch.zeros(4, dtype=torch.complex64, device="cuda")
    loss = torch.empty((), dtype=torch.float32, device="cuda")
    st = L.acf_gain_forward_noalloc(A.ptr(dummy), A.ptr(dummy), A.ptr(dummy), 4096, 64, A.ptr(loss), None,
                                    A.stream_handle())
    assert st == A.EINVAL
