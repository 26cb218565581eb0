"""The two-SM X-engine variant (CTA pairs on 256x256 tiles, tcgen05 cta_group::2)
against the oracle, through the C ABI: every precision mode, ragged input
counts around the 256-row tile edge, multi-push integrations, and the A-12
full-size workload on sampled inputs."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import norm_err

acf = pytest.importorskip("paper_1609_04205_b300")

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _c(V):
    V = V.cpu()
    if V.dtype == torch.complex64:
        return V.numpy().astype(np.complex128)
    return V[..., 0].numpy().astype(np.float64) + 1j * V[..., 1].numpy().astype(np.float64)


@pytest.mark.parametrize("N", [1, 33, 64, 127, 128, 129, 200])
@pytest.mark.parametrize("mode,tol", [("fp16", 3e-3), ("fp16x3", 1e-5)])
def test_pair_channelised_vs_oracle(N, mode, tol):
    _need_gpu()
    C, P, S = 16, 16, 16 * 80 + 5
    sky = synth.make_sky(N, 1, 0.3, 90 + N)
    x = synth.voltages(N, S, 2, "ci16", 512.0, sky, 90 + N, device="cuda")
    with acf.Correlator(N, 2, C, P, 1, mode, "ci16", S, variant=1) as c:
        c.push(x)
        V = c.visibilities()
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(x[sb].cpu().numpy(), P, C)[0]
        assert norm_err(_c(V[sb]), ref, N) <= tol


@pytest.mark.parametrize("N,S", [(1, 100), (96, 20000), (130, 70000)])
def test_pair_int8_exact(N, S):
    _need_gpu()
    x = synth.voltages(N, S, 1, "ci8", 16.0, None, 95 + N, device="cuda")
    with acf.Correlator(N, 1, 1, 1, 1, "int8", "ci8", S, variant=1) as c:
        c.push(x)
        V = c.visibilities()
    torch.cuda.synchronize()
    assert np.array_equal(V[0, 0].cpu().numpy(), oracle.correlate_int(x[0].cpu().numpy()))


def test_pair_accumulates_over_pushes():
    _need_gpu()
    N, C, P = 70, 64, 16
    pushes = [3000, 4100, 2222]
    x = synth.voltages(N, sum(pushes), 1, "ci8", 16.0, None, 97, device="cuda")
    with acf.Correlator(N, 1, C, P, 3, "fp16x3", "ci8", max(pushes), variant=1) as c:
        t0 = 0
        for n in pushes:
            c.push(x[:, t0:t0 + n].contiguous())
            t0 += n
        V = c.visibilities()
    torch.cuda.synchronize()
    ref = oracle.correlator(x[0].cpu().numpy(), P, C, push_sizes=pushes, n_integrate=3)[0]
    assert norm_err(_c(V[0]), ref, N) <= 1e-5


def test_pair_matches_single_sm_variant_bitwise_int8():
    _need_gpu()
    N, S = 200, 9000
    x = synth.voltages(N, S, 2, "ci8", 16.0, None, 98, device="cuda")
    outs = []
    for v in (0, 1):
        with acf.Correlator(N, 2, 1, 1, 1, "int8", "ci8", S, variant=v) as c:
            c.push(x)
            outs.append(c.visibilities().clone())
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    assert acf.device_status() == 0
