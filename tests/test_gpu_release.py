"""Zero-copy hand-out of integrations (acf_release_visibilities +
acf_visibilities_device) through the C ABI: the accumulator read in place
equals the copied integration and the oracle, release re-arms the context for
the next push, and nothing is handed out before an integration completes."""
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


@pytest.mark.parametrize("mode,tol", [("fp16x3", 1e-5), ("fp32", 1e-5)])
def test_release_matches_copy_and_oracle(mode, tol):
    _need_gpu()
    N, C, P, S = 40, 16, 16, 3000
    sky = synth.make_sky(N, 1, 0.3, 501)
    x = synth.voltages(N, 2 * S, 2, "ci16", 512.0, sky, 501, device="cuda")
    xs = x.cpu().numpy()
    with acf.Correlator(N, 2, C, P, 1, mode, "ci16", S) as c:
        c.push(x[:, :S].contiguous())
        V0 = c.visibilities()                                  # copied hand-out
        c.push(x[:, S:].contiguous())
        assert c.release() is True                             # zero-copy hand-out
        V1 = c.device_visibilities().clone()
        assert c.release() is False                            # nothing new is complete
        c.push(x[:, :S].contiguous())                          # release re-armed the context
        assert c.release() is True
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(xs[sb], P, C, push_sizes=[S, S], n_integrate=1)
        assert norm_err(V0[sb].cpu().numpy().astype(np.complex128), ref[0], N) <= tol
        assert norm_err(V1[sb].cpu().numpy().astype(np.complex128), ref[1], N) <= tol


def test_release_int8_exact():
    _need_gpu()
    N, S = 64, 5000
    x = synth.voltages(N, S, 1, "ci8", 16.0, None, 502, device="cuda")
    with acf.Correlator(N, 1, 1, 1, 1, "int8", "ci8", S) as c:
        c.push(x)
        assert c.release() is True
        V = c.device_visibilities().clone()
    torch.cuda.synchronize()
    assert np.array_equal(V[0, 0].cpu().numpy(), oracle.correlate_int(x[0].cpu().numpy()))
