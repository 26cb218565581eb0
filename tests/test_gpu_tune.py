"""The streaming context's X-engine autotuner (acf_tune / acf_query_xengine)
through the C ABI: after tuning, the chosen launch shape is reported and an
integration over several pushes still matches the oracle in every tensor-core
mode; tuning is refused mid-integration and in FP32 mode."""
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


@pytest.mark.parametrize("N,mode,tol", [(40, "fp16x3", 1e-5), (300, "fp16", 3e-3), (130, "fp16x3", 1e-5)])
def test_tuned_context_matches_oracle(N, mode, tol):
    _need_gpu()
    C, P = 16, 16
    pushes = [3000, 2500]
    S = sum(pushes)
    sky = synth.make_sky(N, 1, 0.3, 300 + N)
    x = synth.voltages(N, S, 3, "ci16", 512.0, sky, 300 + N, device="cuda")
    with acf.Correlator(N, 3, C, P, 2, mode, "ci16", max(pushes)) as c:
        before = c.xengine_tuning()
        assert before["tuned"] is False
        t = c.tune()
        assert t["tuned"] is True
        assert t["variant"] in (0, 1) and t["n_tile"] in (128, 256) and t["k_split"] in (1, 2, 4)
        assert t["variant"] == 0 or t["n_tile"] == 256
        t0 = 0
        for n in pushes:
            c.push(x[:, t0:t0 + n].contiguous())
            t0 += n
        V = c.visibilities()
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    for sb in range(3):
        ref = oracle.correlator(xs[sb], P, C, push_sizes=pushes, n_integrate=2)[0]
        assert norm_err(_c(V[sb]), ref, N) <= tol


def test_tuned_int8_exact():
    _need_gpu()
    N, S = 96, 30000
    x = synth.voltages(N, S, 2, "ci8", 16.0, None, 321, device="cuda")
    with acf.Correlator(N, 2, 1, 1, 1, "int8", "ci8", S) as c:
        c.tune()
        c.push(x)
        V = c.visibilities()
    torch.cuda.synchronize()
    for sb in range(2):
        assert np.array_equal(V[sb, 0].cpu().numpy(), oracle.correlate_int(x[sb].cpu().numpy()))


def test_tune_refused_mid_integration_and_in_fp32():
    _need_gpu()
    x = synth.voltages(20, 4000, 1, "ci16", 512.0, None, 5, device="cuda")
    with acf.Correlator(20, 1, 16, 16, 2, "fp16", "ci16", 4000) as c:
        c.push(x)
        with pytest.raises(acf.AcfError):
            c.tune()
    with acf.Correlator(20, 1, 16, 16, 1, "fp32", "ci16", 4000) as c:
        with pytest.raises(acf.AcfError):
            c.tune()
