"""Full-size parity: the workloads bench.py times, in the same launch
configuration (one Correlator context per mode, all subbands in one push),
checked on sampled outputs the oracle can compute directly: a random subset
of inputs on a few subbands and channels.  Tolerances as in the small tests
(normalised metric; FP32 / split FP16 1e-5, FP16 3e-3, INT8 bit-exact)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import tri_index

acf = pytest.importorskip("paper_1609_04205_b300")

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _subset(N, k, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=k, replace=False))


def _gather(V, sb, chans, idx):
    """V on device [n_sb, n_ch, NB, 2] -> complex [len(chans), n(n+1)/2] over the subset idx."""
    n = len(idx)
    ii, jj = tri_index(n)
    gi, gj = idx[ii], idx[jj]
    bl = torch.as_tensor(gi * (gi + 1) // 2 + gj, device=V.device)
    out = V[sb][chans][:, bl].cpu()
    if out.dtype == torch.complex64:
        return out.numpy().astype(np.complex128)
    if out.dtype == torch.float32:
        out = out.double()
        return (out[..., 0] + 1j * out[..., 1]).numpy()
    return out.numpy()          # int64 pairs


def _norm_err(got, ref, n):
    ii, jj = tri_index(n)
    d = np.arange(n) * (np.arange(n) + 1) // 2 + np.arange(n)
    auto = ref[:, d].real
    den = np.sqrt(auto[:, ii] * auto[:, jj])
    return float(np.max(np.abs(got - ref) / den))


@pytest.fixture(scope="module")
def a12_input():
    _need_gpu()
    w = synth.WORKLOADS["a12"]
    sky = synth.make_sky(w["n_inputs"], w["n_sources"], w["flux"], w["seed"])
    x = synth.voltages(w["n_inputs"], w["n_samples"], w["n_subbands"], w["dtype"], w["sigma"], sky, w["seed"],
                       device="cuda")
    yield w, x
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode,tol", [("fp16", 3e-3), ("fp16x3", 1e-5)])
def test_a12_full_size_sampled(a12_input, mode, tol):
    w, x = a12_input
    N, C, P = w["n_inputs"], w["n_channels"], w["n_taps"]
    with acf.Correlator(N, w["n_subbands"], C, P, 1, mode, w["dtype"], w["n_samples"]) as c:
        c.push(x)
        V = torch.view_as_real(c.visibilities())
        T = c.query()["last_spectra"]
        torch.cuda.synchronize()
        # first push of a stream: floor((S - (P-1) C) / C) spectra
        assert T == oracle.n_spectra(w["n_samples"], P, C) == 3036
        chans = [0, 17, 63]
        for sb in (0, 15):
            idx = _subset(N, 16, 100 + sb)
            xs = x[sb][:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
            X = oracle.channelise(xs, oracle.prototype(P, C), P, C, chans=chans)
            ref = oracle.correlate(X)
            got = _gather(torch.view_as_complex(V), sb, chans, idx)
            assert _norm_err(got, ref, len(idx)) <= tol


def test_a6_int8_raw_full_size_exact():
    """576 inputs x 8 subbands x 195,313 raw ci8 samples, INT8 mode: bit-exact."""
    _need_gpu()
    w = synth.WORKLOADS["a6"]
    N, S, n_sb = w["n_inputs"], w["n_samples"], w["n_subbands"]
    x = synth.voltages(N, S, n_sb, "ci8", w["sigma"], None, w["seed"], device="cuda")
    with acf.Correlator(N, n_sb, 1, 1, 1, "int8", "ci8", S) as c:
        c.push(x)
        V = c.visibilities()
        torch.cuda.synchronize()
        for sb in (0, 7):
            idx = _subset(N, 14, 200 + sb)
            xs = x[sb][:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
            ref = oracle.correlate_int(xs)
            got = _gather(V, sb, [0], idx)[0]
            assert np.array_equal(got, ref)
        # the largest values reach well past 2^24: autocorrelations ~ 2 sigma^2 S
        assert int(V[0, 0, 0, 0]) > 2 ** 26


def test_a6_fp32_channelised_full_size_sampled():
    """576 inputs x 8 subbands, 16-tap x 64-channel filter bank, FP32 CUDA-core X-engine."""
    _need_gpu()
    w = synth.WORKLOADS["a6"]
    N, S, n_sb, C, P = w["n_inputs"], w["n_samples"], w["n_subbands"], 64, 16
    x = synth.voltages(N, S, n_sb, "ci8", w["sigma"], None, w["seed"], device="cuda")
    with acf.Correlator(N, n_sb, C, P, 1, "fp32", "ci8", S) as c:
        c.push(x)
        V = c.visibilities()
        torch.cuda.synchronize()
        chans = [5, 40]
        for sb in (3,):
            idx = _subset(N, 16, 300 + sb)
            xs = x[sb][:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
            X = oracle.channelise(xs, oracle.prototype(P, C), P, C, chans=chans)
            ref = oracle.correlate(X)
            got = _gather(V, sb, chans, idx)
            assert _norm_err(got, ref, len(idx)) <= 1e-5


def test_gain_full_size_576_inputs_64_channels():
    """Calibration workload: 576 inputs, 64 channels, 0.5 s of cf32 voltages with
    5 point sources.  R = unit-gain model visibilities, V = visibilities of the
    gain-corrupted voltages (both from the FP32 correlator); the loss vanishes
    at the true gains, and at perturbed gains the adjoint matches fp64 and
    FP32 central differences (h = 1e-3, 1e-3 relative)."""
    _need_gpu()
    w = synth.WORKLOADS["gain"]
    N, S, C, P = w["n_inputs"], w["n_samples"], w["n_channels"], w["n_taps"]
    sky = synth.make_sky(N, w["n_sources"], w["flux"], w["seed"])
    x = synth.voltages(N, S, 1, "cf32", w["sigma"], sky, w["seed"], device="cuda")
    g_true = synth.unit_gains(N, w["seed"] + 1, device="cuda")
    xc = torch.view_as_complex(x) * g_true[None, None, :]
    xg = torch.view_as_real(xc).contiguous()
    # two independent streams (one context each: a context carries filter history)
    with acf.Correlator(N, 1, C, P, 1, "fp32", "cf32", S) as c:
        c.push(x)
        R = c.visibilities()[0].clone()
    with acf.Correlator(N, 1, C, P, 1, "fp32", "cf32", S) as c:
        c.push(xg)
        V = c.visibilities()[0].clone()
    L0, g0 = acf.gain_loss_and_grad(g_true, R, V)
    Ls = (V.abs() ** 2).sum().item()
    assert L0.item() <= 1e-8 * Ls
    rng = np.random.default_rng(5)
    g = (g_true.cpu().numpy() * (1 + 0.05 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))).astype(np.complex64)
    gt = torch.as_tensor(g, device="cuda")
    L, grad = acf.gain_loss_and_grad(gt, R, V)
    Lr, gref = oracle.gain_loss_grad(R.cpu().numpy().astype(np.complex128), V.cpu().numpy().astype(np.complex128),
                                     g.astype(np.complex128))
    assert abs(L.item() - Lr) <= 1e-4 * Lr
    gg = grad.cpu().numpy()
    assert np.linalg.norm(gg - gref) <= 1e-4 * np.linalg.norm(gref)
    # central differences on sampled components
    h = 1e-3
    for k in rng.choice(N, 6, replace=False):
        for unit in (1.0, 1j):
            gp, gm = g.copy(), g.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            lp = acf.gain_loss_and_grad(torch.as_tensor(gp, device="cuda"), R, V, want_grad=False)[0].item()
            lm = acf.gain_loss_and_grad(torch.as_tensor(gm, device="cuda"), R, V, want_grad=False)[0].item()
            fd = (lp - lm) / (2 * h)
            an = gg[k].real if unit == 1.0 else gg[k].imag
            ref = gref[k].real if unit == 1.0 else gref[k].imag
            assert abs(fd - ref) <= 1e-3 * np.max(np.abs(gref)) and abs(an - ref) <= 1e-4 * np.max(np.abs(gref))


def test_ragged_batch_32_jobs_sampled():
    """The 32-job ragged batch (antennas 48..576, channels 16/64/256 or raw),
    one persistent launch captured in a CUDA graph; sampled per job."""
    _need_gpu()
    jobs = synth.ragged_jobs()
    b = acf.Batch(jobs, autotune=False)
    ins = [synth.voltages(j["n_inputs"], j["n_samples"], 1, "ci8", 16.0, None, j["seed"], device="cuda")[0]
           for j in jobs]
    outs = b.outputs()
    b.run(ins, outs)
    b.run(ins, outs)          # graph replay
    torch.cuda.synchronize()
    for k, j in enumerate(jobs):
        N = j["n_inputs"]
        idx = _subset(N, 8, 400 + k)
        xs = ins[k][:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
        Vk = outs[k][None]
        if j["raw"]:
            got = _gather(Vk, 0, [0], idx)[0]
            assert np.array_equal(got, oracle.correlate_int(xs))
        else:
            C, P = j["n_channels"], j["n_taps"]
            chans = [0, C // 3]
            X = oracle.channelise(xs, oracle.prototype(P, C), P, C, chans=chans)
            ref = oracle.correlate(X)
            got = _gather(Vk, 0, chans, idx)
            assert _norm_err(got, ref, len(idx)) <= 1e-5
    b.close()


@pytest.mark.parametrize("mode,tol", [("fp16", 3e-3), ("fp16x3", 1e-5)])
def test_a12_full_size_four_one_second_integrations(a12_input, mode, tol):
    """The A-12 configuration's "1 s integrations x 4": one context with
    n_integrate = 4 takes four consecutive one-second pushes (the stream is
    the benchmark's block four times over, 781,252 samples per subband), so
    the accumulator carries across pushes and the filter history crosses
    three push boundaries; only the fourth push completes the integration.
    Checked on sampled inputs and channels against the oracle's stream
    partition."""
    w, x = a12_input
    N, C, P, S = w["n_inputs"], w["n_channels"], w["n_taps"], w["n_samples"]
    chans = [0, 33]
    with acf.Correlator(N, w["n_subbands"], C, P, 4, mode, w["dtype"], S) as c:
        for k in range(4):
            c.push(x)
            V = c.visibilities()
            assert (V is None) == (k < 3)
        V = torch.view_as_real(V)
        torch.cuda.synchronize()
        for sb in (7,):
            idx = _subset(N, 12, 500 + sb)
            xs = x[sb][:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
            stream = np.concatenate([xs] * 4, axis=0)
            ref = oracle.correlator(stream, P, C, push_sizes=[S] * 4, n_integrate=4, chans=chans)
            assert len(ref) == 1
            got = _gather(torch.view_as_complex(V), sb, chans, idx)
            assert _norm_err(got, ref[0], len(idx)) <= tol
