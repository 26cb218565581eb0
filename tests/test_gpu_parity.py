"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Tolerances (normalised metric max |dV| / sqrt(V_ii V_jj)):
FP32 and split-FP16 1e-5, plain FP16 3e-3, INT8 bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import norm_err, norm_err_subset, tri_index

acf = pytest.importorskip("paper_1609_04205_b300")

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_FP16 = 3e-3


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _samples(N, S, n_sb=1, dtype="ci8", sigma=16.0, n_src=1, flux=0.2, seed=1):
    sky = synth.make_sky(N, n_src, flux, seed) if n_src else None
    return synth.voltages(N, S, n_sb, dtype, sigma, sky, seed, device="cuda")


def _np_complex(V):
    V = V.cpu()
    if V.dtype == torch.complex64:
        return V.numpy().astype(np.complex128)
    return V[..., 0].numpy().astype(np.float64) + 1j * V[..., 1].numpy().astype(np.float64)


def _check_fp16_tc_bound(Xh, X32, w, sc, T):
    """64 channels, fp16 output: the DFT runs on the tensor cores with the FIR
    outputs y and the twiddles W rounded to fp16 (unit roundoff u = 2^-11)
    and fp32 accumulation.  Per (input, spectrum):
        |z_hat_c - z_c| <= (2u + u^2) sum_n |y_n| + 2^-15 sum_n |y_n|,
    and by Parseval sum_n |y_n| <= 8 ||y||_2 = ||z||_2 over the 64
    unweighted channels; the output rounding adds u |v| (v = scaled fp32
    value)."""
    C = X32.shape[1]
    v = (X32 * sc)[..., :T]
    wt = torch.as_tensor(w, dtype=torch.float32, device=X32.device).view(1, C, 1, 1)
    zr, zi = X32[:, :, 0::2, :T] / wt, X32[:, :, 1::2, :T] / wt
    nrm = torch.sqrt((zr * zr + zi * zi).sum(dim=1, keepdim=True))          # [sb, 1, N, T]
    nrm2 = torch.repeat_interleave(nrm, 2, dim=2)                            # per re / im row
    bound = v.abs() * 2.0 ** -11 + 1e-6 * v.abs().max() + (2.0 ** -10 + 2.0 ** -14) * (sc * wt).abs() * nrm2
    assert ((Xh[..., :T].float() - v).abs() <= bound).all()


# ---------------------------------------------------------------- channeliser
@pytest.mark.parametrize("C,P,dtype,N,S", [
    (64, 16, "ci8", 96, 19532),       # the tiny single-station configuration
    (16, 16, "ci16", 33, 5000),       # ragged input count, int16
    (256, 16, "cf32", 5, 256 * 20 + 100),
    (64, 4, "ci8", 130, 3000),
    (64, 16, "ci16", 132, 7000),      # fast path, 16-byte loads, partial last input group
    (16, 16, "ci8", 40, 3000),        # fast path, two inputs per warp
])
def test_channelise_fp32_vs_oracle(C, P, dtype, N, S):
    _dev()
    x = _samples(N, S, 1, dtype, sigma=16.0 if dtype != "ci16" else 512.0, seed=C + N)
    X, _, T = acf.channelise(x, C, P, out_kind="f32")
    torch.cuda.synchronize()
    ref = oracle.channelise(x[0].cpu().numpy(), oracle.prototype(P, C), P, C)      # [C, N, T]
    assert T == ref.shape[2] == oracle.n_spectra(S, P, C)
    got = X[0].cpu().numpy().astype(np.float64)                                   # [C, 2N, ts]
    gc = got[:, 0::2, :T] + 1j * got[:, 1::2, :T]
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(gc - ref)) <= 2e-6 * scale
    assert np.all(got[:, :, T:(T + 63) // 64 * 64] == 0)        # zeroed tail


def test_channelise_fp16_split_reconstructs():
    _dev()
    C, P, N, S = 64, 16, 40, 4000
    x = _samples(N, S, 2, "ci16", sigma=512.0, seed=5)
    X32, _, T = acf.channelise(x, C, P, out_kind="f32")
    Xh, Xl, T2 = acf.channelise(x, C, P, out_kind="f16x3", scale=0.5)
    assert T == T2
    recon = (Xh.float() + Xl.float()) / 0.5
    ref = X32
    err = (recon - ref).abs().max().item()
    assert err <= 1e-6 * ref.abs().max().item() * 4


@pytest.mark.parametrize("C", [64, 256])
@pytest.mark.parametrize("dtype,N", [("ci16", 36), ("ci16", 48), ("ci8", 40)])
@pytest.mark.parametrize("n_hist", [0, 500, 1023, 3000])
def test_channelise_fast_paths_history_and_segments_vs_oracle(C, dtype, N, n_hist):
    """The 64-channel warp-specialised path (N a multiple of one 16-byte row
    of inputs: spectra whose windows reach into the history come from the
    generic kernel, the rest from the TMA-fed kernel) and the 256-channel path
    (history read in place), split into several time segments per (subband,
    input); two subbands; f32 output against the oracle on the concatenated
    stream, zeroed tail."""
    _dev()
    P, n_sb = 16, 2
    S = 64 * 700 + 37 if C == 64 else 256 * 150 + 37
    sig = 512.0 if dtype == "ci16" else 16.0
    full = _samples(N, n_hist + S, n_sb, dtype, sigma=sig, seed=60 + n_hist)
    hist = full[:, :n_hist].contiguous() if n_hist else None
    x = full[:, n_hist:].contiguous()
    X, _, T = acf.channelise(x, C, P, out_kind="f32", hist=hist)
    torch.cuda.synchronize()
    assert T == oracle.n_spectra(n_hist + S, P, C)
    h = oracle.prototype(P, C)
    for sb in range(n_sb):
        ref = oracle.channelise(full[sb].cpu().numpy(), h, P, C)
        got = X[sb].cpu().numpy().astype(np.float64)
        gc = got[:, 0::2, :T] + 1j * got[:, 1::2, :T]
        assert np.max(np.abs(gc - ref)) <= 2e-6 * np.max(np.abs(ref))
        assert np.all(got[:, :, T:(T + 63) // 64 * 64] == 0)
    # fp16 output over the same history (64 channels: the tensor-core kernel
    # reads a history shorter than one window itself)
    sc = 0.25 if dtype == "ci16" else 4.0
    Xh, _, Th = acf.channelise(x, C, P, out_kind="f16", hist=hist, scale=sc)
    torch.cuda.synchronize()
    assert Th == T
    if C == 64 and N % 8 == 0:
        _check_fp16_tc_bound(Xh, X, np.ones(C), sc, T)
    else:
        v = (X * sc)[..., :T]
        assert ((Xh[..., :T].float() - v).abs() <= v.abs() * 2.0 ** -11 + 1e-6 * v.abs().max()).all()
    assert (Xh[..., T:] == 0).all()


@pytest.mark.parametrize("C", [64, 256])
@pytest.mark.parametrize("dtype,N", [("ci16", 48), ("ci8", 64)])
def test_channelise_fast_paths_fp16_outputs_and_bandpass(C, dtype, N):
    """fp16 and split fp16 outputs of the 64- and 256-channel paths with
    non-uniform bandpass weights and an output scale: split hi is the fp16
    rounding of the scaled fp32 value and hi + lo reconstructs it to fp32
    accuracy; plain fp16 output equals split hi for 256 channels and, for 64
    channels (tensor-core DFT on fp16 operands), stays within the rounding
    bound of that arithmetic."""
    _dev()
    P = 16
    S = 64 * 300 + 5 if C == 64 else 256 * 70 + 5
    sig = 512.0 if dtype == "ci16" else 16.0
    x = _samples(N, S, 2, dtype, sigma=sig, seed=70)
    w = synth.bandpass_ripple(C, 9)
    sc = 0.25 if dtype == "ci16" else 4.0
    X32, _, T = acf.channelise(x, C, P, out_kind="f32", bandpass=w)
    Xh, _, _ = acf.channelise(x, C, P, out_kind="f16", bandpass=w, scale=sc)
    Xh3, Xl3, _ = acf.channelise(x, C, P, out_kind="f16x3", bandpass=w, scale=sc)
    torch.cuda.synchronize()
    ref = oracle.channelise(x[0].cpu().numpy(), oracle.prototype(P, C), P, C, bandpass=w.astype(np.float64))
    got = X32[0].cpu().numpy().astype(np.float64)
    gc = got[:, 0::2, :T] + 1j * got[:, 1::2, :T]
    assert np.max(np.abs(gc - ref)) <= 2e-6 * np.max(np.abs(ref))
    v = (X32 * sc)[..., :T]
    half_ulp = v.abs() * 2.0 ** -11 + 1e-6 * v.abs().max()
    # split output: hi is the fp16 rounding of the scaled value (half an ulp, up to fp32 noise)
    assert ((Xh3[..., :T].float() - v).abs() <= half_ulp).all()
    if C == 256:
        assert torch.equal(Xh[..., :T], Xh3[..., :T])
    else:
        _check_fp16_tc_bound(Xh, X32, w, sc, T)
    recon = Xh3[..., :T].float() + Xl3[..., :T].float()
    assert (recon - v).abs().max().item() <= 4e-6 * v.abs().max().item()
    assert (Xh[..., T:] == 0).all() and (Xl3[..., T:] == 0).all()


@pytest.mark.parametrize("C", [64, 256])
def test_correlator_streaming_pushes_ci16(C):
    """Context path over five ragged pushes (64 channels: history carried by
    the generic head of each push, the rest by the TMA-fed kernel; 256
    channels: one kernel reading the history in place), integrations of two
    pushes, split FP16, against the oracle's stream partition."""
    _dev()
    N, P = 44, 16
    pushes = [5000, 1300, 64 * 40 + 7, 260, 9000]
    S = sum(pushes)
    sky = synth.make_sky(N, 2, (0.1, 0.4), 77)
    x = synth.voltages(N, S, 2, "ci16", 512.0, sky, 77, device="cuda")
    xs = x.cpu().numpy()
    with acf.Correlator(N, 2, C, P, 2, "fp16x3", "ci16", max(pushes)) as c:
        outs = []
        t0 = 0
        for n in pushes:
            c.push(x[:, t0:t0 + n].contiguous())
            t0 += n
            V = c.visibilities()
            if V is not None:
                outs.append(V.clone())
        assert len(outs) == 2
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(xs[sb], P, C, push_sizes=pushes, n_integrate=2)
        for k in range(2):
            assert norm_err(_np_complex(outs[k][sb]), ref[k], N) <= TOL_FP32


@pytest.mark.parametrize("dtype,N", [("ci16", 48), ("ci8", 64)])
def test_correlator_streaming_split_tensor_core_channeliser(dtype, N):
    """64-channel split-FP16 context with an input count divisible by eight:
    every push goes through the tensor-core channeliser's split form (hi/lo
    FIR operands and DFT matrix, three MMAs per K step; one operand buffer
    and three input stages for int16, two and two for int8), which reads the
    filter history itself.  Ragged pushes, integrations of two pushes,
    against the oracle's stream partition at the FP32 tolerance."""
    _dev()
    P, C = 16, 64
    pushes = [5000, 1300, 64 * 40 + 7, 260, 9000]
    S = sum(pushes)
    sky = synth.make_sky(N, 2, (0.1, 0.4), 79)
    x = synth.voltages(N, S, 2, dtype, 512.0 if dtype == "ci16" else 16.0, sky, 79, device="cuda")
    xs = x.cpu().numpy()
    with acf.Correlator(N, 2, C, P, 2, "fp16x3", dtype, max(pushes)) as c:
        outs = []
        t0 = 0
        for n in pushes:
            c.push(x[:, t0:t0 + n].contiguous())
            t0 += n
            V = c.visibilities()
            if V is not None:
                outs.append(V.clone())
        assert len(outs) == 2
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(xs[sb], P, C, push_sizes=pushes, n_integrate=2)
        for k in range(2):
            assert norm_err(_np_complex(outs[k][sb]), ref[k], N) <= TOL_FP32


@pytest.mark.parametrize("N", [70, 33])
def test_correlator_streaming_256ch_ci8_corner_turn(N):
    """256-channel context on complex int8 over ragged pushes: each push is
    corner-turned (history, then the samples) into per-input rows before the
    filter bank reads them.  An even input count takes the 4-byte, 64 x 64
    tile form (N = 70 spans two input tiles, the second ragged), an odd one
    the 32 x 32 form; split FP16 against the oracle's stream partition."""
    _dev()
    P, C = 16, 256
    pushes = [4100, 256 * 7 + 3, 9000, 601, 5555]
    S = sum(pushes)
    sky = synth.make_sky(N, 2, (0.1, 0.4), 78)
    x = synth.voltages(N, S, 2, "ci8", 16.0, sky, 78, device="cuda")
    xs = x.cpu().numpy()
    with acf.Correlator(N, 2, C, P, 2, "fp16x3", "ci8", max(pushes)) as c:
        outs = []
        t0 = 0
        for n in pushes:
            c.push(x[:, t0:t0 + n].contiguous())
            t0 += n
            V = c.visibilities()
            if V is not None:
                outs.append(V.clone())
        assert len(outs) == 2
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(xs[sb], P, C, push_sizes=pushes, n_integrate=2)
        for k in range(2):
            assert norm_err(_np_complex(outs[k][sb]), ref[k], N) <= TOL_FP32


@pytest.mark.parametrize("N,S,scale", [(8, 64, 1.0), (64, 1000, 1.0), (72, 777, 1.0), (96, 5000, 0.5),
                                         (1152, 300, 1.0), (5, 130, 1.0)])
def test_transpose_raw_ci8_fp16_exact(N, S, scale):
    """Raw-subband operand (the transpose of Sec. 4.2.4 alone) from complex int8
    to fp16 rows: every value is the exact int8 times the power-of-two scale,
    rows 2n / 2n + 1 hold Re / Im of input n, the tail past S is zero.  N a
    multiple of 8 takes the 16-byte tiled kernel, other counts the generic one."""
    _dev()
    x = _samples(N, S, 2, "ci8", sigma=40.0, n_src=0, seed=N + S)
    Xh, _ = acf.transpose_raw(x, out_kind="f16", scale=scale)
    torch.cuda.synchronize()
    want = x.permute(0, 2, 3, 1).reshape(2, 2 * N, S).float() * scale       # [sb][2n + comp][t]
    assert torch.equal(Xh[..., :S].float(), want)
    assert (Xh[..., S:] == 0).all()


# ---------------------------------------------------------------- X-engines
@pytest.mark.parametrize("N,T", [(1, 1), (3, 37), (64, 100), (97, 500), (130, 64)])
def test_xengine_simt_vs_oracle(N, T):
    dev = _dev()
    g = torch.Generator(device="cuda").manual_seed(N * 7 + T)
    ts = (T + 63) // 64 * 64
    X = torch.zeros((2, 2 * N, ts), device=dev)
    X[..., :T] = torch.randn((2, 2 * N, T), generator=g, device=dev)
    V = acf.xengine("fp32", X, None, N, T)
    torch.cuda.synchronize()
    Xc = X[:, 0::2, :T].double().cpu().numpy() + 1j * X[:, 1::2, :T].double().cpu().numpy()
    ref = oracle.correlate(Xc)
    assert norm_err(_np_complex(V), ref, N) <= TOL_FP32


def _rand_operand(N, T, n_p, seed, scale=1.0):
    g = torch.Generator(device="cuda").manual_seed(seed)
    ts = (T + 63) // 64 * 64
    X = torch.zeros((n_p, 2 * N, ts), device="cuda")
    X[..., :T] = torch.randn((n_p, 2 * N, T), generator=g, device="cuda") * scale
    return X


@pytest.mark.parametrize("N,T", [(1, 64), (33, 100), (64, 128), (96, 1000), (200, 333), (300, 2048)])
def test_xengine_tc_fp16_vs_oracle(N, T):
    _dev()
    X = _rand_operand(N, T, 2, seed=N + T, scale=8.0).half()
    V = acf.xengine("fp16", X, None, N, T)
    torch.cuda.synchronize()
    Xd = X.double().cpu().numpy()
    ref = oracle.correlate(Xd[:, 0::2, :T] + 1j * Xd[:, 1::2, :T])
    # operands are exact fp16 values: only fp32 accumulation separates the two
    assert norm_err(_np_complex(V), ref, N) <= TOL_FP32


@pytest.mark.parametrize("N,T", [(5, 70), (64, 640), (160, 3051)])
def test_xengine_tc_fp16x3_vs_oracle(N, T):
    _dev()
    X = _rand_operand(N, T, 2, seed=3 * N + T, scale=100.0)
    hi = X.half()
    lo = (X - hi.float()).half()
    V = acf.xengine("fp16x3", hi, lo, N, T)
    Vp = acf.xengine("fp16", hi, None, N, T)
    torch.cuda.synchronize()
    Xd = X.double().cpu().numpy()
    ref = oracle.correlate(Xd[:, 0::2, :T] + 1j * Xd[:, 1::2, :T])
    assert norm_err(_np_complex(V), ref, N) <= TOL_FP32
    assert norm_err(_np_complex(Vp), ref, N) <= TOL_FP16


@pytest.mark.parametrize("N,T", [(1, 1), (5, 700), (64, 1000), (65, 513), (130, 4096)])
def test_xengine_tc_int8_exact(N, T):
    _dev()
    g = torch.Generator(device="cuda").manual_seed(11 * N + T)
    x = torch.randint(-127, 128, (1, T, N, 2), generator=g, device="cuda", dtype=torch.int8)
    Xh, _ = acf.transpose_raw(x, out_kind="f16")
    V = acf.xengine("int8", Xh, None, N, T)
    torch.cuda.synchronize()
    ref = oracle.correlate_int(x[0].cpu().numpy())
    assert np.array_equal(V[0].cpu().numpy(), ref)


def test_xengine_tc_int8_full_scale_beyond_int32():
    """Full-scale samples for 140,000 spectra: every partial sum hits its bound
    (chunks of 512, items split at 65,536) and V_ii exceeds 2^31."""
    _dev()
    T, N = 140000, 4
    x = torch.empty((1, T, N, 2), dtype=torch.int8, device="cuda")
    x[..., 0] = 127
    x[..., 1] = -127
    x[0, :, 1, 0] = -127
    x[0, ::3, 2, 1] = 127
    Xh, _ = acf.transpose_raw(x, out_kind="f16")
    V = acf.xengine("int8", Xh, None, N, T)
    torch.cuda.synchronize()
    ref = oracle.correlate_int(x[0].cpu().numpy())
    assert ref[0, 0] > 2 ** 31
    assert np.array_equal(V[0].cpu().numpy(), ref)


# ---------------------------------------------------------------- full stage
def test_correlator_tiny_fp32():
    """One station, one subband of ci8, 64 channels x 16 taps, FP32 path."""
    w = synth.WORKLOADS["tiny"]
    _dev()
    sky = synth.make_sky(w["n_inputs"], w["n_sources"], w["flux"], w["seed"])
    x = synth.voltages(w["n_inputs"], w["n_samples"], 1, "ci8", w["sigma"], sky, w["seed"], device="cuda")
    with acf.Correlator(w["n_inputs"], 1, 64, 16, 1, "fp32", "ci8", w["n_samples"]) as c:
        c.push(x)
        V = c.visibilities()
        assert c.query()["last_spectra"] == 290
    torch.cuda.synchronize()
    ref = oracle.correlator(x[0].cpu().numpy(), 16, 64)[0]
    assert norm_err(_np_complex(V[0]), ref, w["n_inputs"]) <= TOL_FP32


def test_correlator_streaming_history_and_integrations():
    _dev()
    N, C, P = 24, 16, 16
    pushes = [300, 1000, 777, 64, 2000]
    S = sum(pushes)
    x = _samples(N, S, 2, "ci16", sigma=512.0, seed=21)
    xs = x.cpu().numpy()
    # 5 pushes, integrations of 2 pushes -> 2 complete integrations (5th push pending)
    with acf.Correlator(N, 2, C, P, 2, "fp32", "ci16", max(pushes)) as c:
        outs = []
        t0 = 0
        for k, n in enumerate(pushes):
            c.push(x[:, t0:t0 + n].contiguous())
            t0 += n
            V = c.visibilities()
            if V is not None:
                outs.append(V.clone())
        assert len(outs) == 2
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(xs[sb], P, C, push_sizes=pushes, n_integrate=2)
        for k in range(2):
            assert norm_err(_np_complex(outs[k][sb]), ref[k], N) <= TOL_FP32


def test_correlator_rejects_unread_integration():
    _dev()
    x = _samples(8, 2000, 1, "ci8", seed=2)
    with acf.Correlator(8, 1, 16, 16, 1, "fp32", "ci8", 2000) as c:
        c.push(x)
        with pytest.raises(acf.AcfError) as e:
            c.push(x)
        assert e.value.status == 4
        assert c.visibilities() is not None
        c.push(x)


@pytest.mark.parametrize("mode,tol", [("fp16", TOL_FP16), ("fp16x3", TOL_FP32), ("fp32", TOL_FP32)])
def test_correlator_precision_modes_ci16(mode, tol):
    _dev()
    N, C, P, S = 70, 64, 16, 64 * 60 + 9
    sky = synth.make_sky(N, 3, (0.05, 0.5), 31)
    x = synth.voltages(N, S, 2, "ci16", 512.0, sky, 31, device="cuda")
    with acf.Correlator(N, 2, C, P, 1, mode, "ci16", S) as c:
        c.push(x)
        V = c.visibilities()
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlator(x[sb].cpu().numpy(), P, C)[0]
        assert norm_err(_np_complex(V[sb]), ref, N) <= tol


def test_correlator_int8_raw_exact():
    _dev()
    N, S = 96, 20000
    x = _samples(N, S, 2, "ci8", seed=41, n_src=2)
    with acf.Correlator(N, 2, 1, 1, 1, "int8", "ci8", S) as c:
        c.push(x)
        V = c.visibilities()
    torch.cuda.synchronize()
    for sb in range(2):
        ref = oracle.correlate_int(x[sb].cpu().numpy())
        assert np.array_equal(V[sb, 0].cpu().numpy(), ref)


def test_correlator_raw_fp32_and_host_push():
    _dev()
    N, S = 40, 5000
    x = _samples(N, S, 3, "ci8", seed=42)
    with acf.Correlator(N, 3, 1, 1, 1, "fp32", "ci8", S) as c:
        c.push(x.cpu().pin_memory())       # host path: staged copies + overlap
        V = c.visibilities(out=torch.empty((3, 1, N * (N + 1) // 2, 2)).pin_memory())
        torch.cuda.synchronize()
    for sb in range(3):
        ref = oracle.correlate_int(x[sb].cpu().numpy())
        refc = ref[:, 0] + 1j * ref[:, 1]
        assert norm_err(V[sb, 0].numpy().astype(np.complex128), refc[None], N) <= TOL_FP32


@pytest.mark.parametrize("C,mode", [(64, "fp16"), (1, "int8")])
def test_host_pushes_back_to_back_match_device_pushes(C, mode):
    """Consecutive host pushes of different data, each integration read back
    (to host) right after its push and nothing synchronised in between: a
    push's host-to-device copies wait only for the previous push's readers of
    the staging, so they overlap the previous X-engine and read-back.  Every
    integration equals the same pushes made from device memory, bit for bit."""
    _dev()
    N, n_sb, S, n_push = 96, 3, 20000, 4
    P = 16 if C > 1 else 1
    xs = [_samples(N, S, n_sb, "ci8", seed=500 + k) for k in range(n_push)]
    hosts = [x.cpu().pin_memory() for x in xs]
    NB = N * (N + 1) // 2
    dt = torch.int64 if mode == "int8" else torch.float32
    outs = [torch.empty((n_sb, C, NB, 2), dtype=dt).pin_memory() for _ in range(n_push)]
    with acf.Correlator(N, n_sb, C, P, 1, mode, "ci8", S) as c:
        for k in range(n_push):
            c.push(hosts[k])
            c.visibilities(out=outs[k])
        torch.cuda.synchronize()
    with acf.Correlator(N, n_sb, C, P, 1, mode, "ci8", S) as c:
        for k in range(n_push):
            c.push(xs[k])
            ref = c.visibilities().cpu()
            got = outs[k] if mode == "int8" else torch.view_as_complex(outs[k])
            assert torch.equal(got, ref), k


def test_bandpass_weights_apply_per_channel():
    _dev()
    N, C, P, S = 12, 16, 16, 16 * 60
    x = _samples(N, S, 1, "ci8", seed=43)
    w = synth.bandpass_ripple(C, 3)
    with acf.Correlator(N, 1, C, P, 1, "fp32", "ci8", S) as c:
        c.set_bandpass(w)
        c.push(x)
        V = c.visibilities()
    torch.cuda.synchronize()
    ref = oracle.correlator(x[0].cpu().numpy(), P, C, bandpass=w.astype(np.float64))[0]
    assert norm_err(_np_complex(V[0]), ref, N) <= TOL_FP32


# ---------------------------------------------------------------- gain
def _gain_problem(N=48, C=4, seed=51):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((C, N, 6)) + 1j * rng.standard_normal((C, N, 6))
    full = A @ A.conj().transpose(0, 2, 1)
    ii, jj = tri_index(N)
    R = full[:, ii, jj]
    gt = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    Vfull = gt[None, :, None] * full * gt.conj()[None, None, :]
    noise = 0.05 * (rng.standard_normal(R.shape) + 1j * rng.standard_normal(R.shape))
    noise[:, ii == jj] = noise[:, ii == jj].real          # observed autocorrelations are real
    V = Vfull[:, ii, jj] + noise
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))
    return R, V, g


def test_gain_forward_adjoint_vs_oracle():
    _dev()
    for N, C in [(48, 4), (1, 1), (130, 3)]:
        R, V, g = _gain_problem(N, C)
        t = lambda a: torch.as_tensor(a, dtype=torch.complex64, device="cuda")
        loss, grad = acf.gain_loss_and_grad(t(g), t(R), t(V))
        torch.cuda.synchronize()
        Lref, gref = oracle.gain_loss_grad(R, V, g)
        assert abs(loss.item() - Lref) <= 1e-5 * Lref
        assert np.max(np.abs(grad.cpu().numpy() - gref)) <= 1e-4 * np.max(np.abs(gref))
        g2 = acf.gain_grad(t(g), t(R), t(V))
        assert torch.allclose(g2, grad, rtol=1e-5, atol=1e-5 * grad.abs().max().item())


def test_gain_autograd_and_finite_differences():
    """Differentiable calibration: torch autograd through the adjoint kernel;
    FP32 central differences (h = 1e-3) agree to 1e-3 relative."""
    _dev()
    R, V, g = _gain_problem(32, 3, seed=52)
    t = lambda a: torch.as_tensor(a, dtype=torch.complex64, device="cuda")
    gt = t(g).requires_grad_(True)
    loss = acf.GainCorr.apply(gt, t(R), t(V))
    loss.backward()
    grad = gt.grad.detach().cpu().numpy()
    h = 1e-3
    fd = np.zeros_like(g)
    for k in range(len(g)):
        for unit in (1.0, 1j):
            gp, gm = g.copy(), g.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            lp = acf.gain_loss_and_grad(t(gp), t(R), t(V), want_grad=False)[0].item()
            lm = acf.gain_loss_and_grad(t(gm), t(R), t(V), want_grad=False)[0].item()
            fd[k] += (lp - lm) / (2 * h) * unit
    # norm-wise relative error: fp32 loss rounding (~1e-7 L) over 2h dominates single entries
    rel = np.linalg.norm(grad - fd) / np.linalg.norm(fd)
    assert rel <= 1e-3
    _, gref = oracle.gain_loss_grad(R, V, g)
    assert np.linalg.norm(grad - gref) / np.linalg.norm(gref) <= 1e-5
    # and the same gradient from torch's own autograd of the plain formula (fp64)
    gd = torch.as_tensor(g, dtype=torch.complex128).requires_grad_(True)
    Rf = torch.zeros((3, 32, 32), dtype=torch.complex128)
    Vf = torch.zeros_like(Rf)
    ii, jj = tri_index(32)
    Rf[:, ii, jj] = torch.as_tensor(R)
    Rf[:, jj, ii] = torch.as_tensor(R).conj()
    Vf[:, ii, jj] = torch.as_tensor(V)
    Vf[:, jj, ii] = torch.as_tensor(V).conj()
    M = gd[None, :, None] * Rf * gd.conj()[None, None, :]
    ((M - Vf).abs() ** 2).sum().backward()
    assert np.max(np.abs(grad - gd.grad.numpy())) <= 1e-4 * np.max(np.abs(gd.grad.numpy()))


# ---------------------------------------------------------------- ragged batch
def test_batch_ragged_mixed_modes():
    _dev()
    jobs = [dict(n_inputs=10, n_channels=1, n_taps=1, n_samples=3000),
            dict(n_inputs=33, n_channels=16, n_taps=16, n_samples=5000),
            dict(n_inputs=96, n_channels=64, n_taps=16, n_samples=4096 + 64 * 15),
            dict(n_inputs=5, n_channels=256, n_taps=16, n_samples=256 * 20),
            dict(n_inputs=130, n_channels=1, n_taps=1, n_samples=1000)]
    b = acf.Batch(jobs, autotune=False)
    ins = [synth.voltages(j["n_inputs"], j["n_samples"], 1, "ci8", 16.0, None, 60 + k, device="cuda")[0]
           for k, j in enumerate(jobs)]
    outs = b.outputs()
    for rep in range(2):                  # capture, then replay the graph
        b.run(ins, outs)
        torch.cuda.synchronize()
        for k, j in enumerate(jobs):
            x = ins[k].cpu().numpy()
            if j["n_channels"] == 1:
                assert np.array_equal(outs[k][0].cpu().numpy(), oracle.correlate_int(x))
            else:
                ref = oracle.correlator(x, j["n_taps"], j["n_channels"])[0]
                assert norm_err(_np_complex(torch.view_as_complex(outs[k])), ref, j["n_inputs"]) <= TOL_FP32
    b.close()


@pytest.mark.parametrize("pair,n_tile,k_split,order", [(1, 256, 1, 2), (0, 128, 2, 2), (0, 256, 1, 1), (1, 256, 4, 0)])
def test_batch_fixed_plans_match_oracle(pair, n_tile, k_split, order):
    """Plans fixed through acf_batch_set_plan.  Order 2 interleaves the tiles of
    the short-integration jobs (256 channels, 4 and 7 spectra: one K step)
    among those of the raw and 64-channel jobs, through a work-order table;
    every plan, CTA pairs or one SM per tile, gives the oracle's result
    (raw jobs bit-exact), on the captured graph and its replay."""
    _dev()
    jobs = [dict(n_inputs=70, n_channels=256, n_taps=16, n_samples=256 * 19),
            dict(n_inputs=150, n_channels=1, n_taps=1, n_samples=5000),
            dict(n_inputs=33, n_channels=256, n_taps=16, n_samples=256 * 22),
            dict(n_inputs=96, n_channels=64, n_taps=16, n_samples=64 * 315)]
    b = acf.Batch(jobs, autotune=False)
    b.set_plan(pair, n_tile, k_split, order)
    q = b.query()
    assert (q["pair"], q["n_tile"], q["k_split"], q["order"]) == (pair, n_tile, k_split, order)
    ins = [synth.voltages(j["n_inputs"], j["n_samples"], 1, "ci8", 16.0, None, 90 + k, device="cuda")[0]
           for k, j in enumerate(jobs)]
    outs = b.outputs()
    refs = {}
    for rep in range(2):
        b.run(ins, outs)
        torch.cuda.synchronize()
        for k, j in enumerate(jobs):
            x = ins[k].cpu().numpy()
            if j["n_channels"] == 1:
                assert np.array_equal(outs[k][0].cpu().numpy(), oracle.correlate_int(x))
            else:
                if k not in refs:
                    refs[k] = oracle.correlator(x, j["n_taps"], j["n_channels"])[0]
                assert norm_err(_np_complex(torch.view_as_complex(outs[k])), refs[k], j["n_inputs"]) <= TOL_FP32
    with pytest.raises(acf.AcfError):
        b.set_plan(1, 128, 1, 0)          # CTA pairs always use 256-row tiles
    assert b.query()["order"] == order
    b.close()


def test_batch_autotune_picks_valid_tiles():
    _dev()
    jobs = [dict(n_inputs=64, n_channels=1, n_taps=1, n_samples=2000),
            dict(n_inputs=40, n_channels=16, n_taps=16, n_samples=3000)]
    b = acf.Batch(jobs, autotune=True)
    q = b.query()
    assert q["n_tile"] in (128, 256) and q["k_split"] in (1, 2, 4)
    ins = [synth.voltages(j["n_inputs"], j["n_samples"], 1, "ci8", 16.0, None, 70 + k, device="cuda")[0]
           for k, j in enumerate(jobs)]
    outs = b.outputs()
    b.run(ins, outs)
    torch.cuda.synchronize()
    assert np.array_equal(outs[0][0].cpu().numpy(), oracle.correlate_int(ins[0].cpu().numpy()))
    ref = oracle.correlator(ins[1].cpu().numpy(), 16, 16)[0]
    assert norm_err(_np_complex(torch.view_as_complex(outs[1])), ref, 40) <= TOL_FP32
    b.close()


# ---------------------------------------------------------------- device status
def test_no_device_wait_timed_out():
    _dev()
    assert acf.device_status() == 0
