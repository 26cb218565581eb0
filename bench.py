"""Benchmark of the correlator stage on one B300.

Default workload: the AARTFAAC-12-shaped array -- 576 dual-polarisation
antennas (1152 inputs), 16 subbands of complex int16 samples (sigma 512, three
point sources), 195,313 samples per subband per 1 s integration, a 16-tap x
64-channel filter bank.  One step = one 1 s integration pushed through the
whole stage: channeliser (FIR + FFT + bandpass + transpose, fp16 output) and
the tcgen05 X-engine in FP16 mode.  The metric is useful X-engine tera-ops
per second: 8 * N(N+1)/2 * spectra * channels * subbands per step.

Also measured in the same run (reported as extra keys): the split-FP16 mode
and the plain FP32 CUDA-core path on the same workload, the INT8-exact raw
subband X-engine on the AARTFAAC-6-shaped array (576 inputs, 8 subbands), the
channeliser's HBM throughput, an end-to-end pass through the C ABI with host
buffers, and the fp64 CPU oracle on a bounded sample (cpu_baseline).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl acf|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "X-engine TOPS & frac of INT8/FP16 TC peak at 576 ants vs plain FP32 GPU path"
UNIT = "TOPS"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"], src="measured",
                    sm_max_mhz=d.get("sm_max_mhz", 2032.0))
    return dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, src="fallback", sm_max_mhz=2032.0)


def fp32_fma_peak_tflops(torch, sm_max_mhz):
    """FP32 FMA peak of the device: SMs x 128 lanes x 2 flops x max SM clock."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12


def xeng_traffic_per_subband():
    """DRAM bytes per subband of the X-engine launch from the committed ncu
    capture (profiles/xeng_traffic.json), valid only while the kernel source
    is the one that was captured (a one-subband capture, scaled by subbands:
    subbands are independent problems, so traffic grows in proportion)."""
    import hashlib
    side = os.path.join(ROOT, "profiles", "xeng_traffic.json")
    try:
        d = json.load(open(side))
        src = os.path.join(ROOT, d["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == d["source_sha256_16"]:
            return int(d["traffic_per_subband_bytes"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def xops(N, T, n_ch, n_sb):
    """Algorithmic X-engine ops: one complex MAC (8 real ops) per baseline per spectrum."""
    return 8.0 * N * (N + 1) / 2 * T * n_ch * n_sb


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


ACC_CHANS = [0, 17]          # channels of subband 0 the oracle leg computes
INT8_ACC_INPUTS = 64         # inputs of A-6 subband 0 the exact integer oracle sums


def cpu_oracle_sample(x0=None, push=1):
    """fp64 oracle on a bounded slice of the default workload: subband 0, two
    channels, all 1152 inputs, one 1 s push (3036-3052 spectra).  x0 is
    subband 0 of the benchmark's own input ([S, N, 2] int16, host), which the
    benchmark pushes again every step; the oracle then reproduces push number
    `push` of that periodic stream (195,313 is not a multiple of 64, so each
    push's spectra start 49 samples further into the block).  Without x0 the
    slice is drawn here and the first push is computed.  Returns the timing
    and the oracle's V."""
    import numpy as np

    import oracle
    import synth
    w = synth.WORKLOADS["a12"]
    N, S = w["n_inputs"], w["n_samples"]
    if x0 is None:
        sky = synth.make_sky(N, w["n_sources"], w["flux"], w["seed"])
        x0 = synth.voltages(N, S, 1, "ci16", w["sigma"], sky, w["seed"], device="cpu")[0].numpy()
    C, P = w["n_channels"], w["n_taps"]
    h = oracle.prototype(P, C)
    m0 = oracle.n_spectra((push - 1) * S, P, C)
    m1 = oracle.n_spectra(push * S, P, C)
    t = np.arange(m0 * C, (m1 - 1) * C + P * C) % S        # stream samples of those windows
    seg = x0[t]
    t0 = time.perf_counter()
    X = oracle.channelise(seg, h, P, C, m_begin=0, m_end=m1 - m0, chans=ACC_CHANS)
    V = oracle.correlate(X)
    dt = time.perf_counter() - t0
    T = X.shape[2]
    ops = xops(N, T, len(ACC_CHANS), 1)
    assert np.isfinite(V).all()
    return dict(value=ops / dt / 1e12, unit=UNIT, cores=oracle.max_threads(), kind="oracle",
                sample="A-12 workload, subband 0, channels {0, 17}, 1152 inputs, one 1 s push (%d spectra); "
                       "fp64 direct FIR + naive DFT + brute-force pairs, %.1f s" % (T, dt), seconds=dt), V


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample()
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample()[0])
    v = statistics.median([r["value"] for r in vals])
    secs = sum(r["seconds"] for r in vals)
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * secs / max(1, args.steps), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload="A-12: 1152 inputs x 16 subbands x 195313 ci16 samples, 64 ch x 16 taps; "
                                     "oracle timed on subband 0, 2 channels"),
                impl="reference", cpu_baseline=dict(vals[-1], value=v),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    line["cpu_baseline"].pop("seconds", None)
    print(json.dumps(line))
    return 0


def norm_err(V, R, n):
    """max |dV_ij| / sqrt(V_ii V_jj) of V against R ([channels, NB] complex)."""
    import numpy as np
    i = np.repeat(np.arange(n), np.arange(1, n + 1))
    j = np.concatenate([np.arange(k + 1) for k in range(n)])
    d = np.arange(n) * (np.arange(n) + 1) // 2 + np.arange(n)
    auto = R[:, d].real
    return float(np.max(np.abs(V - R) / np.sqrt(auto[:, i] * auto[:, j])))


def xeng_desc(t):
    """Kernel and launch shape of an X-engine tuning (acf_query_xengine)."""
    if not t:
        return "k_xeng_simt"
    kern = "k_xeng_tc2: SM pairs per 256x256 tile" if t["variant"] else "k_xeng_tc: one SM per 128x%d tile" % t["n_tile"]
    return "%s, time split %d, %s" % (kern, t["k_split"], "autotuned" if t["tuned"] else "creation rule")


def time_mode(acf, torch, x, w, mode, steps, warmup, stream, flush=None, keep=None):
    """Steps of the whole stage in one precision mode; returns dict with timings.
    keep(out) -> host copy of the part of the last step's visibilities the
    accuracy check compares with the oracle."""
    N, n_sb, C, P = w["n_inputs"], w["n_subbands"], w["n_channels"], w["n_taps"]
    S = w["n_samples"]
    c = acf.Correlator(N, n_sb, C, P, 1, mode, w["dtype"], S)
    # the context's autotuner picks the X-engine launch shape on this geometry
    # (untimed), on the operands of one warm-up integration of the live
    # samples; the FP32 comparison path has none
    tuning = None
    extra = 0
    if mode != "fp32":
        with torch.cuda.stream(stream):
            c.push(x, stream)
            c.release(stream)
        stream.synchronize()
        tuning = c.tune()
        extra = 1                  # that push counts in the stream the oracle reproduces
    c.enable_timing(True)
    Ts, chan_ms, xeng_ms = [], [], []
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            c.push(x, stream)
            c.release(stream)
        stream.synchronize()
        l0 = acf.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        total_ms = 0.0
        for _ in range(steps):
            # one step: push one second, hand the integration out in place
            # (it stays in HBM for the next stage; the e2e leg copies it out)
            e0.record(stream)
            c.push(x, stream)
            c.release(stream)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            Ts.append(c.query()["last_spectra"])
            a, b = c.last_timing()
            chan_ms.append(a)
            xeng_ms.append(b)
        launches = acf.launch_count() - l0
    kept = keep(c.device_visibilities()) if keep is not None else None
    c.close()
    ops = sum(xops(N, T, C, n_sb) for T in Ts)
    return dict(ms_per_step=total_ms / steps, tops=ops / (total_ms * 1e-3) / 1e12, T=Ts,
                chan_ms=statistics.median(chan_ms), xeng_ms=statistics.median(xeng_ms),
                xeng_tops=xops(N, statistics.median(Ts), C, n_sb) / (statistics.median(xeng_ms) * 1e-3) / 1e12,
                launches=launches, ops_per_step=ops / steps, kept=kept, pushes=extra + warmup + steps,
                xengine_tuning=tuning)


def time_post(acf, torch, pk, N, n_sb, C, oracle_sample=True):
    """The post-correlation kernels (delay compensation, channel integration by
    4, two-stage sigma clip, lost-data weights for one second of 16-sample
    packets, re-weighting) on a full A-12 visibility set [16][64][NB], each
    timed with CUDA events through the C ABI (outputs preallocated), with the
    numpy oracle timed on a bounded sample beside it."""
    import ctypes
    import numpy as np
    from paper_1609_04205_b300 import _lib as A
    L = A.lib()
    NB = N * (N + 1) // 2
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(7)
    V = torch.randn((n_sb, C, NB, 2), generator=g, device=dev)
    Vout = torch.empty((n_sb, C // 4, NB, 2), device=dev)
    flags = torch.empty((n_sb, C, NB), dtype=torch.uint8, device=dev)
    nblk = 195313 // 16 + 1
    mask = (torch.rand((nblk, N), generator=g, device=dev) < 0.97).to(torch.uint8)
    W = torch.empty(NB, dtype=torch.int64, device=dev)
    fs = 195312.5
    d = np.ascontiguousarray(np.random.default_rng(3).uniform(-2e-6, 2e-6, N))
    fc = np.ascontiguousarray((300 + np.arange(n_sb)) * fs)
    vp = ctypes.c_void_p
    hs = A.stream_handle(None)
    vb = V.numel() * 4
    ops = {
        "delay_compensate": (lambda: L.acf_delay_compensate(A.ptr(V), n_sb, C, N, d.ctypes.data_as(vp),
                                                             fc.ctypes.data_as(vp), fs, hs), 2 * vb, n_sb * C * NB),
        "integrate_channels_by4": (lambda: L.acf_integrate_channels(A.ptr(V), A.ptr(Vout), n_sb, C, N, 4, 0, hs),
                                   vb + vb // 4, n_sb * C * NB),
        "sigma_clip": (lambda: L.acf_sigma_clip(A.ptr(V), A.ptr(flags), n_sb, C, N, 5.0, 3.0, hs),
                       2 * vb + flags.numel(), n_sb * C * NB),
        "lost_sample_weights": (lambda: L.acf_lost_sample_weights(A.ptr(mask), nblk, N, 16, A.ptr(W), hs),
                                mask.numel() + W.numel() * 8, NB),
        "reweight": (lambda: L.acf_reweight(A.ptr(V), A.ptr(W), 195313, n_sb * C, N, hs), 2 * vb + W.numel() * 8,
                     n_sb * C * NB),
    }
    out = {}
    for name, (fn, nbytes, elems) in ops.items():
        for _ in range(2):
            A.check(fn())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            A.check(fn())
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = dict(ms=ms, gbs=gbs, frac_hbm=gbs / pk["hbm"], bytes=nbytes, gpu_elems_per_s=elems / (ms * 1e-3))
    out["workload"] = "A-12 visibilities: 16 subbands x 64 channels x 664128 baselines (5.44 GB cf32); " \
                      "weights: 12208 blocks x 1152 inputs"
    del V, Vout, flags, mask, W
    torch.cuda.empty_cache()
    if oracle_sample:
        from oracle import post
        rng = np.random.default_rng(5)
        samples = {}
        Vs = rng.normal(size=(1, 1, NB)) + 1j * rng.normal(size=(1, 1, NB))
        t0 = time.perf_counter(); post.delay_compensate(Vs, d, fc[:1], fs); dt = time.perf_counter() - t0
        samples["delay_compensate"] = (NB / dt, "1 channel of 1 subband, full triangle")
        Vs = rng.normal(size=(1, C, 20000)) + 1j * rng.normal(size=(1, C, 20000))
        t0 = time.perf_counter(); post.integrate_channels(Vs, 4); dt = time.perf_counter() - t0
        samples["integrate_channels_by4"] = (C * 20000 / dt, "64 channels x 20000 baselines")
        n2 = 128
        Vs = rng.normal(size=(1, C, n2 * (n2 + 1) // 2)) + 1j * rng.normal(size=(1, C, n2 * (n2 + 1) // 2))
        t0 = time.perf_counter(); post.sigma_clip(Vs, 5.0, 3.0); dt = time.perf_counter() - t0
        samples["sigma_clip"] = (Vs.size / dt, "128 inputs x 64 channels")
        m = (rng.uniform(size=(nblk, 64)) < 0.97)
        t0 = time.perf_counter(); post.lost_sample_weights(m, 16); dt = time.perf_counter() - t0
        samples["lost_sample_weights"] = (64 * 65 // 2 / dt, "64 inputs, 12208 blocks")
        Vs = rng.normal(size=(1, 1, NB)) + 1j * rng.normal(size=(1, 1, NB))
        Ws = rng.integers(1, 195313, NB)
        t0 = time.perf_counter(); post.reweight(Vs, Ws, 195313); dt = time.perf_counter() - t0
        samples["reweight"] = (NB / dt, "1 channel of 1 subband, full triangle")
        for k, (v, what) in samples.items():
            out[k]["cpu_baseline"] = dict(value=v, unit="elements/s", kind="oracle", cores=1, sample=what)
    return out


def time_batch(acf, torch, synth, pk, steps=10):
    """Ragged batch: 32 independent arrays (48-576 antennas, 16/64/256 channels
    or raw, 0.25 s each; half raw INT8-exact, half channelised split FP16) run
    as one persistent work list in one CUDA graph, autotuned.  Useful X-engine
    ops over the CUDA-event time of whole batch runs (channelisers included)."""
    jobs = synth.ragged_jobs()
    b = acf.Batch(jobs, autotune=True)
    ins = [synth.voltages(j["n_inputs"], j["n_samples"], 1, "ci8", 16.0, None, j["seed"], device="cuda")[0]
           for j in jobs]
    outs = b.outputs()
    for _ in range(3):                      # autotune, graph capture, warm replay
        b.run(ins, outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        b.run(ins, outs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    useful = issued = 0.0
    for j in jobs:
        C, P, S, N = j["n_channels"], j["n_taps"], j["n_samples"], j["n_inputs"]
        T = S if C == 1 else (S - (P - 1) * C) // C
        ops = xops(N, T, C, 1)
        useful += ops
        issued += ops if C == 1 else 3 * ops
    q = b.query()
    b.close()
    tops = useful / (ms * 1e-3) / 1e12
    return dict(ms=ms, useful_tops=tops, issued_tensor_tops=issued / (ms * 1e-3) / 1e12,
                frac_of_sustained_issued=issued / (ms * 1e-3) / 1e12 / pk["bf16_sus"], tuning=q,
                workload="32 arrays: 96-1152 inputs, 16/64/256 channels or raw, 48828 ci8 samples each; "
                         "raw jobs INT8 exact, channelised jobs split FP16; one CUDA-graph replay per run")


def time_channeliser_alone(torch, x, w, pk, steps=5):
    """The headline's channelisation (every subband, 64 channels x 16 taps, fp16
    operand out, no history) launched by itself through acf_channelise on the
    resident input: CUDA events around `steps` back-to-back calls."""
    import ctypes
    from paper_1609_04205_b300 import _lib as A
    L = A.lib()
    n_sb, S, N = x.shape[0], x.shape[1], x.shape[2]
    C, P = w["n_channels"], w["n_taps"]
    T = (S - P * C) // C + 1
    ts = (T + 63) // 64 * 64
    h = torch.as_tensor(prototype_of(P, C), device=x.device)
    bp = torch.ones(C, dtype=torch.float32, device=x.device)
    X = torch.empty((n_sb, C, 2 * N, ts), dtype=torch.float16, device=x.device)
    To = ctypes.c_long(0)
    run = lambda: A.check(L.acf_channelise(None, 0, A.ptr(x), S, A.DTYPES[w["dtype"]], n_sb, N, C, P, A.ptr(h),
                                           A.ptr(bp), A.OUT_F16, A.ptr(X), None, ts, 0.125, ctypes.byref(To),
                                           A.stream_handle(None)))
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nbytes = x.numel() * x.element_size() + X[..., :T].numel() * 2
    del X
    torch.cuda.empty_cache()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return dict(ms=ms, gbs=gbs, frac_hbm=gbs / pk["hbm"], bytes=nbytes, kernel="k_ppf64_tc")


def prototype_of(P, C):
    import paper_1609_04205_b300 as acf
    return acf.prototype(P, C)


def time_gain(acf, torch, pk, N=576, C=64, steps=20):
    """Gain forward (loss) + adjoint (gradient) in one pass over packed R and V:
    576 inputs, 64 channels, complex float32."""
    from paper_1609_04205_b300 import _lib as A
    L = A.lib()
    NB = N * (N + 1) // 2
    g0 = torch.Generator(device="cuda").manual_seed(11)
    R = torch.randn((C, NB, 2), generator=g0, device="cuda")
    V = torch.randn((C, NB, 2), generator=g0, device="cuda")
    g = torch.randn((N, 2), generator=g0, device="cuda")
    loss = torch.empty((), device="cuda")
    grad = torch.empty((N, 2), device="cuda")
    hs = A.stream_handle(None)
    run = lambda: A.check(L.acf_gain_forward(A.ptr(R), A.ptr(V), A.ptr(g), N, C, A.ptr(loss), A.ptr(grad), hs))
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nbytes = 2 * C * NB * 8
    gbs = nbytes / (ms * 1e-3) / 1e9
    return dict(ms=ms, gbs=gbs, frac_hbm=gbs / pk["hbm"], bytes=nbytes,
                workload="576 inputs x 64 channels, packed R and V complex float32 (loss + gradient)")


def aggregate(ms_local, ops_local, device="cpu"):
    """Whole-job figures across ranks: step time = max over ranks, value =
    the ops of all ranks over that time (weak scaling: each rank correlates
    its own subband set; no data moves between ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, ops_local / (ms_local * 1e-3) / 1e12
    t = torch.tensor([ms_local, ops_local], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms = float(mx[0].item())
    return ms, float(tot[1].item()) / (ms * 1e-3) / 1e12


def profile_case_kernels(which):
    """Small cases of single kernels for ncu captures (a few GB on the device):
    sigma_clip -- acf_sigma_clip on four A-12 subbands of visibilities (1.36 GB);
    batch -- the ragged batch: autotune, graph capture, then two replays;
    gain -- acf_gain_forward on 576 inputs x 64 channels;
    chan256 -- acf_channelise, 256 channels x 16 taps, 1152 inputs x 48,828 ci8
    samples to split fp16.  Four calls each."""
    import ctypes

    import torch

    import paper_1609_04205_b300 as acf
    import synth
    from paper_1609_04205_b300 import _lib as A
    L = A.lib()
    hs = A.stream_handle(None)
    g = torch.Generator(device="cuda").manual_seed(7)
    if which == "sigma_clip":
        N, n_sb, C = 1152, 4, 64
        V = torch.randn((n_sb, C, N * (N + 1) // 2, 2), generator=g, device="cuda")
        flags = torch.empty((n_sb, C, N * (N + 1) // 2), dtype=torch.uint8, device="cuda")
        for _ in range(4):
            A.check(L.acf_sigma_clip(A.ptr(V), A.ptr(flags), n_sb, C, N, 5.0, 3.0, hs))
    elif which == "gain":
        time_gain(acf, torch, peaks(), steps=1)
    elif which == "batch":
        time_batch(acf, torch, synth, peaks(), steps=2)
    elif which == "chan256":
        N, S, C, P = 1152, 48828, 256, 16
        x = torch.randint(-100, 100, (1, S, N, 2), dtype=torch.int8, device="cuda", generator=g)
        T = (S - (P - 1) * C) // C
        ts = (T + 63) // 64 * 64
        X = torch.empty((1, C, 2 * N, ts), dtype=torch.float16, device="cuda")
        Xl = torch.empty_like(X)
        h = torch.as_tensor(acf.prototype(P, C), device="cuda")
        bp = torch.ones(C, device="cuda")
        To = ctypes.c_long()
        for _ in range(4):
            A.check(L.acf_channelise(None, 0, A.ptr(x), S, A.DTYPES["ci8"], 1, N, C, P, A.ptr(h), A.ptr(bp), 2,
                                     A.ptr(X), A.ptr(Xl), ts, 0.25, ctypes.byref(To), hs))
    torch.cuda.synchronize()
    print("profile case %s done" % which)
    return 0


def profile_case(mode):
    import torch

    import paper_1609_04205_b300 as acf
    import synth
    if mode in ("sigma_clip", "gain", "chan256", "batch"):
        return profile_case_kernels(mode)
    w = dict(synth.WORKLOADS["a6" if mode == "int8" else "a12"])
    w["n_subbands"] = 1
    if mode == "int8":
        w.update(n_channels=1, n_taps=1, dtype="ci8")
    sky = synth.make_sky(w["n_inputs"], w["n_sources"], w["flux"], w["seed"]) if w["n_sources"] else None
    x = synth.voltages(w["n_inputs"], w["n_samples"], 1, w["dtype"], w["sigma"], sky, w["seed"], device="cuda")
    with acf.Correlator(w["n_inputs"], 1, w["n_channels"], w["n_taps"], 1, mode, w["dtype"], w["n_samples"]) as c:
        out = c.empty_visibilities()
        if mode != "fp32":
            c.push(x)                  # tune on one integration of the live samples
            c.visibilities(out)
            c.tune()
        for _ in range(4):
            c.push(x)
            c.visibilities(out)
        torch.cuda.synchronize()
    print("profile case %s done" % mode)
    return 0


def probe():
    """The tensor-pipe ceiling with resident operands, beside the measured
    cuBLAS peaks: how far above the copy-bound denominators the MMA units
    themselves go.  Clocks are sampled during the runs."""
    import torch

    import paper_1609_04205_b300 as acf
    pk = peaks()
    acf.probe_tensor_peak(8192)                      # warm the clocks and the module
    clk = Clocks(0)
    runs = [acf.probe_tensor_peak(65536) for _ in range(60)]      # ~1 s under the clock sampler
    clocks = clk.stop()
    best = max(r["tflops"] for r in runs)
    print(json.dumps(dict(probe="tcgen05 kind::f16 M128 N256 K16, operands resident in shared memory, one CTA per SM",
                          tflops_median=statistics.median(r["tflops"] for r in runs), ms_median=statistics.median(
                              r["ms"] for r in runs), best_tflops=best, runs=len(runs),
                          vs_measured_bf16_burst=best / pk["bf16"], vs_measured_bf16_sustained=best / pk["bf16_sus"],
                          nominal_dense_fp16_tflops=2250.0, clocks=clocks, torch=torch.__version__)))
    return 0


def post_case():
    """The post-correlation kernels alone on the A-12 visibility set (the same
    calls as the bench line's `post` object, without the oracle), then the gain
    forward/adjoint, for profiling."""
    import torch

    import paper_1609_04205_b300 as acf
    r = time_post(acf, torch, peaks(), 1152, 16, 64, oracle_sample=False)
    for k, v in r.items():
        if isinstance(v, dict):
            print("%-26s %8.3f ms %8.1f GB/s  frac %.3f" % (k, v["ms"], v["gbs"], v["frac_hbm"]))
    v = time_gain(acf, torch, peaks())
    print("%-26s %8.3f ms %8.1f GB/s  frac %.3f" % ("gain_forward", v["ms"], v["gbs"], v["frac_hbm"]))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="acf", choices=["acf", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the comparison modes and the e2e pass")
    ap.add_argument("--post-case", action="store_true",
                    help="run only the post-correlation kernels on the A-12 visibility set (profiling)")
    ap.add_argument("--probe", action="store_true",
                    help="tensor-pipe rate with operands resident in shared memory (one JSON line), then exit")
    ap.add_argument("--profile-case", choices=["fp16", "fp16x3", "fp32", "int8", "sigma_clip", "gain", "chan256", "batch"],
                    default=None,
                    help="small case for ncu captures: one subband of the default workload (one raw "
                         "A-6 subband for int8), warm-up plus three pushes; or one post-correlation, gain "
                         "or 256-channel kernel on a few GB; no JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.probe:
        return probe()
    if args.post_case:
        return post_case()

    import torch

    import paper_1609_04205_b300 as acf
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk = peaks()
    w = dict(synth.WORKLOADS["a12"])
    N, n_sb, S = w["n_inputs"], w["n_subbands"], w["n_samples"]
    sky = synth.make_sky(N, w["n_sources"], w["flux"], w["seed"] + rank)
    x = synth.voltages(N, S, n_sb, w["dtype"], w["sigma"], sky, w["seed"] + rank, device=dev)
    in_bytes = x.numel() * x.element_size()
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()

    # ---- headline: FP16 tensor-core mode, whole stage, inputs resident (14.4 GB > L2)
    if world > 1:
        torch.distributed.barrier()
    # the part of each mode's last integration the oracle leg checks (read in
    # place from the accumulator): subband 0, the oracle's channels, every baseline
    keep_a12 = lambda V: V[0, ACC_CHANS].cpu().numpy().astype("complex128")
    clk = Clocks(local)
    main_r = time_mode(acf, torch, x, w, "fp16", args.steps, args.warmup, stream, keep=keep_a12)
    clocks = clk.stop()
    ms, value = aggregate(main_r["ms_per_step"], main_r["ops_per_step"], dev)

    extra = {}
    if not args.quick:
        r3 = time_mode(acf, torch, x, w, "fp16x3", max(2, args.steps // 2), 2, stream, keep=keep_a12)
        extra["fp16x3"] = dict(tops=r3["tops"], xeng_tops=r3["xeng_tops"], ms_per_step=r3["ms_per_step"],
                               issued_tensor_tops=3 * r3["xeng_tops"], xengine_tuning=r3["xengine_tuning"])
        r32 = time_mode(acf, torch, x, w, "fp32", 2, 1, stream, keep=keep_a12)
        fp32_peak = fp32_fma_peak_tflops(torch, pk["sm_max_mhz"])
        extra["fp32_cuda_core"] = dict(tops=r32["tops"], xeng_tops=r32["xeng_tops"], ms_per_step=r32["ms_per_step"],
                                       fp32_fma_peak_tflops=fp32_peak, frac_of_fp32_peak=r32["xeng_tops"] / fp32_peak)
        extra["fp16_speedup_vs_fp32_path"] = main_r["tops"] / r32["tops"]
        extra["fp16x3_speedup_vs_fp32_path"] = r3["tops"] / r32["tops"]
        # INT8-exact raw subbands, AARTFAAC-6 shape
        w6 = dict(synth.WORKLOADS["a6"])
        w6.update(n_channels=1, n_taps=1)
        del x
        torch.cuda.empty_cache()
        x6 = synth.voltages(w6["n_inputs"], w6["n_samples"], w6["n_subbands"], "ci8", w6["sigma"], None, w6["seed"],
                            device=dev)
        nb64 = INT8_ACC_INPUTS * (INT8_ACC_INPUTS + 1) // 2     # baselines among the first 64 inputs
        r8 = time_mode(acf, torch, x6, w6, "int8", max(2, args.steps // 2), 2, stream,
                       keep=lambda out: out[0, 0, :nb64].cpu().numpy())
        x6_sub = x6[0][:, :INT8_ACC_INPUTS].cpu().numpy()
        extra["int8_raw_a6"] = dict(tops=r8["tops"], xeng_tops=r8["xeng_tops"], ms_per_step=r8["ms_per_step"],
                                    xengine_tuning=r8["xengine_tuning"],
                                    frac_of_fp16_sustained=r8["xeng_tops"] / pk["bf16_sus"],
                                    note="exact INT8 runs on the fp16 tensor path (kind::i8 does not assemble "
                                         "for sm_103a), so its peak is the fp16 one",
                                    workload="576 inputs x 8 subbands x 195313 ci8 samples, raw subband, exact")
        del x6
        torch.cuda.empty_cache()
        x = synth.voltages(N, S, n_sb, w["dtype"], w["sigma"], sky, w["seed"] + rank, device=dev)

    # channeliser HBM throughput (algorithmic bytes: ci16 in + fp16 out)
    out_bytes = n_sb * w["n_channels"] * 2 * N * statistics.median(main_r["T"]) * 2
    chan_gbs = (in_bytes + out_bytes) / (main_r["chan_ms"] * 1e-3) / 1e9
    chan_alone = time_channeliser_alone(torch, x, w, pk)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.quick:
        try:
            xh = x.cpu().pin_memory()
            c = acf.Correlator(N, n_sb, w["n_channels"], w["n_taps"], 1, "fp16", w["dtype"], S)
            outh = torch.empty((n_sb, w["n_channels"], N * (N + 1) // 2, 2), dtype=torch.float32).pin_memory()
            with torch.cuda.stream(stream):
                c.push(xh, stream)               # tune on one integration of the live samples
                c.visibilities(outh, stream)
                stream.synchronize()
                c.tune()
                for _ in range(2):
                    c.push(xh, stream)
                    c.visibilities(outh, stream)
                stream.synchronize()
                k = max(2, args.steps // 2)
                t0 = time.perf_counter()
                ops = 0.0
                for _ in range(k):
                    c.push(xh, stream)
                    c.visibilities(outh, stream)
                    ops += xops(N, c.query()["last_spectra"], w["n_channels"], n_sb)
                stream.synchronize()
                dt = time.perf_counter() - t0
            c.close()
            e2e = dict(value=ops / dt / 1e12, unit=UNIT, h2d_bytes_per_step=in_bytes,
                       d2h_bytes_per_step=outh.numel() * 4)
            del xh, outh
        except Exception as ex:  # pinned host memory may be short on some hosts
            e2e = dict(value=None, unit=UNIT, h2d_bytes_per_step=in_bytes, d2h_bytes_per_step=0,
                       note="e2e failed: %s" % ex)

    post_r = batch_r = gain_r = None
    if not args.quick:
        post_r = time_post(acf, torch, pk, N, n_sb, w["n_channels"], oracle_sample=(rank == 0))
        batch_r = time_batch(acf, torch, synth, pk)
        gain_r = time_gain(acf, torch, pk)

    cpu = None
    accuracy = None
    if rank == 0 and not args.quick:
        # the oracle leg: timed on subband 0 of this input (two channels, all
        # inputs); its visibilities are also the reference for each mode's
        # accuracy, and the exact integer oracle sums 64 inputs of the INT8 run
        import numpy as np

        import oracle
        oracle.build()
        x0 = x[0].cpu().numpy()
        cpu, Vref = cpu_oracle_sample(x0, main_r["pushes"])
        cpu.pop("seconds", None)
        ref_of = lambda r: Vref if r["pushes"] == main_r["pushes"] else cpu_oracle_sample(x0, r["pushes"])[1]
        accuracy = dict(
            metric="max |dV_ij| / sqrt(V_ii V_jj) against the fp64 oracle, subband 0, channels %s, all %d inputs "
                   "(every baseline) of each mode's last timed push; INT8: bit-exact int64 on the first %d inputs "
                   "of A-6 subband 0" % (ACC_CHANS, N, INT8_ACC_INPUTS),
            tolerance=dict(fp16=3e-3, fp16x3=1e-5, fp32=1e-5),
            fp16=norm_err(main_r["kept"], Vref, N), fp16x3=norm_err(r3["kept"], ref_of(r3), N),
            fp32=norm_err(r32["kept"], ref_of(r32), N),
            int8_exact=bool(np.array_equal(r8["kept"], oracle.correlate_int(x6_sub))))

    xeng_ms = main_r["xeng_ms"]
    achieved = main_r["xeng_tops"]
    tps = xeng_traffic_per_subband()
    roof = dict(bound="tensor", achieved=achieved, peak=pk["bf16_sus"], unit="TFLOP/s",
                frac=achieved / pk["bf16_sus"], traffic=None if tps is None else tps * n_sb,
                note="X-engine (%s, FP16 operands, fp32 accumulation); algorithmic ops "
                     "8*N(N+1)/2*spectra*channels*subbands = %.3e per launch over its CUDA-event time %.3f ms; "
                     "peak = %s bf16 sustained (fp16 dense = bf16 dense on B300); frac of burst %.3f"
                     % (xeng_desc(main_r["xengine_tuning"]), main_r["ops_per_step"], xeng_ms, pk["src"],
                        achieved / pk["bf16"]))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="fp16",
                data="synthetic",
                config=dict(workload="A-12: 1152 inputs (576 dual-pol antennas) x 16 subbands x 195313 ci16 "
                                     "samples (1 s), 64 ch x 16 taps, FP16 tensor-core X-engine",
                            global_batch=n_sb * world, l2="inputs 14.4 GB > L2 (no flush needed)",
                            step="push one second of samples per subband (channeliser + X-engine), then "
                                 "acf_release_visibilities: the integration stays in HBM (read in place by the "
                                 "accuracy check); e2e copies it to host memory instead",
                            parallelism="independent subband sets per rank" if world > 1 else "single GPU"),
                roofline=roof, clocks=clocks, gpu_launches=main_r["launches"],
                xengine_tuning=main_r["xengine_tuning"],
                channeliser=dict(ms=main_r["chan_ms"], gbs=chan_gbs, frac_hbm=chan_gbs / pk["hbm"],
                                 bytes=in_bytes + out_bytes,
                                 note="inside the step: history head and filter-state copy included, at the step's "
                                      "power-capped clock; `alone` is the same channelisation launched by itself"),
                channeliser_alone=chan_alone,
                e2e=e2e, cpu_baseline=cpu, accuracy=accuracy, modes=extra, post=post_r, ragged_batch=batch_r,
                gain=gain_r)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
