"""Parity of the post-correlation kernels (delay compensation, channel
integration, lost-data weights and re-weighting, sigma-clip flagging)
against the numpy oracle on the same inputs."""
import numpy as np
import pytest
import torch

import oracle
from oracle import post
from helpers import norm_err

pytestmark = pytest.mark.gpu

FS = 195312.5


def _acf():
    import paper_1609_04205_b300 as acf
    return acf


def _rand_vis(rng, n_sb, C, N, scale=1.0):
    NB = N * (N + 1) // 2
    V = (rng.normal(size=(n_sb, C, NB)) + 1j * rng.normal(size=(n_sb, C, NB))) * scale
    return V.astype(np.complex64)


def _to_dev(V):
    return torch.from_numpy(np.stack([V.real, V.imag], -1).astype(np.float32)).cuda()


def _from_dev(t):
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("N,C", [(101, 16), (64, 64), (9, 1)])
def test_delay_compensate_matches_oracle(N, C):
    acf = _acf()
    rng = np.random.default_rng(10 + N)
    V = _rand_vis(rng, 2, C, N)
    d = rng.uniform(-2e-5, 2e-5, N)
    fc = np.array([300 * FS, 301 * FS])
    Vd = _to_dev(V)
    acf.postproc.delay_compensate(Vd, d, fc, FS)
    got = _from_dev(Vd)
    want = post.delay_compensate(V.astype(np.complex128), d, fc, FS)
    # fp32 rotation of fp32 values: a few ulp per element
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-30)) < 2e-6


def test_delay_in_context_matches_oracle():
    """Correlator with acf_set_delays against oracle correlator + compensation."""
    acf = _acf()
    rng = np.random.default_rng(20)
    N, C, P, S = 24, 16, 16, 16 * 16 * 20
    x = rng.integers(-60, 60, size=(1, S, N, 2)).astype(np.int8)
    d = rng.uniform(-3e-6, 3e-6, N)
    fc = [300 * FS]
    c = acf.Correlator(N, 1, C, P, 1, "fp32", "ci8", S)
    c.set_delays(d, fc, FS)
    c.push(torch.from_numpy(x).cuda())
    out = c.empty_visibilities()
    assert c.visibilities(out) is not None
    got = _from_dev(out)[0]
    ref = oracle.correlator(x[0], P, C)[0]
    want = post.delay_compensate(ref[None], d, fc, FS)[0]
    assert norm_err(got, want, N) < 1e-5
    # switching compensation off returns plain visibilities
    c.set_delays(None, None, 0.0)
    c.push(torch.from_numpy(x).cuda())
    assert c.visibilities(out) is not None
    ref2 = oracle.correlator(np.concatenate([x[0], x[0]]), P, C, push_sizes=[S, S])[1]
    assert norm_err(_from_dev(out)[0], ref2, N) < 1e-5
    c.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_delay_in_context_fused_in_tensor_core_flush(variant):
    """Split-FP16 context (tensor-core X-engine, one SM or SM pairs per tile)
    with acf_set_delays: the rotation is applied in the X-engine's flush to
    every push of a two-push integration (linear, so the integrated V is the
    compensated sum); against the oracle correlator + compensation."""
    acf = _acf()
    rng = np.random.default_rng(21 + variant)
    N, C, P, S = 40, 16, 16, 16 * 16 * 12
    x = rng.integers(-60, 60, size=(1, 2 * S, N, 2)).astype(np.int8)
    d = rng.uniform(-3e-6, 3e-6, N)
    fc = [301 * FS]
    c = acf.Correlator(N, 1, C, P, 2, "fp16x3", "ci8", S, variant=variant)
    c.set_delays(d, fc, FS)
    xd = torch.from_numpy(x).cuda()
    c.push(xd[:, :S].contiguous())
    assert c.visibilities() is None
    c.push(xd[:, S:].contiguous())
    out = c.empty_visibilities()
    assert c.visibilities(out) is not None
    got = _from_dev(out)[0]
    ref = oracle.correlator(x[0], P, C, push_sizes=[S, S], n_integrate=2)[0]
    want = post.delay_compensate(ref[None], d, fc, FS)[0]
    assert norm_err(got, want, N) < 1e-5
    c.close()


def test_set_delays_rejected_for_int8():
    acf = _acf()
    c = acf.Correlator(16, 1, 1, 1, 1, "int8", "ci8", 4096)
    with pytest.raises(acf.AcfError):
        c.set_delays(np.zeros(16), [300 * FS], FS)
    c.close()


@pytest.mark.parametrize("N,group", [(101, 4), (64, 2), (33, 16)])
def test_integrate_channels_float(N, group):
    acf = _acf()
    rng = np.random.default_rng(30 + N)
    V = _rand_vis(rng, 3, 16, N)
    got = _from_dev(acf.postproc.integrate_channels(_to_dev(V), group))
    want = post.integrate_channels(V.astype(np.complex128), group)
    assert np.max(np.abs(got - want)) < 1e-5 * group


@pytest.mark.parametrize("N", [101, 64])
def test_integrate_channels_int64_exact(N):
    acf = _acf()
    rng = np.random.default_rng(40 + N)
    NB = N * (N + 1) // 2
    V = rng.integers(-2**50, 2**50, size=(2, 16, NB, 2), dtype=np.int64)
    got = acf.postproc.integrate_channels(torch.from_numpy(V).cuda(), 8).cpu().numpy()
    assert np.array_equal(got, post.integrate_channels(V, 8))


def test_integrate_channels_rejects_bad_group():
    acf = _acf()
    V = torch.zeros((1, 16, 10, 2), dtype=torch.float32, device="cuda")
    for g in (3, 5, 0):
        with pytest.raises((acf.AcfError, ZeroDivisionError)):
            acf.postproc.integrate_channels(V, g)
    assert acf.postproc.integrate_channels(V, 16).shape == (1, 1, 10, 2)


@pytest.mark.parametrize("n_blocks,N", [(1000, 100), (33, 7), (64, 1)])
def test_lost_sample_weights_exact(n_blocks, N):
    acf = _acf()
    rng = np.random.default_rng(50 + N)
    m = (rng.uniform(size=(n_blocks, N)) < 0.9).astype(np.uint8) * rng.integers(1, 255, size=(n_blocks, N)).astype(np.uint8)
    got = acf.postproc.lost_sample_weights(torch.from_numpy(m).cuda(), 16).cpu().numpy()
    assert np.array_equal(got, post.lost_sample_weights(m != 0, 16))


def test_lost_sample_weights_full_size_sampled():
    """A-12 sized: 1152 inputs, one second of 16-sample packets; every
    autocorrelation and a random sample of pairs checked exactly."""
    acf = _acf()
    rng = np.random.default_rng(60)
    nb, N = 195313 // 16 + 1, 1152
    m = (rng.uniform(size=(nb, N)) < 0.97).astype(np.uint8)
    W = acf.postproc.lost_sample_weights(torch.from_numpy(m).cuda(), 16).cpu().numpy()
    i, j = post.pairs(N)
    mi = m.astype(np.int64)
    assert np.array_equal(W[i == j], 16 * mi.sum(axis=0))
    for b in rng.integers(0, W.size, 300):
        assert W[b] == 16 * int(np.dot(mi[:, i[b]], mi[:, j[b]]))


def test_reweight_matches_oracle():
    acf = _acf()
    rng = np.random.default_rng(70)
    N, C = 50, 4
    V = _rand_vis(rng, 1, C, N)
    m = (rng.uniform(size=(200, N)) < 0.8).astype(np.uint8)
    m[:, 3] = 0                                   # a dead input: W = 0 on its row and column
    Wd = acf.postproc.lost_sample_weights(torch.from_numpy(m).cuda(), 4)
    Vd = _to_dev(V)
    acf.postproc.reweight(Vd, Wd, 800)
    got = _from_dev(Vd)
    want = post.reweight(V.astype(np.complex128), post.lost_sample_weights(m, 4), 800)
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-30)) < 1e-6
    i, j = post.pairs(N)
    assert np.all(got[..., (i == 3) | (j == 3)] == 0)


def _flag_case(seed, N, C, n_sb=2):
    rng = np.random.default_rng(seed)
    V = _rand_vis(rng, n_sb, C, N)
    i, j = post.pairs(N)
    cross = np.nonzero(i != j)[0]
    for s in range(n_sb):                          # planted stage-1 and stage-2 outliers
        V[s, 3, cross[7]] *= 40.0
        V[s, 5, cross[11]] *= 3.5
        V[s, 0, np.nonzero(i == j)[0][2]] *= 1e4   # a huge autocorrelation, never flagged
    return V


@pytest.mark.parametrize("N,C,k1,k2", [(40, 16, 5.0, 3.0), (101, 8, 3.0, 2.5), (64, 64, 4.0, 2.0),
                                       (20, 256, 4.0, 2.5), (33, 100, 3.5, 2.5)])
def test_sigma_clip_matches_oracle(N, C, k1, k2):
    acf = _acf()
    V = _flag_case(80 + N, N, C)
    got = acf.postproc.sigma_clip(_to_dev(V), k1, k2).cpu().numpy()
    V64 = V.astype(np.complex128)                  # the same fp32 values, widened exactly
    want = post.sigma_clip(V64, k1, k2)
    # both sides decide in fp64 on the same fp32 values; only a value within
    # rounding of its threshold could differ, which random data does not hit
    assert np.array_equal(got, want)
    assert got.sum() > 0
    i, j = post.pairs(N)
    assert not got[..., i == j].any()


@pytest.mark.parametrize("N,C", [(24, 16), (25, 80)])
def test_sigma_clip_threshold_ties_settled_in_fp64(N, C):
    """Every |V|^2 equal to its threshold, or within the fp32 guard band of
    it: with k1 = k2 = 1 and a constant V = 0.75 + 1j (|V|^2 = 1.5625, exact
    in fp32 and fp64) each channel mean equals every element, so every test
    is a tie that only the fp64 comparison (a > a is false) settles.  One
    element is raised by 2^-22 in its real part (relative change ~2^-22, well
    inside the band); a second, large element in the same channel lifts that
    channel's stage-1 threshold clear of it, so stage 2 must flag it through
    the fp64 path.  Odd NB (N = 25) takes the scalar sums path."""
    acf = _acf()
    i, j = post.pairs(N)
    cross = np.nonzero(i != j)[0]
    V = np.full((1, C, i.size), 0.75 + 1.0j, dtype=np.complex64)
    x, y = cross[5], cross[9]
    V[0, 4, x] = np.float32(0.75 + 2.0 ** -22) + 1.0j
    V[0, 4, y] = 30.0 + 40.0j
    got = acf.postproc.sigma_clip(_to_dev(V), 1.0, 1.0).cpu().numpy()
    want = post.sigma_clip(V.astype(np.complex128), 1.0, 1.0)
    assert np.array_equal(got, want)
    expect = np.zeros_like(want)
    expect[0, 4, x] = expect[0, 4, y] = 1
    assert np.array_equal(got, expect)


def test_sigma_clip_rejects_bad_threshold():
    acf = _acf()
    V = torch.zeros((1, 4, 10, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(acf.AcfError):
        acf.postproc.sigma_clip(V, 0.0, 1.0)
