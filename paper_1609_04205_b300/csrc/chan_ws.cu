// Warp-specialised polyphase channeliser for the production geometry: 16
// taps, 64 channels, complex int16 or int8 input (Sec. 4.2.3 FIR + FFT,
// Sec. 4.2.4 bandpass + transpose into the X-engine operand layout).
//
// A persistent CTA (one per SM) walks a list of items; an item is NI
// consecutive inputs (one 16-byte row of samples: 4 ci16 or 8 ci8) of one
// subband over a segment of spectra.  Three roles share the CTA:
//   * producer (FIR thread 0): TMA copies of [1024 time rows][NI inputs]
//     tiles into a ring of shared-memory stages, one stage per batch of 16
//     spectra (rows (m0 + 15) * 64 .. (m0 + 31) * 64: the newest sample of
//     every phase of every spectrum in the batch) plus one prologue stage per
//     item (the first 15 window rows);
//   * 8 FIR warps: thread (input pair or input, phase n) keeps its 16 taps
//     and the newest 16 samples of its phase in registers, so every input
//     sample is read from shared memory once and costs 16 packed fp32x2 FMAs
//     (Sec. 4.2.3's FIR held in registers); the FIR outputs y_m[n] of a batch
//     go to one of two Y buffers;
//   * 4 FFT warps, two groups of two, one group per Y buffer: thread
//     (input, spectrum) reads its 64 FIR outputs and computes the whole
//     64-point DFT in registers as radix 8 x 8 with compile-time twiddles, no
//     shared-memory pass between the radix stages; then the bandpass weight
//     times the output scale (Sec. 4.2.4), the conversion, and the store:
//     lanes hold consecutive spectra, so neighbouring lanes swap one word and
//     each writes a time-contiguous pair of one output row (the transpose of
//     Sec. 4.2.4 done in registers).
// The FIR warps and the FFT groups hand batches over through mbarriers; every
// wait is bounded (about one second of SM clock), after which the CTA sets the
// device error word, stops, and lets its TMA copies land before exiting.
// Spectra whose windows reach into the filter history (the first
// ceil(n_hist / 64), rounded up to 16, of a push) are left to the generic
// kernel: this one reads only the pushed samples, through one tensor map.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "acf_internal.h"
#include "tc_ptx.cuh"

namespace acf {
namespace {

constexpr int kC = 64;                  // channels
constexpr int kP = 16;                  // taps
constexpr int kMB = 16;                 // spectra per batch (== taps: window slots stay static)
constexpr int kFirWarps = 8;
constexpr int kFftWarps = 4;            // two groups of two
constexpr int kThreadsWs = 32 * (kFirWarps + kFftWarps);
constexpr int kFirThreads = 32 * kFirWarps;
constexpr int kFftGroup = 64;           // threads per FFT group
constexpr int kRowsPerStage = kMB * kC; // 1024 time rows, 16 bytes each
constexpr int kStageBytes = kRowsPerStage * 16;
constexpr int kBoxRows = 256;
constexpr int kYRow = kC * 8 + 16;      // one spectrum of one input: 64 complex + 16 B
constexpr long long kWaitCyclesWs = 1LL << 31;   // about one second of SM clock

template <typename IN>
struct WsGeo {
    static constexpr int E = sizeof(IN);           // bytes per complex sample
    static constexpr int NI = 16 / E;              // inputs per item (one 16-byte row)
    static constexpr int IPT = NI / 4;             // inputs per FIR thread
    // four 16 KB stages: six (more input in flight) measured 7% slower --
    // the scattered 16-byte input reads then crowd the output stores
    static constexpr int STAGES = 4;
    // Y buffer: [NI][kMB spectra][kYRow]; the per-input stride keeps the FIR
    // stores (lanes = 4 input slots x 8 phases) conflict-free, the 528-byte
    // spectrum stride keeps the FFT's 16-byte reads (lanes = spectra) so.
    static constexpr int SI = kMB * kYRow + 32 / IPT;
    static constexpr int YBUF = NI * SI;
    static constexpr int OFF_Y = STAGES * kStageBytes;
    static constexpr int OFF_W = OFF_Y + 2 * YBUF;              // bandpass x scale, [k1][k2]
    static constexpr int OFF_BAR = OFF_W + kC * 4;
    static constexpr int NBAR = 2 * STAGES + 4;
    static constexpr size_t SMEM = OFF_BAR + 8 * NBAR + 128;   // + alignment slack
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct WsParams {
    CUtensorMap map;      // input [n_sb][n_samples][N] samples; boxes of NI inputs x 256 rows
    const float *h;       // taps, h[k * 64 + n]
    const float *bp;      // bandpass weights, 64
    float osc;            // output scale (fp16 outputs) or 1
    void *out, *out_lo;
    long t_stride;
    long row0;            // input row of stream row 0 (= -n_hist)
    long m_begin, m_end;  // spectra handled, multiples of 16
    long T;               // valid spectra: [T, m_end) are written as zeros
    long seg;             // spectra per item, a multiple of 16
    int groups, n_sb, n_items, N;
    int *err;
    const void *hist;     // tensor-core variant: [n_sb][n_hist][N] samples before the push (n_hist < 1024)
    long n_hist;
};

// ---- small PTX helpers --------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(uint32_t b, uint32_t parity) {
    uint32_t ok;
    // the suspend-time hint (ns) lets a waiting warp sleep in hardware until
    // the phase completes instead of spinning on issue slots the other role
    // needs (4% faster)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(b), "r"(parity), "r"(20000) : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity`: false after the CTA aborted or
// about one second without progress (then it records `code` and aborts).
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, volatile int *abort_flag, int *err, int code) {
    if (bar_test(b, parity)) return true;
    const long long t0 = clock64();
    for (int it = 1;; ++it) {
        if (bar_test(b, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitCyclesWs) {
                *abort_flag = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z) : "memory");
}
// Shared-memory data accesses are plain C++ (the compiler schedules them
// freely between the barrier waits, whose asm carries a memory clobber).
__device__ __forceinline__ uint32_t lds32(const unsigned char *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ float4 lds128(const unsigned char *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts64(unsigned char *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

// ---- complex arithmetic on packed fp32x2 ------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }   // * (-i)

// cos and sin of 2 pi k / n by Taylor series in double, evaluated by the
// compiler (the twiddles below are compile-time constants).
__host__ __device__ constexpr double taylor_cos(double x) {
    double t = 1.0, s = 1.0;
    for (int i = 1; i < 30; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double taylor_sin(double x) {
    double t = x, s = x;
    for (int i = 1; i < 30; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}
constexpr double kTwoPi = 6.283185307179586476925286766559;

// a * W_64^K with W_64 = exp(-2 pi i / 64).
template <int K>
__device__ __forceinline__ float2 mul_w64(float2 a) {
    constexpr int k = K & 63;
    if constexpr (k == 0) {
        return a;
    } else if constexpr (k == 16) {
        return make_float2(a.y, -a.x);
    } else if constexpr (k == 32) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (k == 48) {
        return make_float2(-a.y, a.x);
    } else {
        constexpr float c = (float)taylor_cos(kTwoPi * k / 64.0);
        constexpr float s = (float)taylor_sin(kTwoPi * k / 64.0);
        // (x + i y)(c - i s) = (x c + y s) + i (y c - x s)
        return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -(a.x * s)));
    }
}

// 8-point DFT in place, natural order: A[k] = sum_r a[r] exp(-2 pi i r k / 8)
// (radix-2 decimation in frequency, outputs placed back in natural order).
__device__ __forceinline__ void dft8(float2 (&a)[8]) {
    constexpr float r2 = 0.70710678118654752440f;
    const float2 b0 = cadd(a[0], a[4]), b1 = cadd(a[1], a[5]), b2 = cadd(a[2], a[6]), b3 = cadd(a[3], a[7]);
    const float2 d0 = csub(a[0], a[4]);
    float2 d1 = csub(a[1], a[5]);
    const float2 d2 = mul_mi(csub(a[2], a[6]));
    float2 d3 = csub(a[3], a[7]);
    d1 = make_float2(r2 * (d1.x + d1.y), r2 * (d1.y - d1.x));      // * W_8^1
    d3 = make_float2(r2 * (d3.y - d3.x), -r2 * (d3.x + d3.y));     // * W_8^3
    const float2 e0 = cadd(b0, b2), e1 = cadd(b1, b3), e2 = csub(b0, b2), e3 = mul_mi(csub(b1, b3));
    const float2 f0 = cadd(d0, d2), f1 = cadd(d1, d3), f2 = csub(d0, d2), f3 = mul_mi(csub(d1, d3));
    a[0] = cadd(e0, e1);
    a[4] = csub(e0, e1);
    a[2] = cadd(e2, e3);
    a[6] = csub(e2, e3);
    a[1] = cadd(f0, f1);
    a[5] = csub(f0, f1);
    a[3] = cadd(f2, f3);
    a[7] = csub(f2, f3);
}

// Radix-8 pass 1 on column S (points S + 8 r): 8-point DFT over r, then the
// twiddle W_64^(S k1); results back in place (slot S + 8 k1).
template <int S>
__device__ __forceinline__ void pass1(float2 (&z)[64]) {
    float2 a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = z[S + 8 * r];
    dft8(a);
    z[S] = a[0];
    z[S + 8] = mul_w64<S * 1>(a[1]);
    z[S + 16] = mul_w64<S * 2>(a[2]);
    z[S + 24] = mul_w64<S * 3>(a[3]);
    z[S + 32] = mul_w64<S * 4>(a[4]);
    z[S + 40] = mul_w64<S * 5>(a[5]);
    z[S + 48] = mul_w64<S * 6>(a[6]);
    z[S + 56] = mul_w64<S * 7>(a[7]);
}

template <typename IN, int IPT>
__device__ __forceinline__ void unpack(uint32_t w, float2 (&x)[IPT]);
template <>
__device__ __forceinline__ void unpack<short2, 1>(uint32_t w, float2 (&x)[1]) {
    x[0] = make_float2((float)(short)(w & 0xffffu), (float)(short)(w >> 16));
}
template <>
__device__ __forceinline__ void unpack<char2, 2>(uint32_t w, float2 (&x)[2]) {
    x[0] = make_float2((float)(signed char)(w & 0xffu), (float)(signed char)((w >> 8) & 0xffu));
    x[1] = make_float2((float)(signed char)((w >> 16) & 0xffu), (float)(signed char)(w >> 24));
}

// FIR of one batch: 16 outputs per (input, phase); spectra at or past T
// (MASK) are written as zeros so their DFT is exactly zero.
template <typename IN, int IPT, bool MASK>
__device__ __forceinline__ void fir_batch(const float2 (&hr)[kP], float2 (&win)[IPT][kP], const unsigned char *xs,
                                          unsigned char *ys, int ip, int n, long m0, long T)
{
    using G = WsGeo<IN>;
#pragma unroll
    for (int mm = 0; mm < kMB; ++mm) {
        float2 xv[IPT];
        unpack<IN, IPT>(lds32(xs + (mm * kC + n) * 16 + ip * 4), xv);
#pragma unroll
        for (int u = 0; u < IPT; ++u) {
            win[u][(mm + kP - 1) % kP] = xv[u];
            float2 acc = __fmul2_rn(hr[0], win[u][mm % kP]);
#pragma unroll
            for (int k = 1; k < kP; ++k) acc = __ffma2_rn(hr[k], win[u][(mm + k) % kP], acc);
            if (MASK && m0 + mm >= T) acc = make_float2(0.f, 0.f);
            sts64(ys + (ip * IPT + u) * G::SI + mm * kYRow + n * 8, acc);
        }
    }
}

// Store one channel value of this lane's spectrum: neighbouring lanes hold
// spectra m (even) and m + 1 (odd); the even lane writes the real row's pair,
// the odd lane the imaginary row's pair, at column m.
template <int OUTK>
__device__ __forceinline__ void put(float2 v, float w, bool odd, uint32_t sel, void *out, void *out_lo, long off,
                                    bool ok)
{
    const float re = v.x * w, im = v.y * w;
    if constexpr (OUTK == OUT_F32) {
        const float recv = __shfl_xor_sync(0xffffffffu, odd ? re : im, 1);
        const float2 o = odd ? make_float2(recv, im) : make_float2(re, recv);
        if (ok) *reinterpret_cast<float2 *>(static_cast<float *>(out) + off) = o;
    } else {
        const __half2 hv = __floats2half2_rn(re, im);
        uint32_t hb;
        memcpy(&hb, &hv, 4);
        const uint32_t pb = __shfl_xor_sync(0xffffffffu, hb, 1);
        if (ok) *reinterpret_cast<uint32_t *>(static_cast<__half *>(out) + off) = __byte_perm(hb, pb, sel);
        if constexpr (OUTK == OUT_F16X3) {
            const float2 f = __half22float2(hv);
            const __half2 lv = __floats2half2_rn(re - f.x, im - f.y);
            uint32_t lb;
            memcpy(&lb, &lv, 4);
            const uint32_t pl = __shfl_xor_sync(0xffffffffu, lb, 1);
            if (ok) *reinterpret_cast<uint32_t *>(static_cast<__half *>(out_lo) + off) = __byte_perm(lb, pl, sel);
        }
    }
}

struct ItemPos {
    int sb, grp;
    long m_lo, m_hi;
};
__device__ __forceinline__ ItemPos decode_item(const WsParams &P, int item) {
    ItemPos d;
    const int seg = item / (P.n_sb * P.groups);
    const int rem = item - seg * (P.n_sb * P.groups);
    d.sb = rem / P.groups;
    d.grp = rem - d.sb * P.groups;
    d.m_lo = P.m_begin + (long)seg * P.seg;
    d.m_hi = min(P.m_end, d.m_lo + P.seg);
    return d;
}

template <typename IN, int OUTK>
__global__ void __launch_bounds__(kThreadsWs, 1) k_ppf64_ws(const __grid_constant__ WsParams P)
{
    using G = WsGeo<IN>;
    constexpr int NI = G::NI, IPT = G::IPT, NS = G::STAGES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ int abort_flag;
    const uint32_t s0 = su32(smem);
    const uint32_t bar0 = s0 + G::OFF_BAR;
    auto xfull = [&](int s) { return bar0 + 8u * s; };
    auto xempty = [&](int s) { return bar0 + 8u * (NS + s); };
    auto yfull = [&](int b) { return bar0 + 8u * (2 * NS + b); };
    auto yempty = [&](int b) { return bar0 + 8u * (2 * NS + 2 + b); };
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            bar_init(xfull(s), 1);
            bar_init(xempty(s), kFirThreads);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(yfull(b), kFirThreads);
            bar_init(yempty(b), kFftGroup);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.map)) : "memory");
    }
    if (tid >= kFirThreads && tid < kFirThreads + kC) {
        // bandpass x scale, stored [k1][k2] for channel c = k1 + 8 k2
        const int c = tid - kFirThreads;
        reinterpret_cast<float *>(smem + G::OFF_W)[(c & 7) * 8 + (c >> 3)] = __ldg(P.bp + c) * P.osc;
    }
    __syncthreads();

    if (warp < kFirWarps) {
        // ---------------- FIR warps (thread 0 also produces) ----------------
        const int fi = tid, ip = fi & 3, n = fi >> 2;
        float2 hr[kP];
#pragma unroll
        for (int k = 0; k < kP; ++k) {
            const float hv = __ldg(P.h + k * kC + n);
            hr[k] = make_float2(hv, hv);
        }
        float2 win[IPT][kP];
#pragma unroll
        for (int u = 0; u < IPT; ++u)
#pragma unroll
            for (int k = 0; k < kP; ++k) win[u][k] = make_float2(0.f, 0.f);
        // producer state (thread 0): the next load to issue
        long issued = 0;
        int p_item = blockIdx.x, p_j = 0;
        ItemPos pd = decode_item(P, p_item < P.n_items ? p_item : 0);
        bool p_done = p_item >= P.n_items;
        auto produce = [&](long upto) -> bool {   // issue loads [issued, upto)
            while (!p_done && issued < upto) {
                const int s = (int)(issued % NS);
                if (issued >= NS && !bar_wait(xempty(s), (uint32_t)(((issued / NS) - 1) & 1), &abort_flag, P.err, 21))
                    return false;
                const long srow = p_j == 0 ? pd.m_lo * kC : (pd.m_lo + (long)kMB * (p_j - 1) + (kP - 1)) * kC;
                const long y = srow + P.row0;
                bar_expect(xfull(s), kStageBytes);
#pragma unroll
                for (int q = 0; q < kRowsPerStage / kBoxRows; ++q)
                    tma_3d(s0 + s * kStageBytes + q * kBoxRows * 16, &P.map, xfull(s), pd.grp * NI,
                           (int)(y + q * kBoxRows), pd.sb);
                ++issued;
                const long nb = (pd.m_hi - pd.m_lo) / kMB;
                if (++p_j > nb) {
                    p_j = 0;
                    p_item += gridDim.x;
                    if (p_item >= P.n_items) p_done = true;
                    else pd = decode_item(P, p_item);
                }
            }
            return true;
        };
        long L = 0, gbat = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
            const ItemPos d = decode_item(P, item);
            // prologue: window rows 0 .. 14 of the item's first spectrum
            if (fi == 0) ok = produce(L + NS);
            if (ok) ok = bar_wait(xfull((int)(L % NS)), (uint32_t)((L / NS) & 1), &abort_flag, P.err, 22);
            if (!ok) break;
            {
                const unsigned char *xs = smem + (L % NS) * kStageBytes;
#pragma unroll
                for (int k = 0; k < kP - 1; ++k) {
                    float2 xv[IPT];
                    unpack<IN, IPT>(lds32(xs + (k * kC + n) * 16 + ip * 4), xv);
#pragma unroll
                    for (int u = 0; u < IPT; ++u) win[u][k] = xv[u];
                }
                bar_arrive(xempty((int)(L % NS)));
                ++L;
            }
            for (long m0 = d.m_lo; m0 < d.m_hi; m0 += kMB, ++gbat) {
                if (fi == 0) ok = produce(L + NS);
                const int yb = (int)(gbat & 1);
                if (ok && gbat >= 2)
                    ok = bar_wait(yempty(yb), (uint32_t)(((gbat >> 1) - 1) & 1), &abort_flag, P.err, 23);
                if (ok) ok = bar_wait(xfull((int)(L % NS)), (uint32_t)((L / NS) & 1), &abort_flag, P.err, 24);
                if (!ok) break;
                const unsigned char *xs = smem + (L % NS) * kStageBytes;
                unsigned char *ys = smem + G::OFF_Y + yb * G::YBUF;
                if (m0 + kMB <= P.T) fir_batch<IN, IPT, false>(hr, win, xs, ys, ip, n, m0, P.T);
                else fir_batch<IN, IPT, true>(hr, win, xs, ys, ip, n, m0, P.T);
                bar_arrive(xempty((int)(L % NS)));
                bar_arrive(yfull(yb));
                ++L;
            }
        }
        if (fi == 0) {
            // let every copy this CTA issued land before it exits (all were
            // consumed unless the CTA aborted)
            for (long q = issued - 1; q >= 0 && q >= issued - NS; --q) {
                const int s = (int)(q % NS);
                for (long long it = 0; it < (1LL << 22) && !bar_test(xfull(s), (uint32_t)((q / NS) & 1)); ++it)
                    __nanosleep(256);
            }
        }
    } else {
        // ---------------- FFT warps ----------------
        const int ft = tid - kFirThreads, g = ft >> 6, tt = ft & 63;
        const bool odd = (tt & 1) != 0;
        const uint32_t sel = odd ? 0x3276u : 0x5410u;
        const unsigned char *wsm = smem + G::OFF_W;
        const long cstride = 2L * P.N * P.t_stride;          // elements between channels
        long gbat = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
            const ItemPos d = decode_item(P, item);
            for (long m0 = d.m_lo; m0 < d.m_hi; m0 += kMB, ++gbat) {
                if ((int)(gbat & 1) != g) continue;
                ok = bar_wait(yfull(g), (uint32_t)((gbat >> 1) & 1), &abort_flag, P.err, 25);
                if (!ok) break;
                const unsigned char *ys = smem + G::OFF_Y + g * G::YBUF;
#pragma unroll 1
                for (int q = 0; q < IPT; ++q) {
                    const int job = tt + kFftGroup * q;
                    const int i = job >> 4, mm = job & 15;
                    float2 z[64];
                    const unsigned char *yr = ys + i * G::SI + mm * kYRow;
#pragma unroll
                    for (int p = 0; p < 32; ++p) {
                        const float4 v = lds128(yr + 16 * p);
                        z[2 * p] = make_float2(v.x, v.y);
                        z[2 * p + 1] = make_float2(v.z, v.w);
                    }
                    if (q == IPT - 1) bar_arrive(yempty(g));
                    pass1<0>(z); pass1<1>(z); pass1<2>(z); pass1<3>(z);
                    pass1<4>(z); pass1<5>(z); pass1<6>(z); pass1<7>(z);
                    const int nn = d.grp * NI + i;
                    const bool st = nn < P.N;
                    const long off = ((long)d.sb * kC * 2 * P.N + 2L * nn + (odd ? 1 : 0)) * P.t_stride + m0 + (mm & ~1);
#pragma unroll
                    for (int k1 = 0; k1 < 8; ++k1) {
                        float2 a[8];
#pragma unroll
                        for (int s = 0; s < 8; ++s) a[s] = z[s + 8 * k1];
                        dft8(a);
                        const float4 w0 = lds128(wsm + 32 * k1), w1 = lds128(wsm + 32 * k1 + 16);
                        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                        for (int k2 = 0; k2 < 8; ++k2)
                            put<OUTK>(a[k2], wv[k2], odd, sel, P.out, P.out_lo, off + (long)(k1 + 8 * k2) * cstride, st);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core variant for fp16 and split-fp16 output.  The 64-point DFT of one (input,
// spectrum) is a product with the 64 x 64 complex DFT matrix.  In real form a
// batch (eight inputs x 16 spectra) is one tcgen05.mma of M = 128, N = 128,
// K = 128 (eight K = 16 steps), fp16 operands, fp32 accumulation in TMEM:
//     D[r][2c + o] = sum_k Y[r][k] W[2c + o][k],
// Y row r = one (input, spectrum) of FIR outputs, column k = 2n + [imag part];
// W row 2c + o = channel c's real (o = 0) or imaginary (o = 1) part.  With
// W_64^(nc) = wr + i wi: Re z = sum wr yr - wi yi, Im z = sum wi yr + wr yi.
// The bandpass weight times the output scale is applied in fp32 by the
// epilogue, before the fp16 rounding.  The epilogue reads TMEM in the
// 16-lane x 256-bit shape, which hands each thread two lanes eight apart;
// the Y row map puts spectra mm and mm + 1 of one input there, so a thread
// packs a time-contiguous pair of one output row directly, and each warp
// store writes four whole 32-byte runs of output rows (the transpose of
// Sec. 4.2.4).  Four accumulators (all 512 TMEM columns) let the epilogue
// drain the batches of one 64-spectrum window together: the four 32-byte
// pieces of an output row's 128-byte line leave in consecutive stores, which
// DRAM takes at 5.4 TB/s against 3.5 TB/s for pieces a batch apart.
// The FIR is written in transposed form: every new sample of a phase adds its
// 16 tap products into a ring of 16 open spectra (independent FMAs), and the
// spectrum that received its last tap leaves the ring.  Each spectrum still
// sums h[0] x[s] + h[1] x[s+1] + ... in tap order, so its value equals the
// direct form's.
// Split-fp16 output (SPLIT: the hi and lo operand planes of the FP16x3 mode,
// Sec. 4.2.5) keeps about fp32 accuracy through the transform: the FIR
// outputs and the DFT matrix are each split into fp16 hi and lo parts, and
// three MMAs per K step sum Yl Wh, Yh Wl and then Yh Wh into the fp32
// accumulator (the small products first, so the accumulator's truncating
// adds act on small partial sums; Yl Wl, about 2^-22 of the result, is
// dropped).  The epilogue splits the scaled result into the hi and lo
// planes.  The taps are scaled by 64 (exact) so that the lo parts of small
// int8 samples stay clear of fp16's subnormal range; the bandpass weight
// carries the 1/64.  The doubled operands leave int16 input one FIR operand
// buffer (the FIR writes a batch once the MMAs have read the previous one)
// and three input stages, int8 two of each.  A form with both DFT matrices
// in tensor memory (the MMA's A operand) was slower and not deterministic.
// Roles: warp 0 lane 0 TMA producer (input ring as in k_ppf64_ws, items of
// eight inputs), warp 1 TMEM owner and MMA issuer, warps 2-5 epilogue (TMEM
// lane quadrant = warp % 4), warps 6-13 FIR (thread = phase n, input pair).
constexpr int kTcNI = 8;                 // inputs per item
constexpr int kTcThreads = 448;
constexpr int kTcFir0 = 6;               // first FIR warp
constexpr int kTcEpiThreads = 128;
constexpr uint32_t kTcCols = 512;        // four 128-column fp32 accumulators
constexpr int kTcAcc = 4;
constexpr uint32_t kTcIdesc = tc::idesc_f16_kmajor(128, 128);

constexpr float kTcTapScale = 64.f;      // split output: tap scale, undone in the epilogue

// SPLIT (split-fp16 output): the DFT matrix and the FIR operand each have hi
// and lo halves (32 KB apiece).  ci16 then keeps one FIR operand buffer and
// three input stages, ci8 two buffers and two stages.
template <typename IN, bool SPLIT = false>
struct TcGeo {
    static constexpr int E = sizeof(IN);
    static constexpr int ROWB = kTcNI * E;                 // stage row: 32 B (ci16) or 16 B (ci8)
    static constexpr int STAGE = kRowsPerStage * ROWB;
    static constexpr int STAGES = !SPLIT ? 4 : (E == 4 ? 3 : 2);
    static constexpr int NYB = !SPLIT || E != 4 ? 2 : 1;   // FIR operand buffers
    static constexpr int WB = SPLIT ? 65536 : 32768;       // DFT matrix: hi, then lo 32 KB on (split)
    static constexpr int YB = SPLIT ? 65536 : 32768;       // one FIR operand buffer: hi, then lo
    static constexpr int OFF_W = 0;                        // DFT matrix, 2 x [128 rows][128 B] SW128
    static constexpr int OFF_Y = WB;                       // FIR-output operands
    static constexpr int OFF_X = OFF_Y + NYB * YB;         // input ring
    static constexpr int OFF_BAR = OFF_X + STAGES * STAGE;
    static constexpr int NBAR = 2 * STAGES + 4 + 2 * kTcAcc + 1;
    static constexpr size_t SMEM = OFF_BAR + 8 * NBAR + 1024;   // + alignment slack
    static_assert(SMEM + 1040 <= 227 * 1024, "shared memory (dynamic + the kernel's static arrays)");
};

__device__ __forceinline__ void unpack_pair(const unsigned char *p, float2 (&x)[2], short2) {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    x[0] = make_float2((float)(short)(w.x & 0xffffu), (float)(short)(w.x >> 16));
    x[1] = make_float2((float)(short)(w.y & 0xffffu), (float)(short)(w.y >> 16));
}
__device__ __forceinline__ void unpack_pair(const unsigned char *p, float2 (&x)[2], char2) {
    unpack<char2, 2>(lds32(p), x);
}

// Y row of input 2 ip + u, batch spectrum mm:
//     r = 32 ip + 16 u + 8 (mm & 1) + ((mm >> 1) ^ 2 ip).
// TMEM lanes 32 ip + 16 u .. + 15 hold input 2 ip + u; spectra 2x and 2x + 1
// sit in lanes x ^ 2 ip and x ^ 2 ip + 8 of that group.  The rows one FIR
// store instruction writes (four ip, fixed mm and u) differ in (r & 7) >> 1,
// so under the 128-byte swizzle their 32-byte pieces use distinct banks.
// yx[x]: this thread's byte offset in Y for mm >> 1 = x (K atom, row part
// 32 ip + (x ^ 2 ip), swizzled chunk, position in the chunk); 128 (16u + 8
// (mm & 1)) is added per store.
// This thread's input pair at one stream row of the history (global memory).
__device__ __forceinline__ void hist_pair(const void *h, long e, float2 (&x)[2], short2) {
    unpack_pair(static_cast<const unsigned char *>(h) + e * 4, x, short2{});
}
__device__ __forceinline__ void hist_pair(const void *h, long e, float2 (&x)[2], char2) {
    unpack<char2, 2>(*reinterpret_cast<const uint32_t *>(static_cast<const unsigned char *>(h) + e * 2), x);
}

// h0 >= 0: the batch's first sample lies in the history, at element h0.
template <typename IN, bool MASK, bool SPLIT>
__device__ __forceinline__ void fir_batch_tc(const float2 (&hr)[kP], float2 (&acc)[2][kP], const unsigned char *xs,
                                             unsigned char *yb, int xoff, const int (&yx)[8], long m0, long T,
                                             const void *hist, long h0)
{
    using G = TcGeo<IN>;
    // samples are read and widened two steps ahead of their FMAs
    float2 xa[2], xb[2];
    if (h0 >= 0) hist_pair(hist, h0, xa, IN{});
    else unpack_pair(xs + xoff, xa, IN{});
    unpack_pair(xs + kC * G::ROWB + xoff, xb, IN{});
#pragma unroll
    for (int mm = 0; mm < kMB; ++mm) {
        const float2 xv[2] = {xa[0], xa[1]};
        xa[0] = xb[0];
        xa[1] = xb[1];
        if (mm + 2 < kMB) unpack_pair(xs + (mm + 2) * kC * G::ROWB + xoff, xb, IN{});
        // this sample is tap k of spectrum m0 + mm + 15 - k, whose ring slot is (mm + 15 - k) & 15
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            acc[u][(mm + 15) & 15] = __fmul2_rn(hr[0], xv[u]);
#pragma unroll
            for (int k = 1; k < kP; ++k) acc[u][(mm + 15 - k) & 15] = __ffma2_rn(hr[k], xv[u], acc[u][(mm + 15 - k) & 15]);
        }
        // spectrum m0 + mm received its last tap
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float2 y = acc[u][mm & 15];
            if (MASK && m0 + mm >= T) y = make_float2(0.f, 0.f);
            const int off = 128 * (16 * u + 8 * (mm & 1)) + yx[mm >> 1];
            const __half2 hv = __floats2half2_rn(y.x, y.y);
            *reinterpret_cast<__half2 *>(yb + off) = hv;
            if constexpr (SPLIT) {
                const float2 hf = __half22float2(hv);
                *reinterpret_cast<__half2 *>(yb + 32768 + off) = __floats2half2_rn(y.x - hf.x, y.y - hf.y);
            }
        }
    }
}

// Drain NB consecutive batches (accumulators g .. g + NB - 1, mod 4) of one
// epilogue thread: for each input half u and each pair of its channels, load
// the NB batches' values, scale by the channel's weight, round to fp16 and
// store the (mm, mm + 1) pairs of the real and imaginary rows; the NB stores
// of one row go out back to back (16 NB spectra of the row).  o: real row of
// (channel t4, input 2q) at the window's first spectrum + mm.
template <int NB, bool SPLIT>
__device__ __forceinline__ void epi_window(uint32_t taddr, long g, __half *o, __half *olo, long cstride, long ts,
                                           const float2 *gs, int t4)
{
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll 2
        for (int j8 = 0; j8 < 8; ++j8) {
            uint32_t r[NB][8];
#pragma unroll
            for (int k = 0; k < NB; ++k)
                tc::tmem_ld16x256_x2(taddr + ((uint32_t)(16 * u) << 16) + (uint32_t)(((g + k) & (kTcAcc - 1)) * 128) + 16 * j8,
                                     r[k]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int c = t4 + 4 * (2 * j8 + jj);
                const float2 gc = gs[c];
                const long roff = (long)(c - t4) * cstride + 2L * u * ts;
                __half *orow = o + roff;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const float2 re = __fmul2_rn(make_float2(__uint_as_float(r[k][4 * jj]), __uint_as_float(r[k][4 * jj + 2])), gc);
                    const __half2 h = __floats2half2_rn(re.x, re.y);
                    *reinterpret_cast<__half2 *>(orow + kMB * k) = h;
                    if constexpr (SPLIT) {
                        const float2 hf = __half22float2(h);
                        *reinterpret_cast<__half2 *>(olo + roff + kMB * k) = __floats2half2_rn(re.x - hf.x, re.y - hf.y);
                    }
                }
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const float2 im = __fmul2_rn(make_float2(__uint_as_float(r[k][4 * jj + 1]), __uint_as_float(r[k][4 * jj + 3])), gc);
                    const __half2 h = __floats2half2_rn(im.x, im.y);
                    *reinterpret_cast<__half2 *>(orow + ts + kMB * k) = h;
                    if constexpr (SPLIT) {
                        const float2 hf = __half22float2(h);
                        *reinterpret_cast<__half2 *>(olo + roff + ts + kMB * k) = __floats2half2_rn(im.x - hf.x, im.y - hf.y);
                    }
                }
            }
        }
    }
}

template <typename IN, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1) k_ppf64_tc(const __grid_constant__ WsParams P)
{
    using G = TcGeo<IN, SPLIT>;
    constexpr int NS = G::STAGES, NYB = G::NYB;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ int abort_flag;
    __shared__ uint32_t tmem_slot;
    __shared__ float2 tw[kC];     // W_64^t = cos - i sin: (cos, sin)
    __shared__ float2 gs[kC];     // bandpass x output scale, both halves
    const uint32_t s0 = su32(smem);
    const uint32_t bar0 = s0 + G::OFF_BAR;
    auto xfull = [&](int s) { return bar0 + 8u * s; };
    auto xempty = [&](int s) { return bar0 + 8u * (NS + s); };
    auto yfull = [&](int b) { return bar0 + 8u * (2 * NS + b); };
    auto yempty = [&](int b) { return bar0 + 8u * (2 * NS + 2 + b); };
    auto dfull = [&](int b) { return bar0 + 8u * (2 * NS + 4 + b); };
    auto dempty = [&](int b) { return bar0 + 8u * (2 * NS + 4 + kTcAcc + b); };
    const uint32_t done = bar0 + 8u * (2 * NS + 4 + 2 * kTcAcc);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            bar_init(xfull(s), 1);
            bar_init(xempty(s), kFirThreads);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(yfull(b), kFirThreads);
            bar_init(yempty(b), 1);
        }
        for (int b = 0; b < kTcAcc; ++b) {
            bar_init(dfull(b), 1);
            bar_init(dempty(b), kTcEpiThreads);
        }
        bar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.map)) : "memory");
    }
    if (warp == 1) tc::tmem_alloc(tc::smem_addr(&tmem_slot), kTcCols);
    if (tid < kC) {
        double sn, cs;
        sincospi((double)tid / 32.0, &sn, &cs);
        tw[tid] = make_float2((float)cs, (float)sn);
        const float g = __ldg(P.bp + tid) * P.osc / (SPLIT ? kTcTapScale : 1.f);
        gs[tid] = make_float2(g, g);
    }
    __syncthreads();
    // W row l = 2c + o, column pair (2n, 2n + 1): o = 0 (wr, -wi) = (cos, sin), o = 1 (wi, wr) = (-sin, cos);
    // split output also stores lo = fp16(w - hi) 32 KB on
    for (int e = tid; e < 128 * kC; e += kTcThreads) {
        const int l = e >> 6, n = e & 63, c = l >> 1;
        const float2 t = tw[(n * c) & 63];
        const float2 w = (l & 1) == 0 ? t : make_float2(-t.y, t.x);
        const __half2 v = __floats2half2_rn(w.x, w.y);
        const int off = (n >> 5) * 16384 + l * 128 + ((((n & 31) >> 2) ^ (l & 7)) << 4) + 4 * (n & 3);
        *reinterpret_cast<__half2 *>(smem + G::OFF_W + off) = v;
        if constexpr (SPLIT) {
            const float2 vf = __half22float2(v);
            *reinterpret_cast<__half2 *>(smem + G::OFF_W + 32768 + off) = __floats2half2_rn(w.x - vf.x, w.y - vf.y);
        }
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            long issued = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
                const ItemPos d = decode_item(P, item);
                const long nb = (d.m_hi - d.m_lo) / kMB;
                for (long j = 0; j <= nb && ok; ++j) {
                    const int s = (int)(issued % NS);
                    if (issued >= NS &&
                        !bar_wait(xempty(s), (uint32_t)(((issued / NS) - 1) & 1), &abort_flag, P.err, 31)) {
                        ok = false;
                        break;
                    }
                    const long srow = j == 0 ? d.m_lo * kC : (d.m_lo + kMB * (j - 1) + (kP - 1)) * kC;
                    const long y = srow + P.row0;
                    bar_expect(xfull(s), G::STAGE);
#pragma unroll
                    for (int q = 0; q < kRowsPerStage / kBoxRows; ++q)
                        tma_3d(s0 + G::OFF_X + s * G::STAGE + q * kBoxRows * G::ROWB, &P.map, xfull(s), d.grp * kTcNI,
                               (int)(y + q * kBoxRows), d.sb);
                    ++issued;
                }
            }
            // let the copies in flight land (all were consumed unless the CTA aborted)
            for (long q = issued - 1; q >= 0 && q >= issued - NS; --q) {
                const int s = (int)(q % NS);
                for (long long it = 0; it < (1LL << 22) && !bar_test(xfull(s), (uint32_t)((q / NS) & 1)); ++it)
                    __nanosleep(256);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            long g = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
                const ItemPos d = decode_item(P, item);
                for (long m0 = d.m_lo; m0 < d.m_hi; m0 += kMB, ++g) {
                    // FIR operand buffer and its round (NYB is 1 or 2)
                    const int b = NYB == 2 ? (int)(g & 1) : 0, da = (int)(g & (kTcAcc - 1));
                    const long yr = NYB == 2 ? (g >> 1) : g;
                    ok = bar_wait(yfull(b), (uint32_t)(yr & 1), &abort_flag, P.err, 32);
                    if (ok && g >= kTcAcc)
                        ok = bar_wait(dempty(da), (uint32_t)(((g / kTcAcc) - 1) & 1), &abort_flag, P.err, 33);
                    if (!ok) break;
                    tc::fence_after();
                    const uint32_t ya = s0 + G::OFF_Y + b * G::YB, wa = s0 + G::OFF_W;
                    if constexpr (SPLIT) {
                        // Yl Wh and Yh Wl first (small partial sums for the
                        // accumulator's truncating adds), then Yh Wh
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            const uint32_t koff = (ks >> 2) * 16384 + (ks & 3) * 32;
                            tc::mma_f16(tmem + da * 128, tc::desc_kmajor_sw128(ya + 32768 + koff),
                                        tc::desc_kmajor_sw128(wa + koff), kTcIdesc, ks > 0 ? 1u : 0u);
                        }
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            const uint32_t koff = (ks >> 2) * 16384 + (ks & 3) * 32;
                            tc::mma_f16(tmem + da * 128, tc::desc_kmajor_sw128(ya + koff),
                                        tc::desc_kmajor_sw128(wa + 32768 + koff), kTcIdesc, 1u);
                        }
                    }
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint32_t koff = (ks >> 2) * 16384 + (ks & 3) * 32;
                        tc::mma_f16(tmem + da * 128, tc::desc_kmajor_sw128(ya + koff), tc::desc_kmajor_sw128(wa + koff),
                                    kTcIdesc, (SPLIT || ks > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(yempty(b));
                    tc::mma_commit(dfull(da));
                }
            }
            // every MMA issued completes before TMEM is released
            tc::mma_commit(done);
            for (long long it = 0; it < (1LL << 22) && !bar_test(done, 0); ++it) __nanosleep(256);
        }
    } else if (warp < kTcFir0) {
        // ---------------- epilogue ----------------
        // warp quadrant q holds inputs 2q (lanes 32q .. + 15) and 2q + 1; in a
        // 16-lane group thread t reads lanes t / 4 and t / 4 + 8, i.e.
        // spectra mm = 2 ((t / 4) ^ 2q) and mm + 1, and channels t % 4 + 4k.
        // The batches of one 64-spectrum window (1 to 4 of them) are drained
        // together.
        const int q = warp & 3, t4 = lane & 3;
        const int mm = 2 * ((lane >> 2) ^ (2 * q));
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16);
        const long cstride = 2L * P.N * P.t_stride;           // elements between channels
        __half *out = static_cast<__half *>(P.out);
        __half *out_lo = static_cast<__half *>(P.out_lo);
        long g = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
            const ItemPos d = decode_item(P, item);
            // real row of (channel t4, input 2q), time mm
            const long obo = ((long)d.sb * kC * 2 * P.N + 2L * (d.grp * kTcNI + 2 * q)) * P.t_stride + t4 * cstride + mm;
            __half *ob = out + obo;
            __half *obl = SPLIT ? out_lo + obo : nullptr;
            for (long m0 = d.m_lo; m0 < d.m_hi && ok;) {
                const long wend = min(d.m_hi, (m0 / (kTcAcc * kMB) + 1) * (kTcAcc * kMB));
                const int nbw = (int)((wend - m0) / kMB);
                for (int k = 0; k < nbw && ok; ++k)
                    ok = bar_wait(dfull((int)((g + k) & (kTcAcc - 1))), (uint32_t)(((g + k) / kTcAcc) & 1), &abort_flag,
                                  P.err, 34);
                if (!ok) break;
                tc::fence_after();
                __half *wl = SPLIT ? obl + m0 : nullptr;
                switch (nbw) {
                case 1: epi_window<1, SPLIT>(taddr, g, ob + m0, wl, cstride, P.t_stride, gs, t4); break;
                case 2: epi_window<2, SPLIT>(taddr, g, ob + m0, wl, cstride, P.t_stride, gs, t4); break;
                case 3: epi_window<3, SPLIT>(taddr, g, ob + m0, wl, cstride, P.t_stride, gs, t4); break;
                default: epi_window<4, SPLIT>(taddr, g, ob + m0, wl, cstride, P.t_stride, gs, t4); break;
                }
                tc::fence_before();
                for (int k = 0; k < nbw; ++k) bar_arrive(dempty((int)((g + k) & (kTcAcc - 1))));
                g += nbw;
                m0 = wend;
            }
        }
    } else {
        // ---------------- FIR warps ----------------
        const int fi = tid - 32 * kTcFir0, ip = fi & 3, n = fi >> 2;
        float2 hr[kP];
#pragma unroll
        for (int k = 0; k < kP; ++k) {
            const float hv = __ldg(P.h + k * kC + n) * (SPLIT ? kTcTapScale : 1.f);
            hr[k] = make_float2(hv, hv);
        }
        float2 acc[2][kP];
        const int xoff = n * G::ROWB + ip * 2 * G::E;
        const int ch = (n & 31) >> 2, kb = (n >> 5) * 16384 + 32 * ip * 128 + 4 * (n & 3);
        int yx[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int xr = x ^ (2 * ip);
            yx[x] = kb + xr * 128 + ((ch ^ xr) << 4);
        }
        long L = 0, g = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
            const ItemPos d = decode_item(P, item);
            // prologue: the first 15 rows of the item's first window; sample k
            // is tap k - s of spectrum m_lo + s, s = 0 .. k.  An item that
            // starts at spectrum 0 of a push with history reads the stream rows
            // before the push from the history (the TMA stage holds zeros there).
            const bool from_hist = d.m_lo == 0 && P.n_hist > 0;
            const long hrow0 = ((long)d.sb * P.n_hist) * P.N + d.grp * kTcNI + 2 * ip;   // history element of row 0
            ok = bar_wait(xfull((int)(L % NS)), (uint32_t)((L / NS) & 1), &abort_flag, P.err, 35);
            if (!ok) break;
            {
                const unsigned char *xs = smem + G::OFF_X + (L % NS) * G::STAGE;
#pragma unroll
                for (int k = 0; k < kP - 1; ++k) {
                    float2 xv[2];
                    const long row = (long)k * kC + n;
                    if (from_hist && row < P.n_hist) hist_pair(P.hist, hrow0 + row * P.N, xv, IN{});
                    else unpack_pair(xs + k * kC * G::ROWB + xoff, xv, IN{});
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        acc[u][k] = __fmul2_rn(hr[0], xv[u]);
#pragma unroll
                        for (int s = 0; s < k; ++s) acc[u][s] = __ffma2_rn(hr[k - s], xv[u], acc[u][s]);
                    }
                }
                bar_arrive(xempty((int)(L % NS)));
                ++L;
            }
            for (long m0 = d.m_lo; m0 < d.m_hi; m0 += kMB, ++g) {
                const int b = NYB == 2 ? (int)(g & 1) : 0;
                const long yr = NYB == 2 ? (g >> 1) : g;
                if (g >= NYB) ok = bar_wait(yempty(b), (uint32_t)((yr - 1) & 1), &abort_flag, P.err, 36);
                if (ok) ok = bar_wait(xfull((int)(L % NS)), (uint32_t)((L / NS) & 1), &abort_flag, P.err, 37);
                if (!ok) break;
                const unsigned char *xs = smem + G::OFF_X + (L % NS) * G::STAGE;
                unsigned char *yb = smem + G::OFF_Y + b * G::YB;
                // the first batch's first sample is stream row 15 * 64 + n
                const long r0 = (long)(kP - 1) * kC + n;
                const long h0 = (from_hist && m0 == 0 && r0 < P.n_hist) ? hrow0 + r0 * P.N : -1;
                if (m0 + kMB <= P.T) fir_batch_tc<IN, false, SPLIT>(hr, acc, xs, yb, xoff, yx, m0, P.T, P.hist, h0);
                else fir_batch_tc<IN, true, SPLIT>(hr, acc, xs, yb, xoff, yx, m0, P.T, P.hist, h0);
                tc::fence_proxy_async();
                bar_arrive(xempty((int)(L % NS)));
                bar_arrive(yfull(b));
                ++L;
            }
        }
    }

    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTcCols);
    }
}

template <typename IN, bool SPLIT>
cudaError_t launch_tc_t(WsParams &P, int grid, cudaStream_t s)
{
    using G = TcGeo<IN, SPLIT>;
    auto kern = k_ppf64_tc<IN, SPLIT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    // a block's warps spread over the SM's four register-file partitions:
    // refuse a build whose register count leaves no room for the whole block
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < kTcThreads) return cudaErrorLaunchOutOfResources;
    kern<<<grid, kTcThreads, G::SMEM, s>>>(P);
    g_launches++;
    return cudaGetLastError();
}

template <typename IN, int OUTK>
cudaError_t launch_ws_t(WsParams &P, int grid, cudaStream_t s)
{
    using G = WsGeo<IN>;
    auto kern = k_ppf64_ws<IN, OUTK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreadsWs, G::SMEM, s>>>(P);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace

bool chan_ws_supported(acf_in_dtype dt, int C, int P, int N, const void *samples, long n_samples)
{
    if (C != kC || P != kP || (dt != ACF_IN_CI8 && dt != ACF_IN_CI16)) return false;
    if (n_samples < kBoxRows || n_samples > 0x7fffffffL) return false;   // a box never exceeds the rows
    const int ni = dt == ACF_IN_CI16 ? 4 : 8;
    return N % ni == 0 && reinterpret_cast<uintptr_t>(samples) % 16 == 0 && tensor_map_encoder() != nullptr;
}

// fp16 and split fp16 output take the tensor-core DFT (items of eight inputs)
static bool tc_variant(acf_in_dtype, int out_kind, int N, long t_stride, const void *out, const void *out_lo)
{
    auto a4 = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 4 == 0; };
    if (N % kTcNI != 0 || t_stride % 2 != 0 || !a4(out)) return false;
    return out_kind == OUT_F16 || (out_kind == OUT_F16X3 && out_lo && a4(out_lo));
}
// ... which also covers the spectra whose windows reach into a history
// shorter than one window (the streaming context's filter state)
static bool tc_reads_history(acf_in_dtype dt, const void *hist, long n_hist)
{
    return hist && n_hist > 0 && n_hist < (long)kC * kP &&
           reinterpret_cast<uintptr_t>(hist) % (dt == ACF_IN_CI16 ? 8 : 4) == 0;
}

long chan_ws_first_spectrum(long n_hist)
{
    // first spectrum whose window starts inside the pushed samples, rounded up to a batch
    return round_up((n_hist + kC - 1) / kC, kMB);
}

long chan_ws_begin(acf_in_dtype dt, int out_kind, int N, long t_stride, const void *out, const void *out_lo,
                   const void *hist, long n_hist)
{
    if (tc_variant(dt, out_kind, N, t_stride, out, out_lo) && (n_hist == 0 || tc_reads_history(dt, hist, n_hist)))
        return 0;
    return chan_ws_first_spectrum(n_hist);
}

cudaError_t launch_chan_ws(const void *hist, const void *samples, long n_samples, long n_hist, acf_in_dtype dt,
                           int n_sb, int N, const float *h, const float *bp, float scale, int out_kind, void *out,
                           void *out_lo, long t_stride, long T, cudaStream_t s)
{
    const long m_begin = chan_ws_begin(dt, out_kind, N, t_stride, out, out_lo, hist, n_hist);
    const long m_end = round_up(T, 64);
    if (m_end <= m_begin) return cudaSuccess;
    const int E = in_elem_bytes(dt);
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!enc) return cudaErrorNotSupported;
    WsParams P;
    std::memset(&P, 0, sizeof(P));
    const bool use_tc = tc_variant(dt, out_kind, N, t_stride, out, out_lo);
    if (use_tc && m_begin == 0 && n_hist > 0) {
        P.hist = hist;
        P.n_hist = n_hist;
    }
    const int NI = use_tc ? kTcNI : 16 / E;
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)n_samples, (cuuint64_t)n_sb};
    cuuint64_t strides[2] = {(cuuint64_t)N * E, (cuuint64_t)n_samples * N * E};
    cuuint32_t box[3] = {(cuuint32_t)NI, (cuuint32_t)kBoxRows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(&P.map, E == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                     const_cast<void *>(samples), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    P.h = h;
    P.bp = bp;
    P.osc = out_kind == OUT_F32 ? 1.f : scale;
    P.out = out;
    P.out_lo = out_lo;
    P.t_stride = t_stride;
    P.row0 = -n_hist;
    P.m_begin = m_begin;
    P.m_end = m_end;
    P.T = T;
    P.groups = (N + NI - 1) / NI;
    P.n_sb = n_sb;
    P.N = N;
    P.err = device_error_word();
    if (!P.err) return cudaErrorMemoryAllocation;
    // split each (subband, input group) into nseg time segments: the fewest
    // whose per-CTA load count (items per CTA x loads per item, prologue
    // included) is smallest
    const long nbat = (m_end - m_begin) / kMB;
    const long pairs = (long)n_sb * P.groups;
    long best = -1, best_cost = 0;
    for (long ns = 1; ns <= 8 && ns <= nbat; ++ns) {
        const long segb = (nbat + ns - 1) / ns;
        const long items = pairs * ((nbat + segb - 1) / segb);
        const long grid = std::min<long>(items, sms);
        const long cost = (items + grid - 1) / grid * (segb + 1);
        if (best < 0 || cost < best_cost) {
            best = segb;
            best_cost = cost;
        }
    }
    P.seg = best * kMB;
    const long nseg = (nbat + best - 1) / best;
    const long items = pairs * nseg;
    if (items > 0x7fffffffL) return cudaErrorInvalidValue;
    P.n_items = (int)items;
    const int grid = (int)std::min<long>(items, sms);
    if (use_tc && out_kind == OUT_F16X3)
        return dt == ACF_IN_CI16 ? launch_tc_t<short2, true>(P, grid, s) : launch_tc_t<char2, true>(P, grid, s);
    if (use_tc) return dt == ACF_IN_CI16 ? launch_tc_t<short2, false>(P, grid, s) : launch_tc_t<char2, false>(P, grid, s);
    if (dt == ACF_IN_CI16) {
        switch (out_kind) {
        case OUT_F32: return launch_ws_t<short2, OUT_F32>(P, grid, s);
        case OUT_F16: return launch_ws_t<short2, OUT_F16>(P, grid, s);
        default: return launch_ws_t<short2, OUT_F16X3>(P, grid, s);
        }
    }
    switch (out_kind) {
    case OUT_F32: return launch_ws_t<char2, OUT_F32>(P, grid, s);
    case OUT_F16: return launch_ws_t<char2, OUT_F16>(P, grid, s);
    default: return launch_ws_t<char2, OUT_F16X3>(P, grid, s);
    }
}

}  // namespace acf
