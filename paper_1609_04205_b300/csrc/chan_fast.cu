// Fast path of the polyphase channeliser (Sec. 4.2.3 FIR + FFT, Sec. 4.2.4
// bandpass + transpose) for the production geometries: 16 taps, 16 or 64
// channels, complex int8 / int16 input.
//
// A block owns NI inputs of one subband and slides along time.  Each thread
// owns one input and two channel phases q and q + C/2 (L = C/2 lanes per
// input), keeping the last 16 samples of each phase in registers, so every
// input sample is read from DRAM once (apart from a 15-row prologue per block)
// and the FIR costs exactly 32 FMAs per complex sample.  The C-point FFT of
// one spectrum lives in the L lanes of its input as a radix-2 DIF: the first
// stage pairs the thread's own two points; before each later stage a lane
// swaps one register with its partner (lane ^ 2^s) so that both points of the
// next butterfly sit in one thread, which then computes it without any
// predication.  Lane l ends with channels bitrev(l) and bitrev(l) + C/2.
// Input rows are fetched with 16-byte loads into registers one
// batch ahead (hiding DRAM latency behind the batch's arithmetic), transposed
// through shared memory, and results leave through shared memory as 16-byte
// stores of 8 consecutive spectra per output row.
#include "acf_internal.h"

namespace acf {
namespace {

constexpr int kNW = 8;            // warps per block
constexpr int kMB = 16;           // spectra per batch (== taps, so window slots are static)
constexpr int kP = 16;            // taps

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ int brev(int v, int bits) {
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}
__host__ __device__ constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v >> 1); }

template <typename T> __device__ __forceinline__ float2 tof2(T v);
template <> __device__ __forceinline__ float2 tof2<char2>(char2 v) { return make_float2(v.x, v.y); }
template <> __device__ __forceinline__ float2 tof2<short2>(short2 v) { return make_float2(v.x, v.y); }

template <int C, typename IN, int OUTK>
struct Geo {
    static constexpr int R = 2;                             // phases (points) per lane
    static constexpr int L = C / R;                         // lanes per input
    static constexpr int IPW = 32 / L;                      // inputs per warp
    static constexpr int NI = kNW * IPW;                    // inputs per block
    static constexpr int E = sizeof(IN);                    // bytes per sample
    static constexpr int VEC = 16 / E;                      // samples per 16-byte vector
    static constexpr int VPR = NI / VEC;                    // vectors per time row
    static constexpr int ROWS = kMB * C;                    // time rows per batch
    static constexpr int NV = ROWS * VPR;                   // vectors per batch
    static constexpr int VPT = NV / (kNW * 32);             // vectors per thread
    // row padding (elements) that keeps the FIR reads and the transposing deposit
    // writes free of shared-memory bank conflicts for 1 and 4 inputs per warp
    static constexpr int PADI = IPW == 1 ? 4 : 9;
    static constexpr int ROWI = ROWS + PADI;                // smem input row (per input)
    static constexpr int OE = OUTK == OUT_F32 ? 4 : 2;      // output element bytes
    static constexpr int NOUT = OUTK == OUT_F16X3 ? 2 : 1;  // output planes
    static constexpr size_t SIN = (size_t)NI * ROWI * E;
    static constexpr size_t SOUT = (size_t)kMB * NI * C * 2 * OE;
    static constexpr size_t SMEM = SIN + SOUT * NOUT;
    static_assert(NV % (kNW * 32) == 0, "batch must split evenly");
    static_assert(L <= 32 && 32 % L == 0, "lanes per input");
};

template <int C, typename IN, int OUTK>
__global__ void __launch_bounds__(kNW * 32, 1)
k_chan_fast(const IN *__restrict__ hist, long n_hist, const IN *__restrict__ in, long n_samples, int N,
            const float *__restrict__ h, const float *__restrict__ bp, const float2 *__restrict__ tw,
            void *__restrict__ out, void *__restrict__ out_lo, long t_stride, float scale, long T,
            long m_per_block, int vec_ok)
{
    using G = Geo<C, IN, OUTK>;
    constexpr int L = G::L, R = G::R, NI = G::NI, LB = clog2(L);
    extern __shared__ __align__(16) unsigned char smem[];
    IN *sin = reinterpret_cast<IN *>(smem);
    unsigned char *sout = smem + G::SIN;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int il = warp * G::IPW + lane / L;       // local input
    const int ql = lane % L;                       // lane within the input's group
    const int n0 = blockIdx.x * NI;

    const int sb = blockIdx.z;
    const long T64 = (T + 63) / 64 * 64;
    const long m_lo = (long)blockIdx.y * m_per_block;
    const long m_hi = min(T64, m_lo + m_per_block);
    const long stream_len = n_hist + n_samples;
    const IN *hsb = hist ? hist + (long)sb * n_hist * N : nullptr;
    const IN *isb = in + (long)sb * n_samples * N;

    // per-thread constants: taps, twiddles, bandpass * scale
    float2 hr[R][kP];           // (h, h) pairs for packed fp32x2 FMAs
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < kP; ++k) {
            const float hv = __ldg(h + k * C + ql + L * r);
            hr[r][k] = make_float2(hv, hv);
        }
    // stage LB (span L): W_C^{ql}; stage s < LB (span 2^s): W_{2^{s+1}}^{ql mod 2^s}
    const float2 tw_top = tw[ql];
    float2 tws[LB > 0 ? LB : 1];
#pragma unroll
    for (int st = 0; st < LB; ++st) {
        const int hh = 1 << st;
        tws[st] = tw[((ql & (hh - 1)) * (C / (2 * hh))) & (C - 1)];
    }
    const int c0 = brev(ql, LB), c1 = c0 + L;
    const float osc = (OUTK == OUT_F32 ? 1.f : scale);
    const float wsc0 = __ldg(bp + c0) * osc, wsc1 = __ldg(bp + c1) * osc;

    // global -> registers: VPT 16-byte vectors of block rows [b0, b0 + rows)
    uint4 pre[G::VPT];
    auto fetch = [&](long b0, int rows) {
#pragma unroll
        for (int v = 0; v < G::VPT; ++v) {
            const int e = tid + v * kNW * 32;
            const int row = e / G::VPR, vc = e % G::VPR;
            uint4 val = make_uint4(0, 0, 0, 0);
            const long t = b0 * C + row;
            if (row < rows * C && t < stream_len) {
                const int nn = n0 + vc * G::VEC;
                const IN *src = (t < n_hist) ? hsb + t * N + nn : isb + (t - n_hist) * N + nn;
                if (vec_ok && nn + G::VEC <= N) {
                    val = __ldg(reinterpret_cast<const uint4 *>(src));
                } else {
                    IN tmp[G::VEC];
#pragma unroll
                    for (int k = 0; k < G::VEC; ++k) tmp[k] = (nn + k < N) ? src[k] : IN{};
                    val = *reinterpret_cast<const uint4 *>(tmp);
                }
            }
            pre[v] = val;
        }
    };
    // registers -> smem, transposed to [input][time]
    auto deposit = [&]() {
#pragma unroll
        for (int v = 0; v < G::VPT; ++v) {
            const int e = tid + v * kNW * 32;
            const int row = e / G::VPR, vc = e % G::VPR;
            const IN *vals = reinterpret_cast<const IN *>(&pre[v]);
#pragma unroll
            for (int k = 0; k < G::VEC; ++k) sin[(vc * G::VEC + k) * G::ROWI + row] = vals[k];
        }
    };

    float2 win[R][kP];
    // prologue: the first kP-1 rows of every window
    fetch(m_lo, kP - 1);
    deposit();
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < kP - 1; ++k) win[r][k] = tof2(sin[il * G::ROWI + k * C + ql + L * r]);
    __syncthreads();
    fetch(m_lo + kP - 1, kMB);

    for (long m0 = m_lo; m0 < m_hi; m0 += kMB) {
        deposit();
        __syncthreads();
        if (m0 + kMB < m_hi) fetch(m0 + kMB + kP - 1, kMB);   // next batch, in flight during compute
#pragma unroll
        for (int mm = 0; mm < kMB; ++mm) {
            float2 z[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                win[r][(mm + kP - 1) % kP] = tof2(sin[il * G::ROWI + mm * C + ql + L * r]);
                float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < kP; k += 2) {
                    a0 = __ffma2_rn(hr[r][k], win[r][(mm + k) % kP], a0);
                    a1 = __ffma2_rn(hr[r][k + 1], win[r][(mm + k + 1) % kP], a1);
                }
                z[r] = __fadd2_rn(a0, a1);
            }
            // stage LB: the thread's own pair (q, q + L)
            {
                const float2 u = z[0], v = z[1];
                z[0] = make_float2(u.x + v.x, u.y + v.y);
                z[1] = cmul(make_float2(u.x - v.x, u.y - v.y), tw_top);
            }
            // stages LB-1 .. 0: exchange one point with lane ^ 2^s, then a local butterfly
#pragma unroll
            for (int st = LB - 1; st >= 0; --st) {
                const bool v = (ql >> st) & 1;
                const float2 snd = v ? z[0] : z[1];
                float2 rcv;
                rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, 1 << st);
                rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, 1 << st);
                if (v) z[0] = rcv;
                else z[1] = rcv;
                const float2 u = z[0], w = z[1];
                z[0] = make_float2(u.x + w.x, u.y + w.y);
                const float2 d = make_float2(u.x - w.x, u.y - w.y);
                z[1] = (st == 0) ? d : cmul(d, tws[st]);
            }
            // lane holds channels c0 = bitrev(ql) (z[0]) and c1 = c0 + L (z[1])
            const long ob0 = ((long)(mm * NI + il) * C + c0) * 2;
            const long ob1 = ((long)(mm * NI + il) * C + c1) * 2;
            if (OUTK == OUT_F32) {
                float *so = reinterpret_cast<float *>(sout);
                *reinterpret_cast<float2 *>(so + ob0) = make_float2(z[0].x * wsc0, z[0].y * wsc0);
                *reinterpret_cast<float2 *>(so + ob1) = make_float2(z[1].x * wsc1, z[1].y * wsc1);
            } else {
                const float a0 = z[0].x * wsc0, b0 = z[0].y * wsc0, a1 = z[1].x * wsc1, b1 = z[1].y * wsc1;
                const __half2 h0 = __floats2half2_rn(a0, b0), h1 = __floats2half2_rn(a1, b1);
                __half *so = reinterpret_cast<__half *>(sout);
                *reinterpret_cast<__half2 *>(so + ob0) = h0;
                *reinterpret_cast<__half2 *>(so + ob1) = h1;
                if (OUTK == OUT_F16X3) {
                    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
                    __half *sl = reinterpret_cast<__half *>(sout + G::SOUT);
                    *reinterpret_cast<__half2 *>(sl + ob0) = __floats2half2_rn(a0 - f0.x, b0 - f0.y);
                    *reinterpret_cast<__half2 *>(sl + ob1) = __floats2half2_rn(a1 - f1.x, b1 - f1.y);
                }
            }
        }
        __syncthreads();
        // store: rows (input, channel, re|im), 8 consecutive spectra per 16-byte piece
        constexpr int NROW = NI * C * 2;
        constexpr int GPR = kMB / 8;
        for (int e = tid; e < NROW * GPR * G::NOUT; e += kNW * 32) {
            const int plane = e / (NROW * GPR);
            const int rem = e % (NROW * GPR);
            const int row = rem % NROW, g = rem / NROW;
            const int comp = row & 1, c = (row >> 1) % C, li = row / (2 * C);
            const int nn = n0 + li;
            if (nn >= N) continue;
            const long grow = ((long)sb * C + c) * (2L * N) + 2L * nn + comp;
            const long m = m0 + g * 8;
            if (OUTK == OUT_F32) {
                const float *so = reinterpret_cast<const float *>(sout);
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    v[k] = (m + k < T) ? so[((long)((g * 8 + k) * NI + li) * C + c) * 2 + comp] : 0.f;
                float4 *d = reinterpret_cast<float4 *>(static_cast<float *>(out) + grow * t_stride + m);
                d[0] = make_float4(v[0], v[1], v[2], v[3]);
                d[1] = make_float4(v[4], v[5], v[6], v[7]);
            } else {
                const __half *so = reinterpret_cast<const __half *>(sout + plane * G::SOUT);
                __half v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    v[k] = (m + k < T) ? so[((long)((g * 8 + k) * NI + li) * C + c) * 2 + comp] : __float2half(0.f);
                __half *dst = static_cast<__half *>(plane ? out_lo : out);
                *reinterpret_cast<uint4 *>(dst + grow * t_stride + m) = *reinterpret_cast<const uint4 *>(v);
            }
        }
        // the next deposit overwrites sin only after this barrier (FIR reads are done)
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 64-channel variant: same FIR and I/O staging, but the FFT goes through shared
// memory as 8 x 8 (two passes of in-register radix-8 DFTs), which costs about
// half the instructions of the cross-lane radix-2 stages.  Warp w owns input w
// of the block; its FIR outputs y[mm][q] (16 spectra x 64 phases) are written to
// a warp-private buffer with rows of 65 complex values (a stride that keeps the
// strided radix-8 reads at two 8-byte wavefronts per warp access).
//   pass 1: for s < 8:   Z_s[k1] = sum_r y[s + 8r] W_8^{r k1} * W_64^{s k1} -> slot s + 8 k1
//   pass 2: for k1 < 8:  X[k1 + 8 k2] = sum_s Z_s[k1] W_8^{s k2}
// ---------------------------------------------------------------------------
// Complex add / subtract as one packed fp32x2 operation each.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }   // * (-i)

// In-register 8-point DFT, natural-order output: A[k] = sum_r a[r] exp(-2 pi i r k / 8).
__device__ __forceinline__ void dft8(float2 (&a)[8])
{
    const float r2 = 0.70710678118654752440f;
    float2 b[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        b[r] = cadd(a[r], a[r + 4]);
        b[r + 4] = csub(a[r], a[r + 4]);
    }
    // twiddles W_8^1, W_8^2 = -i, W_8^3 on the odd half
    b[5] = make_float2(r2 * (b[5].x + b[5].y), r2 * (b[5].y - b[5].x));
    b[6] = mul_mi(b[6]);
    b[7] = make_float2(r2 * (b[7].y - b[7].x), -r2 * (b[7].x + b[7].y));
    float2 c[8];
#pragma unroll
    for (int base = 0; base < 8; base += 4) {
        c[base + 0] = cadd(b[base + 0], b[base + 2]);
        c[base + 1] = cadd(b[base + 1], b[base + 3]);
        c[base + 2] = csub(b[base + 0], b[base + 2]);
        c[base + 3] = mul_mi(csub(b[base + 1], b[base + 3]));
    }
    // last stage, bit-reversed positions -> natural order
    a[0] = cadd(c[0], c[1]);
    a[4] = csub(c[0], c[1]);
    a[2] = cadd(c[2], c[3]);
    a[6] = csub(c[2], c[3]);
    a[1] = cadd(c[4], c[5]);
    a[5] = csub(c[4], c[5]);
    a[3] = cadd(c[6], c[7]);
    a[7] = csub(c[6], c[7]);
}

template <typename IN, int OUTK>
struct Geo64 {
    static constexpr int C = 64, NI = 4, NT = 256, E = sizeof(IN);   // 2 warps per input, 1 phase per thread
    static constexpr int VB = NI * E < 16 ? NI * E : 16;             // bytes per vector load
    static constexpr int VEC = VB / E, VPR = NI / VEC, ROWS = kMB * C, NV = ROWS * VPR;
    static constexpr int VPT = NV / NT;
    static constexpr int ROWI = ROWS + 4;
    // y rows: 64 complex + 8 of padding, so consecutive spectra start 8 bank
    // pairs apart; columns are XOR-swizzled by (spectrum & 7) in their low three
    // bits.  With the thread maps below, the FIR stores and both FFT passes touch
    // 16 distinct 8-byte bank pairs per half-warp.
    static constexpr int YS = C + 8;
    static constexpr int OE = OUTK == OUT_F32 ? 4 : 2;       // output element bytes
    static constexpr int NOUT = OUTK == OUT_F16X3 ? 2 : 1;   // output planes
    static constexpr int NROW = NI * C * 2;                  // output rows (input, channel, re|im)
    // staging row: the batch's 16 spectra of one output row, time-contiguous,
    // padded so the paired 32-bit stores and the 16-byte reads are conflict-free
    static constexpr int ORB = OUTK == OUT_F32 ? 96 : 48;
    static constexpr int PIECES = kMB * OE / 16;             // 16-byte pieces per row per batch
    static constexpr int SPT = NROW * PIECES * NOUT / NT;    // 16-byte stores per thread per batch
    static constexpr size_t SIN = ((size_t)NI * ROWI * E + 15) / 16 * 16;
    static constexpr size_t SY = (size_t)NI * kMB * YS * 8;
    static constexpr size_t SOUT = (size_t)NROW * ORB;
    static constexpr size_t STW = C * 8 + C * 4;              // twiddles + bandpass x scale
    static constexpr size_t SMEM = SIN + SY + SOUT * NOUT + STW;
    static_assert(NV % NT == 0 && (NROW * PIECES * NOUT) % NT == 0, "work must split evenly");
};

template <int VB> struct VecT;
template <> struct VecT<16> { using T = uint4; };
template <> struct VecT<8> { using T = uint2; };

// 64-channel channeliser.  Per batch of 16 spectra:
//   deposit   the batch's input rows (fetched one batch ahead into registers)
//             are transposed into one shared-memory row per input;
//   FIR       thread (input, phase q) slides its 16-tap window along the
//             batch: y[mm][q] for 16 spectra;
//   pass 1    thread (input, column s = q / 8) takes spectra q % 8 and q % 8 + 8:
//             8-point DFT over y[s + 8r], times W_64^(s k1) (twiddles held in
//             registers, fixed per thread), back to slot s + 8 k1;
//   pass 2    thread (input, k1 = q / 8), same two spectra: 8-point DFT over
//             slots 8 k1 + s gives channels c = k1 + 8 k2; bandpass x scale
//             (registers, fixed per thread); neighbouring lanes hold
//             consecutive spectra and swap one value per channel so that each
//             writes a time-contiguous pair of one output row (real or
//             imaginary part) to the staging buffer;
//   store     16-byte pieces of 8 spectra per output row go to global memory.
template <typename IN, int OUTK>
__global__ void __launch_bounds__(256, 2)
k_chan64(const IN *__restrict__ hist, long n_hist, const IN *__restrict__ in, long n_samples, int N,
         const float *__restrict__ h, const float *__restrict__ bp, const float2 *__restrict__ tw_g,
         void *__restrict__ out, void *__restrict__ out_lo, long t_stride, float scale, long T,
         long m_per_block, int vec_ok)
{
    using G = Geo64<IN, OUTK>;
    constexpr int C = 64, NI = G::NI, NT = G::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    IN *sin = reinterpret_cast<IN *>(smem);
    float2 *ybuf = reinterpret_cast<float2 *>(smem + G::SIN);
    unsigned char *sout = smem + G::SIN + G::SY;
    float2 *stw = reinterpret_cast<float2 *>(smem + G::SIN + G::SY + G::SOUT * G::NOUT);
    float *sbp = reinterpret_cast<float *>(stw + C);

    const int tid = threadIdx.x;
    const int il = tid >> 6;               // local input (two warps each)
    static_assert(NT == NI * 64, "one thread per (input, phase)");
    const int q = tid & 63;                // channel phase (FIR); FFT column / channel group (passes)
    const int n0 = blockIdx.x * NI;
    const int sb = blockIdx.z;
    const long T64 = (T + 63) / 64 * 64;
    const long m_lo = (long)blockIdx.y * m_per_block;
    const long m_hi = min(T64, m_lo + m_per_block);
    const long stream_len = n_hist + n_samples;
    const IN *hsb = hist ? hist + (long)sb * n_hist * N : nullptr;
    const IN *isb = in + (long)sb * n_samples * N;
    float2 *yw = ybuf + (size_t)il * kMB * G::YS;            // this input's y rows

    float2 hr[kP];              // (h, h): one packed fp32x2 FMA per tap updates (re, im)
#pragma unroll
    for (int k = 0; k < kP; ++k) {
        const float hv = __ldg(h + k * C + q);
        hr[k] = make_float2(hv, hv);
    }
    const int sw = q & 7;       // column swizzle of this thread's spectra (mm & 7)
    const int grp = q >> 3;     // pass-1 column s, pass-2 channel group k1
    if (tid < C) {             // read after the first barrier
        stw[tid] = tw_g[tid];
        sbp[tid] = __ldg(bp + tid) * (OUTK == OUT_F32 ? 1.f : scale);
    }

    using V = typename VecT<G::VB>::T;
    V pre[G::VPT];
    auto fetch = [&](long b0, int rows) {
#pragma unroll
        for (int v = 0; v < G::VPT; ++v) {
            const int e = tid + v * NT;
            const int row = e / G::VPR, vc = e % G::VPR;
            V val{};
            const long t = b0 * C + row;
            if (row < rows * C && t < stream_len) {
                const int nn = n0 + vc * G::VEC;
                const IN *src = (t < n_hist) ? hsb + t * N + nn : isb + (t - n_hist) * N + nn;
                if (vec_ok && nn + G::VEC <= N) {
                    val = __ldg(reinterpret_cast<const V *>(src));
                } else {
                    IN tmp[G::VEC];
#pragma unroll
                    for (int k = 0; k < G::VEC; ++k) tmp[k] = (nn + k < N) ? src[k] : IN{};
                    val = *reinterpret_cast<const V *>(tmp);
                }
            }
            pre[v] = val;
        }
    };
    auto deposit = [&]() {
#pragma unroll
        for (int v = 0; v < G::VPT; ++v) {
            const int e = tid + v * NT;
            const int row = e / G::VPR, vc = e % G::VPR;
            const IN *vals = reinterpret_cast<const IN *>(&pre[v]);
#pragma unroll
            for (int k = 0; k < G::VEC; ++k) sin[(vc * G::VEC + k) * G::ROWI + row] = vals[k];
        }
    };

    float2 win[kP];
    fetch(m_lo, kP - 1);
    deposit();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kP - 1; ++k) win[k] = tof2(sin[il * G::ROWI + k * C + q]);
    __syncthreads();
    fetch(m_lo + kP - 1, kMB);

    for (long m0 = m_lo; m0 < m_hi; m0 += kMB) {
        deposit();
        __syncthreads();
        if (m0 + kMB < m_hi) fetch(m0 + kMB + kP - 1, kMB);
        // FIR: y[mm][q]
#pragma unroll
        for (int mm = 0; mm < kMB; ++mm) {
            win[(mm + kP - 1) % kP] = tof2(sin[il * G::ROWI + mm * C + q]);
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kP; k += 2) {
                a0 = __ffma2_rn(hr[k], win[(mm + k) % kP], a0);
                a1 = __ffma2_rn(hr[k + 1], win[(mm + k + 1) % kP], a1);
            }
            yw[mm * G::YS + (q ^ (mm & 7))] = __fadd2_rn(a0, a1);
        }
        __syncthreads();
        // pass 1: column s = grp of spectra sw and sw + 8
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float2 *row = yw + (sw + 8 * j) * G::YS + (grp ^ sw);
            float2 a[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) a[r] = row[8 * r];
            dft8(a);
#pragma unroll
            for (int k1 = 1; k1 < 8; ++k1) a[k1] = cmul(a[k1], stw[(grp * k1) & 63]);
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) row[8 * k1] = a[k1];
        }
        __syncthreads();
        // pass 2: channels grp + 8 k2 of spectra sw and sw + 8
        const int odd = q & 1;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int mm = sw + 8 * j;
            const float2 *row = yw + mm * G::YS + 8 * grp;
            float2 a[8];
#pragma unroll
            for (int sx = 0; sx < 8; ++sx) a[sx] = row[sx ^ sw];
            dft8(a);
            const bool live = m0 + mm < T;          // spectra past T are written as zeros
            const int pcol = mm >> 1;               // pair of spectra (mm & ~1, mm | 1)
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                const float wc = sbp[grp + 8 * k2];
                float2 v = __fmul2_rn(a[k2], make_float2(wc, wc));
                if (!live) v = make_float2(0.f, 0.f);
                // even lane keeps Re of both spectra, odd lane Im of both
                const float recv = __shfl_xor_sync(0xffffffffu, odd ? v.x : v.y, 1);
                const float first = odd ? recv : v.x, second = odd ? v.y : recv;
                const int orow = il * 2 * C + 2 * (grp + 8 * k2) + odd;
                if (OUTK == OUT_F32) {
                    *reinterpret_cast<float2 *>(sout + (size_t)orow * G::ORB + 8 * pcol) = make_float2(first, second);
                } else {
                    const __half2 hv = __floats2half2_rn(first, second);
                    *reinterpret_cast<__half2 *>(sout + (size_t)orow * G::ORB + 4 * pcol) = hv;
                    if (OUTK == OUT_F16X3) {
                        const float2 f = __half22float2(hv);
                        *reinterpret_cast<__half2 *>(sout + G::SOUT + (size_t)orow * G::ORB + 4 * pcol) =
                            __floats2half2_rn(first - f.x, second - f.y);
                    }
                }
            }
        }
        __syncthreads();
        // store: 16-byte pieces; a quarter-warp reads one piece of 8 rows
        // (conflict-free staging reads), a warp writes whole 32-byte sectors.
        // Not unrolled: at the 128-register cap an unrolled store loop made
        // ptxas spill, and the spill reloads cost ~50% of the kernel time.
#pragma unroll 1
        for (int v = 0; v < G::SPT; ++v) {
            const int e = tid + v * NT;
            const int plane = e / (G::NROW * G::PIECES);
            const int e2 = e % (G::NROW * G::PIECES);
            const int piece = (e2 >> 3) % G::PIECES;
            const int row = (e2 & 7) + 8 * (e2 / (8 * G::PIECES));
            const int li = row / (2 * C), c = (row >> 1) % C, comp = row & 1;
            const int nn = n0 + li;
            if (nn < N) {
                const uint4 val = *reinterpret_cast<const uint4 *>(sout + plane * G::SOUT + (size_t)row * G::ORB + 16 * piece);
                const long gofs = (((long)sb * C + c) * (2L * N) + 2L * nn + comp) * t_stride + m0 + piece * (16 / G::OE);
                if (OUTK == OUT_F32) {
                    *reinterpret_cast<uint4 *>(static_cast<float *>(out) + gofs) = val;
                } else {
                    __half *dst = static_cast<__half *>(plane ? out_lo : out);
                    *reinterpret_cast<uint4 *>(dst + gofs) = val;
                }
            }
        }
        // no barrier here: the next writes to the staging buffer (pass 2) come
        // after the next batch's deposit, FIR and pass-1 barriers
    }
}

template <typename IN, int OUTK>
cudaError_t launch_64_t(const void *hist, long n_hist, const void *samples, long n_samples, int n_sb, int N,
                        const float *h, const float *bp, const float2 *tw, void *out, void *out_lo,
                        long t_stride, float scale, long T, cudaStream_t s)
{
    using G = Geo64<IN, OUTK>;
    const long T64 = (T + 63) / 64 * 64;
    if (T64 == 0) return cudaSuccess;
    auto kern = k_chan64<IN, OUTK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long groups = (N + G::NI - 1) / G::NI;
    long seg = 512;
    while (seg > 64 && groups * n_sb * ((T64 + seg - 1) / seg) < 8L * sms) seg /= 2;
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(samples) | reinterpret_cast<uintptr_t>(hist)) % G::VB == 0) &&
                        ((long)N * sizeof(IN)) % G::VB == 0;
    dim3 grid((unsigned)groups, (unsigned)((T64 + seg - 1) / seg), n_sb);
    kern<<<grid, G::NT, G::SMEM, s>>>(static_cast<const IN *>(hist), n_hist, static_cast<const IN *>(samples),
                                      n_samples, N, h, bp, tw, out, out_lo, t_stride, scale, T, seg,
                                      vec_ok ? 1 : 0);
    g_launches++;
    return cudaGetLastError();
}

template <int C, typename IN, int OUTK>
cudaError_t launch_fast_t(const void *hist, long n_hist, const void *samples, long n_samples, int n_sb, int N,
                          const float *h, const float *bp, const float2 *tw, void *out, void *out_lo,
                          long t_stride, float scale, long T, cudaStream_t s)
{
    using G = Geo<C, IN, OUTK>;
    const long T64 = (T + 63) / 64 * 64;
    if (T64 == 0) return cudaSuccess;
    auto kern = k_chan_fast<C, IN, OUTK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // segments long enough to amortise the 15-row prologue, enough blocks for the GPU
    const long groups = (N + G::NI - 1) / G::NI;
    long seg = 512;
    while (seg > 64 && groups * n_sb * ((T64 + seg - 1) / seg) < 4L * sms) seg /= 2;
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(samples) | reinterpret_cast<uintptr_t>(hist)) % 16 == 0) &&
                        ((long)N * sizeof(IN)) % 16 == 0;
    dim3 grid((unsigned)groups, (unsigned)((T64 + seg - 1) / seg), n_sb);
    kern<<<grid, kNW * 32, G::SMEM, s>>>(static_cast<const IN *>(hist), n_hist, static_cast<const IN *>(samples),
                                         n_samples, N, h, bp, tw, out, out_lo, t_stride, scale, T, seg,
                                         vec_ok ? 1 : 0);
    g_launches++;
    return cudaGetLastError();
}

template <int C, typename IN>
cudaError_t launch_fast_o(int out_kind, const void *hist, long n_hist, const void *samples, long n_samples, int n_sb,
                          int N, const float *h, const float *bp, const float2 *tw, void *out, void *out_lo,
                          long t_stride, float scale, long T, cudaStream_t s)
{
    if (C == 64) {
        switch (out_kind) {
        case OUT_F32: return launch_64_t<IN, OUT_F32>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
        case OUT_F16: return launch_64_t<IN, OUT_F16>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
        default:      return launch_64_t<IN, OUT_F16X3>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
        }
    }
    switch (out_kind) {
    case OUT_F32: return launch_fast_t<C, IN, OUT_F32>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
    case OUT_F16: return launch_fast_t<C, IN, OUT_F16>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
    default:      return launch_fast_t<C, IN, OUT_F16X3>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
    }
}

}  // namespace

bool chan_fast_supported(acf_in_dtype dt, int C, int P)
{
    return P == kP && (C == 16 || C == 64) && (dt == ACF_IN_CI8 || dt == ACF_IN_CI16);
}

cudaError_t launch_chan_fast(const void *hist, long n_hist, const void *samples, long n_samples, acf_in_dtype dt,
                             int n_sb, int N, int C, const float *h, const float *bp, const float2 *tw, int out_kind,
                             void *out, void *out_lo, long t_stride, float scale, long T, cudaStream_t s)
{
    if (dt == ACF_IN_CI8) {
        if (C == 64) return launch_fast_o<64, char2>(out_kind, hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
        if (C == 16) return launch_fast_o<16, char2>(out_kind, hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
    } else if (dt == ACF_IN_CI16) {
        if (C == 64) return launch_fast_o<64, short2>(out_kind, hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
        if (C == 16) return launch_fast_o<16, short2>(out_kind, hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace acf
