// 256-channel polyphase channeliser (Sec. 4.2.3: FIR + FFT) with the bandpass
// weights and the transpose into the X-engine operand rows (Sec. 4.2.4), for
// 16 taps and complex int8 / int16 input.
//
// A block owns one input of one subband over a segment of spectra (a multiple
// of 16) and has 256 threads.  Thread c owns polyphase phase c: its 16 taps
// and the last 16 samples of the phase stay in registers (a ring whose slot
// indices are static inside a 16-spectrum batch), so each input sample is
// read once, apart from a 15-row prologue per block, and the FIR costs 32 FMAs
// per complex sample.  The 256-point DFT of a spectrum is a four-step 16 x 16
// transform with c = q + 16 j and channel k = k1 + 16 k2:
//   pass 1 (thread q):  Z_q[k1] = W_256^{q k1} sum_j y[q + 16 j] W_16^{j k1}
//   pass 2 (thread k1): X[k1 + 16 k2] = sum_q Z_q[k1] W_16^{q k2}
// each a 16-point DFT in registers.  A batch holds the transforms of 16
// spectra, one pass task per thread.  The spectra sit in a shared buffer with
// entry (q, j) at 16 j + (q ^ j), which keeps the FIR writes and both passes
// free of bank conflicts; the 16 threads of one transform form a half-warp, so
// the passes need only warp-level ordering.  The weighted, converted results
// are staged spectrum-major and each output row (channel, input, re|im) leaves
// as one run of 16 spectra: 32 bytes in fp16, 64 in fp32, whole sectors.
#include <algorithm>
#include <type_traits>

#include "acf_internal.h"

namespace acf {
namespace {

constexpr int kC = 256;     // channels = threads per block
constexpr int kMB = 16;     // spectra per batch (== taps: static ring slots)

template <typename T> __device__ __forceinline__ float2 in2f(T v);
template <> __device__ __forceinline__ float2 in2f<char2>(char2 v) { return make_float2(v.x, v.y); }
template <> __device__ __forceinline__ float2 in2f<short2>(short2 v) { return make_float2(v.x, v.y); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In place: a_k <- sum_n a_n W_4^{nk}, W_4 = exp(-2 pi i / 4) = -i.
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
    const float2 d = csub(a1, a3);
    const float2 b3 = make_float2(d.y, -d.x);    // -i (a1 - a3)
    a0 = cadd(b0, b2);
    a2 = csub(b0, b2);
    a1 = cadd(b1, b3);
    a3 = csub(b1, b3);
}

// 16-point DFT, Z[k] = sum_n z[n] W_16^{nk}, as 4 x 4 (n = n1 + 4 n2,
// k = k1 + 4 k2).  Output Z[k] is left at z[dft16_slot(k)].
__host__ __device__ constexpr int dft16_slot(int k) { return 4 * (k & 3) + (k >> 2); }

__device__ __forceinline__ void dft16(float2 (&z)[16])
{
    // W_16^e for the products n1 k1 in {1, 2, 3, 4, 6, 9}: cos and sin of
    // multiples of pi/8
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) dft4(z[n1], z[n1 + 4], z[n1 + 8], z[n1 + 12]);
    // z[n1 + 4 k1] now holds the inner transform; twiddle by W_16^{n1 k1}
    z[5] = cmulf(z[5], make_float2(c1, -s1));      // n1 = 1, k1 = 1: W^1
    z[9] = cmulf(z[9], make_float2(r2, -r2));      // n1 = 1, k1 = 2: W^2
    z[13] = cmulf(z[13], make_float2(s1, -c1));    // n1 = 1, k1 = 3: W^3
    z[6] = cmulf(z[6], make_float2(r2, -r2));      // n1 = 2, k1 = 1: W^2
    z[10] = make_float2(z[10].y, -z[10].x);        // n1 = 2, k1 = 2: W^4 = -i
    z[14] = cmulf(z[14], make_float2(-r2, -r2));   // n1 = 2, k1 = 3: W^6
    z[7] = cmulf(z[7], make_float2(s1, -c1));      // n1 = 3, k1 = 1: W^3
    z[11] = cmulf(z[11], make_float2(-r2, -r2));   // n1 = 3, k1 = 2: W^6
    z[15] = cmulf(z[15], make_float2(-c1, s1));    // n1 = 3, k1 = 3: W^9
    // outer transform over n1 for each k1: Z[k1 + 4 k2] -> z[4 k1 + k2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(z[4 * k1], z[4 * k1 + 1], z[4 * k1 + 2], z[4 * k1 + 3]);
}

// entry (q, j) of one spectrum's buffer
__device__ __forceinline__ int spos(int q, int j) { return 16 * j + (q ^ j); }

// Corner turn of the stream (history, then the push) into input-major rows,
// out[subband][input][q] with row pitch ld, so that k_chan256 reads each
// phase's samples as contiguous runs: 32 x 32 tiles through shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
k_corner_turn(const T *__restrict__ hist, long n_hist, const T *__restrict__ in, long n_samples, int N,
              T *__restrict__ out, long ld)
{
    __shared__ T tile[32][33];
    const int sb = blockIdx.z;
    const long q0 = (long)blockIdx.x * 32;
    const int n0 = blockIdx.y * 32;
    const long L = n_hist + n_samples;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const long q = q0 + r;
        const int n = n0 + tx;
        T v = T(0);
        if (q < L && n < N)
            v = q < n_hist ? hist[((long)sb * n_hist + q) * N + n] : in[((long)sb * n_samples + (q - n_hist)) * N + n];
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int n = n0 + r;
        const long q = q0 + tx;
        if (n < N && q < L) out[((long)sb * N + n) * ld + q] = tile[tx][r];
    }
}

// The same corner turn for 2-byte elements (complex int8) when the input rows
// allow 4-byte access (N even, aligned buffers): 64 x 64 tiles, each warp
// loading 64 inputs of one stream row and storing 64 samples of one input row
// as single 128-byte lines.  The odd row pitch of 65 halfwords keeps the
// column reads of the second phase free of bank conflicts.  A pair whose
// second sample lies past the stream is padded with zero inside the row pitch.
__global__ void __launch_bounds__(256)
k_corner_turn16(const uint16_t *__restrict__ hist, long n_hist, const uint16_t *__restrict__ in, long n_samples,
                int N, uint16_t *__restrict__ out, long ld)
{
    __shared__ uint16_t tile[64][65];
    const int sb = blockIdx.z;
    const long q0 = (long)blockIdx.x * 64;
    const int n0 = blockIdx.y * 64;
    const long L = n_hist + n_samples;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = n0 + 2 * tx;
#pragma unroll
    for (int r = w; r < 64; r += 8) {
        const long q = q0 + r;
        uint32_t v = 0;
        if (q < L && n < N) {
            const uint16_t *src = q < n_hist ? hist + ((long)sb * n_hist + q) * N + n
                                             : in + ((long)sb * n_samples + (q - n_hist)) * N + n;
            v = __ldg(reinterpret_cast<const unsigned int *>(src));
        }
        tile[r][2 * tx] = (uint16_t)(v & 0xffffu);
        tile[r][2 * tx + 1] = (uint16_t)(v >> 16);
    }
    __syncthreads();
    const long q = q0 + 2 * tx;
#pragma unroll
    for (int c = w; c < 64; c += 8) {
        const int nc = n0 + c;
        if (nc < N && q < L) {
            const uint32_t v = (uint32_t)tile[2 * tx][c] | ((uint32_t)tile[2 * tx + 1][c] << 16);
            *reinterpret_cast<uint32_t *>(out + ((long)sb * N + nc) * ld + q) = v;
        }
    }
}

// IM: samples come from the corner-turned rows xim[subband][input][q] (pitch
// ld, history included) instead of the [time][input] stream.
// The corner-turned form needs fewer registers (no strided sample addresses):
// capped for two blocks per SM, it spills at most 12 bytes.
template <typename IN, int OUTK, bool IM>
__global__ void __launch_bounds__(kC, IM ? 2 : 1)
k_chan256(const IN *__restrict__ hist, long n_hist, const IN *__restrict__ in, long n_samples, int N,
          const float *__restrict__ h, const float *__restrict__ bp, const float2 *__restrict__ tw_g,
          void *__restrict__ out, void *__restrict__ out_lo, long t_stride, float scale, long T, long m_per_block,
          const IN *__restrict__ xim, long ld)
{
    __shared__ __align__(16) float2 buf[kMB * kC];   // 32 KB: spectra, then the staged results
    __shared__ float2 tw[kC];
    const int c = threadIdx.x;
    const int n = blockIdx.x;
    const int sb = blockIdx.z;
    const long T64 = (T + 63) / 64 * 64;
    const long m_lo = (long)blockIdx.y * m_per_block;
    const long m_hi = min(T64, m_lo + m_per_block);
    const long stream_len = n_hist + n_samples;
    const IN *hsb = hist ? hist + (long)sb * n_hist * N : nullptr;
    const IN *isb = in + (long)sb * n_samples * N;

    tw[c] = tw_g[c];
    float hk[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) hk[k] = __ldg(h + k * kC + c);
    const float osc = OUTK == OUT_F32 ? 1.f : scale;

    // sample of phase c in spectrum row r (stream index r * 256 + c)
    const IN *row = IM ? xim + ((long)sb * N + n) * ld : nullptr;
    auto fetch = [&](long r) -> IN {
        const long q = r * kC + c;
        if (q >= stream_len) return IN{};
        if (IM) return row[q];
        return q < n_hist ? hsb[q * N + n] : isb[(q - n_hist) * N + n];
    };
    float2 w[16];                       // ring: row r in slot r & 15
#pragma unroll
    for (int k = 0; k < 15; ++k) w[k] = in2f(fetch(m_lo + k));
    w[15] = make_float2(0.f, 0.f);
    IN nx[kMB];                         // the batch's new rows m0 + 15 .. m0 + 30
#pragma unroll
    for (int mm = 0; mm < kMB; ++mm) nx[mm] = fetch(m_lo + 15 + mm);

    const long R0 = ((long)sb * kC) * (2L * N) + 2L * n;   // operand row of (channel 0, input n, re)
    const long rstride = 2L * N;                            // rows between consecutive channels

    for (long m0 = m_lo; m0 < m_hi; m0 += kMB) {
        // 1. FIR of 16 spectra: y_m[c] = sum_k h[k C + c] u[(m + k) C + c]
#pragma unroll
        for (int mm = 0; mm < kMB; ++mm) {
            w[(mm + 15) & 15] = in2f(nx[mm]);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                acc.x = fmaf(hk[k], w[(mm + k) & 15].x, acc.x);
                acc.y = fmaf(hk[k], w[(mm + k) & 15].y, acc.y);
            }
            buf[mm * kC + spos(c & 15, c >> 4)] = acc;
        }
        // the next batch's rows: in flight during the transforms and the write-out
        if (m0 + kMB < m_hi) {
#pragma unroll
            for (int mm = 0; mm < kMB; ++mm) nx[mm] = fetch(m0 + kMB + 15 + mm);
        }
        __syncthreads();
        const int f = c >> 4, t16 = c & 15;     // transform (spectrum m0 + f), task within it
        float2 *yb = buf + f * kC;
        // 2. pass 1, thread q = t16
        {
            float2 z[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = yb[spos(t16, j)];
            dft16(z);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                float2 v = z[dft16_slot(k1)];
                if (k1 != 0) v = cmulf(v, tw[(t16 * k1) & (kC - 1)]);
                yb[spos(t16, k1)] = v;
            }
        }
        __syncwarp();
        // 3. pass 2, thread k1 = t16: channels k1 + 16 k2
        float2 z[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) z[q] = yb[spos(q, t16)];
        dft16(z);
        __syncthreads();                        // every transform read before the buffer is reused
        // 4. stage spectrum-major: word (f, ch ^ 16 (f & 1)) -- the two transforms of a
        //    warp write opposite bank halves
        const bool live = m0 + f < T;
        if constexpr (OUTK == OUT_F32) {
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int ch = t16 + 16 * k2;
                const float wc = __ldg(bp + ch);
                const float2 v = live ? make_float2(z[dft16_slot(k2)].x * wc, z[dft16_slot(k2)].y * wc)
                                      : make_float2(0.f, 0.f);
                buf[f * kC + (ch ^ (16 * (f & 1)))] = v;
            }
        } else {
            uint32_t *hw = reinterpret_cast<uint32_t *>(buf);          // [16][256] hi pairs
            uint32_t *lw = hw + kMB * kC;                              // [16][256] lo pairs
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int ch = t16 + 16 * k2;
                const float wc = __ldg(bp + ch) * osc;
                const float vr = live ? z[dft16_slot(k2)].x * wc : 0.f;
                const float vi = live ? z[dft16_slot(k2)].y * wc : 0.f;
                const __half2 hi = __floats2half2_rn(vr, vi);
                const int sidx = f * kC + (ch ^ (16 * (f & 1)));
                hw[sidx] = *reinterpret_cast<const uint32_t *>(&hi);
                if constexpr (OUTK == OUT_F16X3) {
                    const float2 hf = __half22float2(hi);
                    const __half2 lo = __floats2half2_rn(vr - hf.x, vi - hf.y);
                    lw[sidx] = *reinterpret_cast<const uint32_t *>(&lo);
                }
            }
        }
        __syncthreads();
        // 5. write-out: thread c stores channel c's re and im rows, spectra [m0, m0 + 16)
        const long row = R0 + (long)c * rstride;
        if constexpr (OUT_F32 == OUTK) {
            float re[16], im[16];
#pragma unroll
            for (int mm = 0; mm < kMB; ++mm) {
                const float2 v = buf[mm * kC + (c ^ (16 * (mm & 1)))];
                re[mm] = v.x;
                im[mm] = v.y;
            }
            float4 *dr = reinterpret_cast<float4 *>(static_cast<float *>(out) + row * t_stride + m0);
            float4 *di = reinterpret_cast<float4 *>(static_cast<float *>(out) + (row + 1) * t_stride + m0);
#pragma unroll
            for (int v4 = 0; v4 < 4; ++v4) {
                dr[v4] = make_float4(re[4 * v4], re[4 * v4 + 1], re[4 * v4 + 2], re[4 * v4 + 3]);
                di[v4] = make_float4(im[4 * v4], im[4 * v4 + 1], im[4 * v4 + 2], im[4 * v4 + 3]);
            }
        } else {
            const uint32_t *hw = reinterpret_cast<const uint32_t *>(buf);
#pragma unroll
            for (int plane = 0; plane < (OUTK == OUT_F16X3 ? 2 : 1); ++plane) {
                const uint32_t *pw = hw + plane * kMB * kC;
                uint32_t re[8], im[8];          // 16 halves each
#pragma unroll
                for (int p2 = 0; p2 < 8; ++p2) {
                    const uint32_t a = pw[(2 * p2) * kC + (c ^ (16 * ((2 * p2) & 1)))];
                    const uint32_t b = pw[(2 * p2 + 1) * kC + (c ^ (16 * ((2 * p2 + 1) & 1)))];
                    re[p2] = __byte_perm(a, b, 0x5410);     // (re_a, re_b)
                    im[p2] = __byte_perm(a, b, 0x7632);     // (im_a, im_b)
                }
                __half *base = static_cast<__half *>(plane ? out_lo : out);
                uint4 *dr = reinterpret_cast<uint4 *>(base + row * t_stride + m0);
                uint4 *di = reinterpret_cast<uint4 *>(base + (row + 1) * t_stride + m0);
                dr[0] = make_uint4(re[0], re[1], re[2], re[3]);
                dr[1] = make_uint4(re[4], re[5], re[6], re[7]);
                di[0] = make_uint4(im[0], im[1], im[2], im[3]);
                di[1] = make_uint4(im[4], im[5], im[6], im[7]);
            }
        }
        __syncthreads();                        // buffer free for the next batch
    }
}

template <typename IN, int OUTK>
cudaError_t launch_k(const void *hist, long n_hist, const void *samples, long n_samples, int n_sb, int N,
                     const float *h, const float *bp, const float2 *tw, void *out, void *out_lo, long t_stride,
                     float scale, long T, long mpb, dim3 grid, const void *xim, long ld, cudaStream_t s)
{
    if (xim)
        k_chan256<IN, OUTK, true><<<grid, kC, 0, s>>>(static_cast<const IN *>(hist), n_hist,
                                                     static_cast<const IN *>(samples), n_samples, N, h, bp, tw, out,
                                                     out_lo, t_stride, scale, T, mpb, static_cast<const IN *>(xim), ld);
    else
        k_chan256<IN, OUTK, false><<<grid, kC, 0, s>>>(static_cast<const IN *>(hist), n_hist,
                                                      static_cast<const IN *>(samples), n_samples, N, h, bp, tw, out,
                                                      out_lo, t_stride, scale, T, mpb, nullptr, 0);
    g_launches++;
    return cudaGetLastError();
}

template <typename IN>
cudaError_t launch_dt(int out_kind, const void *hist, long n_hist, const void *samples, long n_samples, int n_sb,
                      int N, const float *h, const float *bp, const float2 *tw, void *out, void *out_lo,
                      long t_stride, float scale, long T, long mpb, dim3 grid, void *scratch, cudaStream_t s)
{
    long ld = 0;
    if (scratch) {
        // corner turn first: [subband][input][q], q over history and push
        using W = typename std::conditional<sizeof(IN) == 2, uint16_t, uint32_t>::type;
        ld = chan256_row_pitch(n_hist, n_samples);
        const long L = n_hist + n_samples;
        auto a4 = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 4 == 0; };
        if (sizeof(IN) == 2 && N % 2 == 0 && a4(samples) && a4(scratch) && (!hist || a4(hist))) {
            const dim3 g((unsigned)((L + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)n_sb);
            k_corner_turn16<<<g, 256, 0, s>>>(static_cast<const uint16_t *>(hist), n_hist,
                                              static_cast<const uint16_t *>(samples), n_samples, N,
                                              static_cast<uint16_t *>(scratch), ld);
        } else {
            const dim3 g((unsigned)((L + 31) / 32), (unsigned)((N + 31) / 32), (unsigned)n_sb);
            k_corner_turn<W><<<g, 256, 0, s>>>(static_cast<const W *>(hist), n_hist, static_cast<const W *>(samples),
                                              n_samples, N, static_cast<W *>(scratch), ld);
        }
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    switch (out_kind) {
    case OUT_F32: return launch_k<IN, OUT_F32>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, mpb, grid, scratch, ld, s);
    case OUT_F16: return launch_k<IN, OUT_F16>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, mpb, grid, scratch, ld, s);
    case OUT_F16X3: return launch_k<IN, OUT_F16X3>(hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, mpb, grid, scratch, ld, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

long chan256_row_pitch(long n_hist, long n_samples) { return round_up(n_hist + n_samples, 16); }

size_t chan256_scratch_bytes(acf_in_dtype dt, int n_sb, int N, long n_hist, long n_samples)
{
    return (size_t)n_sb * N * chan256_row_pitch(n_hist, n_samples) * in_elem_bytes(dt);
}

bool chan256_supported(acf_in_dtype dt, int C, int P, long t_stride)
{
    return C == kC && P == 16 && (dt == ACF_IN_CI8 || dt == ACF_IN_CI16) && t_stride % 16 == 0;
}

cudaError_t launch_chan256(const void *hist, long n_hist, const void *samples, long n_samples, acf_in_dtype dt,
                           int n_sb, int N, const float *h, const float *bp, const float2 *tw, int out_kind,
                           void *out, void *out_lo, long t_stride, float scale, long T, cudaStream_t s,
                           void *scratch, size_t scratch_bytes)
{
    // the corner-turned path when the caller lends a buffer large enough
    if (scratch && scratch_bytes < chan256_scratch_bytes(dt, n_sb, N, n_hist, n_samples)) scratch = nullptr;
    const long T64 = round_up(T, 64);
    if (T64 == 0) return cudaSuccess;
    if (N < 1 || n_sb < 1 || n_sb > 65535) return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // a shorter segment per block costs a 15-row prologue; split until the
    // grid holds a few blocks per SM
    long mpb = T64;
    while (mpb > kMB && (long)N * n_sb * ((T64 + mpb - 1) / mpb) < 4L * sms) mpb = std::max<long>(kMB, mpb / 2 / kMB * kMB);
    const long segs = (T64 + mpb - 1) / mpb;
    if (segs > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)N, (unsigned)segs, (unsigned)n_sb);
    switch (dt) {
    case ACF_IN_CI8: return launch_dt<char2>(out_kind, hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, mpb, grid, scratch, s);
    case ACF_IN_CI16: return launch_dt<short2>(out_kind, hist, n_hist, samples, n_samples, n_sb, N, h, bp, tw, out, out_lo, t_stride, scale, T, mpb, grid, scratch, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace acf
