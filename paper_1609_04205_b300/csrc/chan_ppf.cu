// Polyphase filter-bank channeliser (Sec. 4.2.3: FIR + FFT) fused with the
// bandpass weights and the transpose into the X-engine operand layout
// (Sec. 4.2.4).  One kernel per block of spectra; HBM-bound by design.
//
// Block = (subband, NI consecutive inputs, a segment of spectra).  For each
// batch of MS spectra the block
//   1. stages the raw samples of the batch's FIR windows, [(MS+P-1)*C][NI],
//      in shared memory (loads of NI consecutive inputs per time row);
//   2. runs the FIR: thread <-> (input, channel phase), P taps per output;
//   3. runs one C-point FFT per (input, spectrum) with a four-step split:
//      R = C/L points per lane DFT'd in registers, a twiddle, then an L-lane
//      radix-2 DIF across the warp with shuffles (L = min(C, 32));
//   4. applies w_c, converts (fp32 / fp16 / fp16 hi+lo) and stores each
//      output row (channel, input, re|im) as MS consecutive spectra.
#include <algorithm>
#include <cstring>

#include "acf_internal.h"

namespace acf {

namespace {

template <typename T> struct InT;
template <> struct InT<char2>  { __device__ static float2 f(char2 v)  { return make_float2(v.x, v.y); } };
template <> struct InT<short2> { __device__ static float2 f(short2 v) { return make_float2(v.x, v.y); } };
template <> struct InT<float2> { __device__ static float2 f(float2 v) { return v; } };

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// exp(-2 pi i j / n) for the in-register stages (n <= 8).
__device__ __forceinline__ float2 small_twiddle(int j, int n) {
    const float r = 0.70710678118654752440f;
    if (j == 0) return make_float2(1.f, 0.f);
    if (n == 4) return make_float2(0.f, -1.f);
    // n == 8
    if (j == 1) return make_float2(r, -r);
    if (j == 2) return make_float2(0.f, -1.f);
    return make_float2(-r, -r);
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

__device__ __forceinline__ int bitrev(int v, int bits) {
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

constexpr int kThreads = 256;

__device__ __forceinline__ long round_up_dev(long a) { return (a + 63) / 64 * 64; }

template <int C, int MS, int NI, typename IN>
__global__ void __launch_bounds__(kThreads)
k_channelise(const IN *__restrict__ hist, long n_hist, const IN *__restrict__ in, long n_samples,
             int N, int P, const float *__restrict__ h, const float *__restrict__ bp,
             const float2 *__restrict__ tw_g, int out_kind, void *__restrict__ out,
             void *__restrict__ out_lo, long t_stride, float scale, long T, long m_per_block)
{
    constexpr int L = C < 32 ? C : 32;       // lanes per FFT
    constexpr int R = C / L;                 // points per lane
    constexpr int LB = ilog2c(L), RB = ilog2c(R);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);                   // [C]
    float2 *ybuf = tw + C;                                           // [NI][MS][C]
    IN *win = reinterpret_cast<IN *>(ybuf + NI * MS * C);            // [(MS+P-1)*C][NI]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n0 = blockIdx.x * NI;
    const int sb = blockIdx.z;
    const long T64 = round_up_dev(T);
    const long m_lo = (long)blockIdx.y * m_per_block;
    const long m_hi = min(T64, m_lo + m_per_block);
    const long stream_len = n_hist + n_samples;
    const int win_rows = (MS + P - 1) * C;

    for (int k = tid; k < C; k += kThreads) tw[k] = tw_g[k];

    const IN *hist_sb = hist ? hist + (long)sb * n_hist * N : nullptr;
    const IN *in_sb = in + (long)sb * n_samples * N;
    const long row_stride = t_stride;
    const long prob0 = (long)sb * C;

    for (long m0 = m_lo; m0 < m_hi; m0 += MS) {
        __syncthreads();   // previous batch fully stored; tw visible on first pass
        // 1. stage the FIR windows of spectra [m0, m0+MS)
        const long q0 = m0 * C;
        for (int e = tid; e < win_rows * NI; e += kThreads) {
            const int r = e / NI, ni = e - r * NI;
            const long q = q0 + r;
            const int n = n0 + ni;
            IN v;
            if (n < N && q < stream_len) {
                v = (q < n_hist) ? hist_sb[q * N + n] : in_sb[(q - n_hist) * N + n];
            } else {
                v = IN{};
            }
            win[e] = v;
        }
        __syncthreads();
        // 2. FIR: y_m[c] = sum_k h[kC + c] u[(m + k) C + c]
        constexpr int PAIRS = NI * C;
        if (P == 16) {
            // 16 taps: per (input, phase) the taps sit in registers and the
            // batch's MS + 15 samples slide through a register window, so a
            // sample is read from shared memory once per batch, not per tap
            for (int w = tid; w < PAIRS; w += kThreads) {
                const int c = w % C, ni = w / C;
                float hk[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) hk[k] = __ldg(h + k * C + c);
                float2 u[MS + 15];
#pragma unroll
                for (int r = 0; r < MS + 15; ++r) u[r] = InT<IN>::f(win[(r * C + c) * NI + ni]);
#pragma unroll
                for (int mm = 0; mm < MS; ++mm) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        acc.x = fmaf(hk[k], u[mm + k].x, acc.x);
                        acc.y = fmaf(hk[k], u[mm + k].y, acc.y);
                    }
                    ybuf[(ni * MS + mm) * C + c] = acc;
                }
            }
        } else
        {
        constexpr int G = PAIRS >= kThreads ? 1 : kThreads / PAIRS;
        constexpr int MSG = MS / G > 0 ? MS / G : 1;
        for (int w = tid; w < PAIRS * G; w += kThreads) {
            const int ni = w % NI;
            const int c = (w / NI) % C;
            const int g = w / PAIRS;
            for (int mm = g * MSG; mm < (g + 1) * MSG && mm < MS; ++mm) {
                float2 acc = make_float2(0.f, 0.f);
                for (int k = 0; k < P; ++k) {
                    const float hk = __ldg(h + k * C + c);
                    const float2 x = InT<IN>::f(win[((mm + k) * C + c) * NI + ni]);
                    acc.x = fmaf(hk, x.x, acc.x);
                    acc.y = fmaf(hk, x.y, acc.y);
                }
                ybuf[(ni * MS + mm) * C + c] = acc;
            }
        }
        }
        __syncthreads();
        // 3. FFT per (input, spectrum)
        constexpr int FPW = 32 / L;                 // FFTs per warp pass
        constexpr int NFFT = NI * MS;
        for (int f0 = warp * FPW; f0 < NFFT; f0 += (kThreads / 32) * FPW) {
            const int f = f0 + lane / L;
            const int l = lane % L;
            const bool act = f < NFFT;
            float2 z[R];
#pragma unroll
            for (int r = 0; r < R; ++r) z[r] = act ? ybuf[f * C + l + L * r] : make_float2(0.f, 0.f);
            // step 1: R-point DIF in registers (output index bit-reversed)
#pragma unroll
            for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
                for (int blk = 0; blk < R; blk += 2 * span) {
#pragma unroll
                    for (int j = 0; j < span; ++j) {
                        const float2 u = z[blk + j], v = z[blk + j + span];
                        z[blk + j] = make_float2(u.x + v.x, u.y + v.y);
                        const float2 d = make_float2(u.x - v.x, u.y - v.y);
                        z[blk + j + span] = (j == 0) ? d : cmul(d, small_twiddle(j, 2 * span));
                    }
                }
            }
            // step 2: twiddle W_C^{s l}, s = bitrev_R(k)
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int s = bitrev(k, RB);
                if (s != 0) z[k] = cmul(z[k], tw[(s * l) & (C - 1)]);
            }
            // step 3: L-point radix-2 DIF across lanes
#pragma unroll
            for (int hh = L / 2; hh >= 1; hh >>= 1) {
                const bool upper = (l & hh) != 0;
                const float2 w = tw[((l & (hh - 1)) * (C / (2 * hh))) & (C - 1)];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    float2 p;
                    p.x = __shfl_xor_sync(0xffffffffu, z[k].x, hh);
                    p.y = __shfl_xor_sync(0xffffffffu, z[k].y, hh);
                    if (!upper) {
                        z[k] = make_float2(z[k].x + p.x, z[k].y + p.y);
                    } else {
                        z[k] = cmul(make_float2(p.x - z[k].x, p.y - z[k].y), w);
                    }
                }
            }
            __syncwarp();
            if (act) {
                const int q = bitrev(l, LB);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int c = bitrev(k, RB) + R * q;
                    const float wc = __ldg(bp + c);
                    ybuf[f * C + c] = make_float2(z[k].x * wc, z[k].y * wc);
                }
            }
        }
        __syncthreads();
        // 4. store rows (channel c, input n, re|im): MS consecutive spectra
        const int nrows = C * NI * 2;
        for (int rr = tid; rr < nrows; rr += kThreads) {
            const int c = rr % C;
            const int comp = (rr / C) & 1;
            const int ni = rr / (2 * C);
            const int n = n0 + ni;
            if (n >= N) continue;
            const long row = (prob0 + c) * (2L * N) + 2L * n + comp;
            float vals[MS];
#pragma unroll
            for (int mm = 0; mm < MS; ++mm) {
                const float2 v = ybuf[(ni * MS + mm) * C + c];
                vals[mm] = (m0 + mm < T) ? (comp ? v.y : v.x) : 0.f;
            }
            if (out_kind == OUT_F32) {
                float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(out) + row * row_stride + m0);
#pragma unroll
                for (int v4 = 0; v4 < MS / 4; ++v4)
                    dst[v4] = make_float4(vals[4 * v4], vals[4 * v4 + 1], vals[4 * v4 + 2], vals[4 * v4 + 3]);
            } else {
                __half hi[MS], lo[MS];
#pragma unroll
                for (int mm = 0; mm < MS; ++mm) {
                    const float v = vals[mm] * scale;
                    hi[mm] = __float2half_rn(v);
                    lo[mm] = __float2half_rn(v - __half2float(hi[mm]));
                }
                uint4 *dh = reinterpret_cast<uint4 *>(static_cast<__half *>(out) + row * row_stride + m0);
#pragma unroll
                for (int v8 = 0; v8 < MS / 8; ++v8) dh[v8] = *reinterpret_cast<const uint4 *>(&hi[8 * v8]);
                if (out_kind == OUT_F16X3) {
                    uint4 *dl = reinterpret_cast<uint4 *>(static_cast<__half *>(out_lo) + row * row_stride + m0);
#pragma unroll
                    for (int v8 = 0; v8 < MS / 8; ++v8) dl[v8] = *reinterpret_cast<const uint4 *>(&lo[8 * v8]);
                }
            }
        }
    }
}

// Raw subband operand: [sb][t][N] complex -> rows (2n + comp) of t, tail zeroed.
template <typename IN>
__global__ void __launch_bounds__(256)
k_transpose_raw(const IN *__restrict__ in, long S, int N, int out_kind, void *__restrict__ out,
                void *__restrict__ out_lo, long t_stride, float scale)
{
    __shared__ float2 tile[64][33];
    const int sb = blockIdx.z;
    const long t0 = (long)blockIdx.x * 64;
    const int nb = blockIdx.y * 32;
    const int tid = threadIdx.x;
    for (int e = tid; e < 64 * 32; e += 256) {
        const int tt = e / 32, nn = e % 32;
        const long t = t0 + tt;
        const int n = nb + nn;
        float2 v = make_float2(0.f, 0.f);
        if (t < S && n < N) v = InT<IN>::f(in[((long)sb * S + t) * N + n]);
        tile[tt][nn] = v;
    }
    __syncthreads();
    // 64 rows (32 inputs x re|im) of 64 spectra; thread = (row, 8-sample group)
    for (int e = tid; e < 64 * 8; e += 256) {
        const int rowl = e / 8, grp = e % 8;
        const int nn = rowl >> 1, comp = rowl & 1;
        const int n = nb + nn;
        if (n >= N) continue;
        const long row = ((long)sb * 2 * N) + 2L * n + comp;
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 x = tile[grp * 8 + k][nn];
            v[k] = comp ? x.y : x.x;
        }
        const long off = row * t_stride + t0 + grp * 8;
        if (out_kind == OUT_F32) {
            float4 *d = reinterpret_cast<float4 *>(static_cast<float *>(out) + off);
            d[0] = make_float4(v[0], v[1], v[2], v[3]);
            d[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
            __half hi[8], lo[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float s = v[k] * scale;
                hi[k] = __float2half_rn(s);
                lo[k] = __float2half_rn(s - __half2float(hi[k]));
            }
            *reinterpret_cast<uint4 *>(static_cast<__half *>(out) + off) = *reinterpret_cast<const uint4 *>(hi);
            if (out_kind == OUT_F16X3)
                *reinterpret_cast<uint4 *>(static_cast<__half *>(out_lo) + off) = *reinterpret_cast<const uint4 *>(lo);
        }
    }
}

// Raw complex int8 subband -> fp16 operand rows (the INT8-exact path: int8
// values, and scaled by a power of two, are exact in fp16).  A block moves 64
// samples x 64 inputs: 16-byte loads of 8 inputs per time row (a row of the
// tile is one 128-byte line), converted to half2 (re, im) into a shared tile
// [input][time] whose 65-word rows keep the transposed reads conflict-free,
// then 16-byte stores of 8 consecutive samples of one output row (eight lanes
// per row: full 128-byte lines).  N must be a multiple of 8 and the samples
// 16-byte aligned.
__global__ void __launch_bounds__(256)
k_transpose_ci8_f16(const uint4 *__restrict__ in, long S, int N, __half *__restrict__ out, long t_stride, float scale)
{
    __shared__ uint32_t tile[64 * 65];
    const int sb = blockIdx.z;
    const long t0 = (long)blockIdx.x * 64;
    const int n0 = blockIdx.y * 64;
    const int tid = threadIdx.x;
    const __half2 sc = __float2half2_rn(scale);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = tid + 256 * k, r = e >> 3, c = e & 7;
        const long t = t0 + r;
        const int n = n0 + 8 * c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t < S && n < N) v = __ldg(in + (((long)sb * S + t) * N + n) / 8);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const short re = (signed char)((w[q] >> (16 * h)) & 0xffu);
                const short im = (signed char)((w[q] >> (16 * h + 8)) & 0xffu);
                __half2 hv = __halves2half2(__short2half_rn(re), __short2half_rn(im));
                if (scale != 1.f) hv = __hmul2(hv, sc);
                uint32_t u;
                memcpy(&u, &hv, 4);
                tile[(8 * c + 2 * q + h) * 65 + r] = u;
            }
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, g = lane & 7;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int nl = (warp + 8 * k) * 4 + (lane >> 3);
        const int n = n0 + nl;
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = tile[nl * 65 + 8 * g + j];
        const uint4 re = make_uint4(__byte_perm(v[0], v[1], 0x5410), __byte_perm(v[2], v[3], 0x5410),
                                    __byte_perm(v[4], v[5], 0x5410), __byte_perm(v[6], v[7], 0x5410));
        const uint4 im = make_uint4(__byte_perm(v[0], v[1], 0x7632), __byte_perm(v[2], v[3], 0x7632),
                                    __byte_perm(v[4], v[5], 0x7632), __byte_perm(v[6], v[7], 0x7632));
        if (n < N) {
            const long col = t0 + 8 * g;
            *reinterpret_cast<uint4 *>(out + ((long)sb * 2 * N + 2L * n) * t_stride + col) = re;
            *reinterpret_cast<uint4 *>(out + ((long)sb * 2 * N + 2L * n + 1) * t_stride + col) = im;
        }
    }
}

template <typename E>
__global__ void k_history(const E *__restrict__ hist, long n_hist, const E *__restrict__ in,
                          long n_samples, int N, long from, long count, E *__restrict__ dst,
                          long dst_cap)
{
    const int sb = blockIdx.y;
    const long total = count * N;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long q = from + e / N;
        const int n = (int)(e % N);
        E v = (q < n_hist) ? hist[((long)sb * n_hist + q) * N + n]
                           : in[((long)sb * n_samples + (q - n_hist)) * N + n];
        dst[((long)sb * dst_cap + e / N) * N + n] = v;
    }
}

template <int C, int MS, int NI, typename IN>
cudaError_t launch_t(const void *hist, long n_hist, const void *samples, long n_samples, int n_sb,
                     int N, int P, const float *h, const float *bp, const float2 *tw, int out_kind,
                     void *out, void *out_lo, long t_stride, float scale, long T, long m_head, cudaStream_t s)
{
    long T64 = round_up(T, 64);
    if (T64 == 0) return cudaSuccess;
    // Every batch re-stages its own FIR windows, so a shorter time segment per
    // block costs nothing extra: halve it until the grid fills the GPU.
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long groups = (N + NI - 1) / NI;
    long m_per_block = 256;
    while (m_per_block > MS && groups * n_sb * ((T64 + m_per_block - 1) / m_per_block) < 4L * sms) m_per_block /= 2;
    if (m_head > 0) {
        // only spectra [0, m_head): one segment per block, m_head a multiple of MS
        if (m_head % MS != 0) return cudaErrorInvalidValue;
        m_per_block = m_head;
        T64 = std::min(T64, m_head);
    }
    const size_t smem = C * sizeof(float2) + (size_t)NI * MS * C * sizeof(float2) +
                        (size_t)(MS + P - 1) * C * NI * sizeof(IN);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_channelise<C, MS, NI, IN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((N + NI - 1) / NI, (unsigned)((T64 + m_per_block - 1) / m_per_block), n_sb);
    kern<<<grid, kThreads, smem, s>>>(static_cast<const IN *>(hist), n_hist, static_cast<const IN *>(samples),
                                      n_samples, N, P, h, bp, tw, out_kind, out, out_lo, t_stride, scale, T,
                                      m_per_block);
    g_launches++;
    return cudaGetLastError();
}

template <typename IN>
cudaError_t launch_by_c(int C, const void *hist, long n_hist, const void *samples, long n_samples,
                        int n_sb, int N, int P, const float *h, const float *bp, const float2 *tw,
                        int out_kind, void *out, void *out_lo, long t_stride, float scale, long T,
                        long m_head, cudaStream_t s)
{
    constexpr int NI = sizeof(IN) == 8 ? 2 : 4;
    switch (C) {
    case 16:  return launch_t<16, 32, NI, IN>(hist, n_hist, samples, n_samples, n_sb, N, P, h, bp, tw, out_kind, out, out_lo, t_stride, scale, T, m_head, s);
    case 64:  return launch_t<64, 16, NI, IN>(hist, n_hist, samples, n_samples, n_sb, N, P, h, bp, tw, out_kind, out, out_lo, t_stride, scale, T, m_head, s);
    case 256: return launch_t<256, 8, NI, IN>(hist, n_hist, samples, n_samples, n_sb, N, P, h, bp, tw, out_kind, out, out_lo, t_stride, scale, T, m_head, s);
    default:  return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t make_twiddles(int C, float2 **d_tw)
{
    float2 *host = new float2[C];
    for (int k = 0; k < C; ++k) {
        const double a = -2.0 * 3.14159265358979323846 * (double)k / (double)C;
        host[k] = make_float2((float)cos(a), (float)sin(a));
    }
    cudaError_t e = cudaMalloc(d_tw, sizeof(float2) * C);
    if (e == cudaSuccess) e = cudaMemcpy(*d_tw, host, sizeof(float2) * C, cudaMemcpyHostToDevice);
    delete[] host;
    return e;
}

cudaError_t launch_channelise(const void *hist, long n_hist, const void *samples, long n_samples,
                              acf_in_dtype dt, int n_sb, int N, int C, int P, const float *h,
                              const float *bandpass, const float2 *tw, int out_kind, void *out,
                              void *out_lo, long t_stride, float scale, long T, cudaStream_t s, void *scratch,
                              size_t scratch_bytes)
{
    if (chan_ws_supported(dt, C, P, N, samples, n_samples)) {
        // spectra whose windows reach into the history and that the
        // warp-specialised kernel does not read itself: generic kernel
        const long m_head = std::min(chan_ws_begin(dt, out_kind, N, t_stride, out, out_lo, hist, n_hist), round_up(T, 64));
        cudaError_t e = cudaSuccess;
        if (m_head > 0)
            e = launch_channelise_head(hist, n_hist, samples, n_samples, dt, n_sb, N, C, P, h, bandpass, tw, out_kind,
                                       out, out_lo, t_stride, scale, T, m_head, s);
        if (e != cudaSuccess) return e;
        return launch_chan_ws(hist, samples, n_samples, n_hist, dt, n_sb, N, h, bandpass, scale, out_kind, out, out_lo,
                              t_stride, T, s);
    }
    if (chan256_supported(dt, C, P, t_stride))
        return launch_chan256(hist, n_hist, samples, n_samples, dt, n_sb, N, h, bandpass, tw, out_kind, out, out_lo,
                              t_stride, scale, T, s, scratch, scratch_bytes);
    if (chan_fast_supported(dt, C, P))
        return launch_chan_fast(hist, n_hist, samples, n_samples, dt, n_sb, N, C, h, bandpass, tw, out_kind, out,
                                out_lo, t_stride, scale, T, s);
    return launch_channelise_generic(hist, n_hist, samples, n_samples, dt, n_sb, N, C, P, h, bandpass, tw, out_kind,
                                     out, out_lo, t_stride, scale, T, s);
}

cudaError_t launch_channelise_head(const void *hist, long n_hist, const void *samples, long n_samples,
                                   acf_in_dtype dt, int n_sb, int N, int C, int P, const float *h,
                                   const float *bandpass, const float2 *tw, int out_kind, void *out,
                                   void *out_lo, long t_stride, float scale, long T, long m_head, cudaStream_t s)
{
    switch (dt) {
    case ACF_IN_CI8:  return launch_by_c<char2>(C, hist, n_hist, samples, n_samples, n_sb, N, P, h, bandpass, tw, out_kind, out, out_lo, t_stride, scale, T, m_head, s);
    case ACF_IN_CI16: return launch_by_c<short2>(C, hist, n_hist, samples, n_samples, n_sb, N, P, h, bandpass, tw, out_kind, out, out_lo, t_stride, scale, T, m_head, s);
    case ACF_IN_CF32: return launch_by_c<float2>(C, hist, n_hist, samples, n_samples, n_sb, N, P, h, bandpass, tw, out_kind, out, out_lo, t_stride, scale, T, m_head, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_channelise_generic(const void *hist, long n_hist, const void *samples, long n_samples,
                                      acf_in_dtype dt, int n_sb, int N, int C, int P, const float *h,
                                      const float *bandpass, const float2 *tw, int out_kind, void *out,
                                      void *out_lo, long t_stride, float scale, long T, cudaStream_t s)
{
    return launch_channelise_head(hist, n_hist, samples, n_samples, dt, n_sb, N, C, P, h, bandpass, tw, out_kind, out,
                                  out_lo, t_stride, scale, T, 0, s);
}

cudaError_t launch_transpose_raw(const void *samples, long n_samples, acf_in_dtype dt, int n_sb,
                                 int N, int out_kind, void *out, void *out_lo, long t_stride,
                                 float scale, cudaStream_t s)
{
    const long T64 = round_up(n_samples, 64);
    if (T64 == 0) return cudaSuccess;
    if (dt == ACF_IN_CI8 && out_kind == OUT_F16 && N % 8 == 0 && reinterpret_cast<uintptr_t>(samples) % 16 == 0) {
        dim3 g8((unsigned)(T64 / 64), (N + 63) / 64, n_sb);
        k_transpose_ci8_f16<<<g8, 256, 0, s>>>(static_cast<const uint4 *>(samples), n_samples, N,
                                                static_cast<__half *>(out), t_stride, scale);
        g_launches++;
        return cudaGetLastError();
    }
    dim3 grid((unsigned)(T64 / 64), (N + 31) / 32, n_sb);
    switch (dt) {
    case ACF_IN_CI8:  k_transpose_raw<char2><<<grid, 256, 0, s>>>(static_cast<const char2 *>(samples), n_samples, N, out_kind, out, out_lo, t_stride, scale); break;
    case ACF_IN_CI16: k_transpose_raw<short2><<<grid, 256, 0, s>>>(static_cast<const short2 *>(samples), n_samples, N, out_kind, out, out_lo, t_stride, scale); break;
    case ACF_IN_CF32: k_transpose_raw<float2><<<grid, 256, 0, s>>>(static_cast<const float2 *>(samples), n_samples, N, out_kind, out, out_lo, t_stride, scale); break;
    }
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_history(const void *hist, long n_hist, const void *samples, long n_samples,
                           acf_in_dtype dt, int n_sb, int N, long from, long count, void *dst,
                           long dst_cap, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const long total = count * N;
    dim3 grid((unsigned)std::min<long>((total + 255) / 256, 4096), n_sb);
    switch (in_elem_bytes(dt)) {
    case 2: k_history<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t *>(hist), n_hist, static_cast<const uint16_t *>(samples), n_samples, N, from, count, static_cast<uint16_t *>(dst), dst_cap); break;
    case 4: k_history<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t *>(hist), n_hist, static_cast<const uint32_t *>(samples), n_samples, N, from, count, static_cast<uint32_t *>(dst), dst_cap); break;
    default: k_history<uint64_t><<<grid, 256, 0, s>>>(static_cast<const uint64_t *>(hist), n_hist, static_cast<const uint64_t *>(samples), n_samples, N, from, count, static_cast<uint64_t *>(dst), dst_cap); break;
    }
    g_launches++;
    return cudaGetLastError();
}

}  // namespace acf
