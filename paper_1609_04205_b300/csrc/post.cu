// Post-correlation steps on the visibilities V (packed lower triangles,
// [problem][bl], bl = i(i+1)/2 + j, problem = subband * n_channels + channel):
//   delay compensation as phase rotations of V (Sec. 4.2.4),
//   channel integration to a coarser resolution (Sec. 4.2.4),
//   the weighting matrix for lost data and re-weighting (Sec. 4.2.1, 4.3),
//   two-stage sigma-clip flagging (Sec. 4.3).
// All are single passes over V, bound by HBM bandwidth; the lost-data weights
// are a 1-bit correlation done with AND + popcount on bit-packed masks.
#include <cmath>

#include "acf_internal.h"

namespace acf {
namespace {

// Row i of packed baseline bl (largest i with i(i+1)/2 <= bl): an fp32
// estimate corrected in integers (fp64 throughput is low on this part).
__device__ __forceinline__ int tri_row(long bl)
{
    int i = (int)((sqrtf(8.f * (float)bl + 1.f) - 1.f) * 0.5f);
    i = max(i, 0);
    while ((long)i * (i + 1) / 2 > bl) --i;
    while ((long)(i + 1) * (i + 2) / 2 <= bl) ++i;
    return i;
}

// Double-float accumulation in fp32 (fp64 throughput is low on this part):
// (sh, sl) holds an unevaluated sum; a square a*a enters exactly as the pair
// (a*a, fma(a, a, -a*a)) through TwoSum (Knuth), so sums of squares keep
// ~2^-44 relative accuracy over the short runs used here.
__device__ __forceinline__ void df_add_sq(float a, float &sh, float &sl)
{
    const float ph = a * a, pl = fmaf(a, a, -ph);
    const float t = sh + ph;
    const float bb = t - sh;
    const float e = (sh - (t - bb)) + (ph - bb);
    sh = t;
    sl += e + pl;
}
__device__ __forceinline__ double df_value(float sh, float sl) { return (double)sh + (double)sl; }

// Exact-in-effect tests of |v|^2 > t: the fp32 square pf = fma(x, x, y*y)
// (relative error below 2^-23) is compared with a threshold tf that carries a
// relative error of at most 2^-22, widened by a 2^-20 guard band on either
// side; outside the band the fp32 decision equals the exact one, inside it the
// caller settles the element with the fp64 square (exact for fp32 inputs up
// to the final rounding) against the fp64 threshold.  The fp64 work stays out
// of the per-element loops (band hits are collected in bit masks and settled
// afterwards), so the loops run at fp32 rate.
constexpr float kBandLo = 1.f - 0x1p-20f, kBandHi = 1.f + 0x1p-20f;
__device__ __forceinline__ double pow2_f64(float2 v) { return (double)v.x * v.x + (double)v.y * v.y; }

// a[p][i] = exp(+2 pi i f_p d_i), f_p the sky frequency of problem p's channel
// (natural DFT order: channel c at f_centre + c' fs / C, c' = c for 2c < C,
// else c - C).  The phase is reduced to turns in fp64 before the sine.
__global__ void k_delay_table(const double *__restrict__ delays, const double *__restrict__ fc, double fs, int C,
                              int N, long n_prob, float2 *__restrict__ tab)
{
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= n_prob * N) return;
    const long p = idx / N;
    const int i = (int)(idx - p * N);
    const int s = (int)(p / C), c = (int)(p % C);
    const int cc = 2 * c < C ? c : c - C;
    const double f = fc[s] + (double)cc * (fs / C);
    const double cyc = f * delays[i];
    const double turns = cyc - rint(cyc);
    double sn, cs;
    sincospi(2.0 * turns, &sn, &cs);
    tab[idx] = make_float2((float)cs, (float)sn);
}

// V_ij <- V_ij * a_i * conj(a_j); two baselines per thread (16-byte access).
__global__ void k_delay_apply(float2 *__restrict__ V, const float2 *__restrict__ tab, long NB, int N)
{
    const long p = blockIdx.y;
    const long b0 = 2 * (blockIdx.x * (long)blockDim.x + threadIdx.x);
    if (b0 >= NB) return;
    float2 *row = V + p * NB;
    const float2 *a = tab + p * N;
    int i = tri_row(b0);
    int j = (int)(b0 - (long)i * (i + 1) / 2);
    const bool two = b0 + 1 < NB;
    float2 v[2];
    const bool vec = two && ((reinterpret_cast<uintptr_t>(row + b0) & 15) == 0);
    if (vec) {
        const float4 q = *reinterpret_cast<const float4 *>(row + b0);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    } else {
        v[0] = row[b0];
        v[1] = two ? row[b0 + 1] : make_float2(0.f, 0.f);
    }
    float2 o[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 ai = a[i], aj = a[j];
        const float wr = ai.x * aj.x + ai.y * aj.y, wi = ai.y * aj.x - ai.x * aj.y;
        o[k] = make_float2(v[k].x * wr - v[k].y * wi, v[k].x * wi + v[k].y * wr);
        if (++j > i) {
            ++i;
            j = 0;
        }
    }
    if (vec) {
        *reinterpret_cast<float4 *>(row + b0) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    } else {
        row[b0] = o[0];
        if (two) row[b0 + 1] = o[1];
    }
}

// out[s][k][e] = sum_{g < G} in[s][k G + g][e] over 16-byte units e (two
// complex float32 or one complex int64) when every row is 16-byte aligned.
template <typename T4>
__global__ void k_integrate_vec(const T4 *__restrict__ in, T4 *__restrict__ out, long units, int C, int G)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= units) return;
    const int s = blockIdx.z, k = blockIdx.y;
    const T4 *src = in + ((long)s * C + (long)k * G) * units + e;
    T4 acc = src[0];
    for (int g = 1; g < G; ++g) {
        const T4 v = src[(long)g * units];
        acc.x += v.x;
        acc.y += v.y;
        if constexpr (sizeof(T4) == 16 && sizeof(acc.x) == 4) {
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    out[((long)s * (C / G) + k) * units + e] = acc;
}

// Scalar fallback: element type T (float for cf32 components, long long for ci64).
template <typename T>
__global__ void k_integrate_scalar(const T *__restrict__ in, T *__restrict__ out, long units, int C, int G)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= units) return;
    const int s = blockIdx.z, k = blockIdx.y;
    const T *src = in + ((long)s * C + (long)k * G) * units + e;
    T acc = src[0];
    for (int g = 1; g < G; ++g) acc += src[(long)g * units];
    out[((long)s * (C / G) + k) * units + e] = acc;
}

// Per problem: sum of |V|^2 over all baselines and over the autocorrelations,
// in fp64 (sum[p][0] all, sum[p][1] autos).  With NB even every problem row
// starts on a 16-byte boundary and a thread reads two baselines per float4,
// four loads in flight.
template <bool VEC>
__global__ void k_clip_sums(const float2 *__restrict__ V, long NB, int N, double *__restrict__ sums)
{
    const long p = blockIdx.y;
    const float2 *row = V + p * NB;
    float sh = 0.f, sl = 0.f;
    const long stride = (long)gridDim.x * blockDim.x;
    const long first = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (VEC) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
        const long n4 = NB / 2;
#pragma unroll 4
        for (long b = first; b < n4; b += stride) {
            const float4 v = __ldcs(r4 + b);
            df_add_sq(v.x, sh, sl);
            df_add_sq(v.y, sh, sl);
            df_add_sq(v.z, sh, sl);
            df_add_sq(v.w, sh, sl);
        }
    } else {
        for (long b = first; b < NB; b += stride) {
            const float2 v = row[b];
            df_add_sq(v.x, sh, sl);
            df_add_sq(v.y, sh, sl);
        }
    }
    double all = df_value(sh, sl), aut = 0.0;
    for (long i = first; i < N; i += stride) {
        const float2 v = row[i * (i + 1) / 2 + i];
        aut += (double)v.x * v.x + (double)v.y * v.y;
    }
    __shared__ double sa[32], su[32];
    for (int o = 16; o > 0; o >>= 1) {
        all += __shfl_down_sync(0xffffffffu, all, o);
        aut += __shfl_down_sync(0xffffffffu, aut, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = all;
        su[w] = aut;
    }
    __syncthreads();
    if (w == 0) {
        all = l < (int)(blockDim.x >> 5) ? sa[l] : 0.0;
        aut = l < (int)(blockDim.x >> 5) ? su[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            all += __shfl_down_sync(0xffffffffu, all, o);
            aut += __shfl_down_sync(0xffffffffu, aut, o);
        }
        if (l == 0) {
            atomicAdd(&sums[2 * p], all);
            atomicAdd(&sums[2 * p + 1], aut);
        }
    }
}

// Stage-1 threshold per problem: k1^2 * (mean |V|^2 over cross-correlations),
// evaluated in the oracle's order (mean first).
__global__ void k_clip_thr(const double *__restrict__ sums, long n_prob, long n_cross, double k1sq,
                           double *__restrict__ thr, float *__restrict__ thr_f)
{
    const long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (p >= n_prob) return;
    const double ms = n_cross > 0 ? (sums[2 * p] - sums[2 * p + 1]) / (double)n_cross : 0.0;
    thr[p] = k1sq * ms;
    thr_f[p] = (float)(k1sq * ms);
}

// Flags for one (subband, baseline) across its C <= CMAX channels, one thread
// per baseline, 128 baselines per block.  Stage 1 (per channel): |V|^2 >
// thr[channel] = k1^2 * mean over the channel's cross-correlations.  Stage 2
// (per baseline): |V|^2 > k2^2 * mean of |V|^2 over the channels stage 1
// kept, the mean a double-float sum of exact squares.  Both tests are exact in
// effect (fp32 outside a guard band, fp64 inside it), so every decision
// equals the fp64 comparison of the exact squares.  The stage-2 fp32
// threshold k2^2 * ((sh + sl) / n) takes four fp32 roundings (at most 2^-22
// relative); its fp64 form is formed only when some element lands in the band.
// Loads go out in branch-free batches of 8 channels; stage 2 re-reads the
// baseline's values, which are still in L2.  The flag bytes are collected in
// shared memory and written per channel as one 128-byte run with 16-byte
// stores (single-byte stores from scattered warps leave partial lines that
// cost DRAM read-modify-writes).  Autocorrelations are never flagged.
template <int CMAX>
__global__ void __launch_bounds__(128)
k_clip_flags(const float2 *__restrict__ V, long NB, int N, int C, const double *__restrict__ thr,
             const float *__restrict__ thr_f, double k2sq, unsigned char *__restrict__ flags)
{
    constexpr int NW = CMAX / 64, D = 8;
    __shared__ double th[CMAX];
    __shared__ float lo1[CMAX], hi1[CMAX];
    __shared__ __align__(16) unsigned char sf[CMAX][128];
    const int s = blockIdx.y, tid = threadIdx.x;
    for (int c = tid; c < C; c += blockDim.x) {
        th[c] = thr[(long)s * C + c];
        const float tf = thr_f[(long)s * C + c];
        lo1[c] = tf * kBandLo;
        hi1[c] = tf * kBandHi;
    }
    __syncthreads();
    const long b0 = (long)blockIdx.x * 128, b = b0 + tid;
    if (b < NB) {
        const int i = tri_row(b);
        if ((long)i * (i + 1) / 2 + i == b) {
            for (int c = 0; c < C; ++c) sf[c][tid] = 0;
        } else {
            const float2 *col = V + (long)s * C * NB + b;
            uint64_t f1[NW];
            float sh = 0.f, sl = 0.f;
            int n_keep = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                f1[w] = 0;
                uint64_t amb = 0;
                const int cb = 64 * w, ce = min(C, cb + 64);
                for (int c0 = cb; c0 < ce; c0 += D) {
                    float2 v[D];
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        v[k] = c0 + k < ce ? __ldcg(col + (long)(c0 + k) * NB) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const int c = c0 + k;
                        if (c < ce) {
                            const float pf = fmaf(v[k].x, v[k].x, v[k].y * v[k].y);
                            const uint64_t bit = 1ull << (c - cb);
                            if (pf > hi1[c]) {
                                f1[w] |= bit;
                            } else if (pf < lo1[c]) {
                                df_add_sq(v[k].x, sh, sl);
                                df_add_sq(v[k].y, sh, sl);
                                ++n_keep;
                            } else {
                                amb |= bit;
                            }
                        }
                    }
                }
                while (amb) {                       // guard-band channels, in fp64
                    const int k = __ffsll((long long)amb) - 1;
                    amb &= amb - 1;
                    const float2 v = col[(long)(cb + k) * NB];
                    if (pow2_f64(v) > th[cb + k]) {
                        f1[w] |= 1ull << k;
                    } else {
                        df_add_sq(v.x, sh, sl);
                        df_add_sq(v.y, sh, sl);
                        ++n_keep;
                    }
                }
            }
            const float t2f = n_keep > 0 ? (float)k2sq * ((sh + sl) / (float)n_keep) : 0.f;
            const float lo2 = t2f * kBandLo, hi2 = t2f * kBandHi;
            uint64_t amb2[NW];
            bool any = false;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                amb2[w] = 0;
                const int cb = 64 * w, ce = min(C, cb + 64);
                for (int c0 = cb; c0 < ce; c0 += D) {
                    float2 v[D];
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        v[k] = c0 + k < ce ? __ldcs(col + (long)(c0 + k) * NB) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const int c = c0 + k;
                        if (c < ce) {
                            unsigned char f = (f1[w] >> (c - cb)) & 1u;
                            if (!f) {
                                const float pf = fmaf(v[k].x, v[k].x, v[k].y * v[k].y);
                                if (pf > hi2) f = 1;
                                else if (pf >= lo2) amb2[w] |= 1ull << (c - cb);
                            }
                            sf[c][tid] = f;
                        }
                    }
                }
                any |= amb2[w] != 0;
            }
            if (any) {
                const double t2 = n_keep > 0 ? k2sq * (df_value(sh, sl) / n_keep) : 0.0;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    while (amb2[w]) {
                        const int k = __ffsll((long long)amb2[w]) - 1;
                        amb2[w] &= amb2[w] - 1;
                        sf[64 * w + k][tid] = pow2_f64(col[(long)(64 * w + k) * NB]) > t2 ? 1 : 0;
                    }
                }
            }
        }
    }
    __syncthreads();
    const long nval = NB - b0 < 128 ? NB - b0 : 128;
    unsigned char *fs = flags + (long)s * C * NB + b0;
    for (int idx = tid; idx < C * 8; idx += blockDim.x) {
        const int c = idx >> 3, q = idx & 7;
        unsigned char *dst = fs + (long)c * NB;
        if (nval == 128 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            __stcs(reinterpret_cast<uint4 *>(dst) + q, reinterpret_cast<const uint4 *>(sf[c])[q]);
        } else {
            for (int k = 16 * q; k < 16 * q + 16 && k < nval; ++k) dst[k] = sf[c][k];
        }
    }
}

// Bit-pack the masks: bits[n][w] bit k = (mask[32 w + k][n] != 0).
__global__ void k_pack_mask(const unsigned char *__restrict__ mask, long n_blocks, int N, long n_words,
                            uint32_t *__restrict__ bits)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const long w = blockIdx.y;
    if (n >= N) return;
    uint32_t v = 0;
    for (int k = 0; k < 32; ++k) {
        const long b = 32 * w + k;
        if (b < n_blocks && mask[b * N + n]) v |= 1u << k;
    }
    bits[(long)n * n_words + w] = v;
}

// W_ij = spb * sum_w popc(bits_i[w] & bits_j[w]) on 32 x 32 tiles of the
// lower triangle; masks staged through shared memory 32 words at a time.
__global__ void __launch_bounds__(256) k_weights(const uint32_t *__restrict__ bits, int N, long n_words, long spb,
                                                 long long *__restrict__ W)
{
    // tile (ti, tj) with ti >= tj from the linear block index
    const int t = blockIdx.x;
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    __shared__ uint32_t si[32][33], sj[32][33];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;   // 8 rows of 32
    int cnt[4] = {0, 0, 0, 0};
    for (long w0 = 0; w0 < n_words; w0 += 32) {
        for (int r = ly; r < 32; r += 8) {
            const int gi = 32 * ti + r, gj = 32 * tj + r;
            const long w = w0 + lx;
            si[r][lx] = (gi < N && w < n_words) ? bits[(long)gi * n_words + w] : 0u;
            sj[r][lx] = (gj < N && w < n_words) ? bits[(long)gj * n_words + w] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = ly + 8 * q;
#pragma unroll 8
            for (int k = 0; k < 32; ++k) cnt[q] += __popc(si[r][k] & sj[lx][k]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 32 * ti + ly + 8 * q, j = 32 * tj + lx;
        if (i < N && j <= i) W[(long)i * (i + 1) / 2 + j] = (long long)cnt[q] * spb;
    }
}

// V_ij <- V_ij * n_total / W_ij (0 where W_ij == 0) for every problem: the
// factor is formed once per baseline, then applied down the problems.
__global__ void k_reweight(float2 *__restrict__ V, const long long *__restrict__ W, long NB, long n_prob,
                           double n_total)
{
    const long b = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (b >= NB) return;
    const long long w = W[b];
    const float f = w > 0 ? (float)(n_total / (double)w) : 0.f;
    for (long p = blockIdx.y; p < n_prob; p += gridDim.y) {
        const float2 v = V[p * NB + b];
        V[p * NB + b] = make_float2(v.x * f, v.y * f);
    }
}

long n_bl(int N) { return (long)N * (N + 1) / 2; }

}  // namespace

cudaError_t launch_delay_table(const double *d_delays, const double *d_fc, double fs, int n_sb, int C, int N,
                               float2 *d_tab, cudaStream_t s)
{
    const long nt = (long)n_sb * C * N;
    k_delay_table<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(d_delays, d_fc, fs, C, N, (long)n_sb * C, d_tab);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_delay_apply(float2 *V, const float2 *d_tab, long n_prob, int N, cudaStream_t s)
{
    const long NB = n_bl(N);
    dim3 grid((unsigned)((NB / 2 + 1 + 255) / 256), (unsigned)n_prob);
    k_delay_apply<<<grid, 256, 0, s>>>(V, d_tab, NB, N);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_integrate(const void *in, void *out, int n_sb, int C, int N, int G, int int64, cudaStream_t s)
{
    const long NB = n_bl(N);
    const long bytes = NB * (int64 ? 16 : 8);
    const bool vec = bytes % 16 == 0 && (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16 == 0;
    if (vec) {
        const long units = bytes / 16;
        dim3 grid((unsigned)((units + 255) / 256), (unsigned)(C / G), (unsigned)n_sb);
        if (int64)
            k_integrate_vec<longlong2><<<grid, 256, 0, s>>>(static_cast<const longlong2 *>(in), static_cast<longlong2 *>(out), units, C, G);
        else
            k_integrate_vec<float4><<<grid, 256, 0, s>>>(static_cast<const float4 *>(in), static_cast<float4 *>(out), units, C, G);
    } else {
        const long units = NB * 2;
        dim3 grid((unsigned)((units + 255) / 256), (unsigned)(C / G), (unsigned)n_sb);
        if (int64)
            k_integrate_scalar<long long><<<grid, 256, 0, s>>>(static_cast<const long long *>(in), static_cast<long long *>(out), units, C, G);
        else
            k_integrate_scalar<float><<<grid, 256, 0, s>>>(static_cast<const float *>(in), static_cast<float *>(out), units, C, G);
    }
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_sigma_clip(const float2 *V, int n_sb, int C, int N, double k1, double k2, double *d_sums,
                              unsigned char *flags, cudaStream_t s)
{
    const long NB = n_bl(N);
    const long n_prob = (long)n_sb * C;
    cudaError_t e = cudaMemsetAsync(d_sums, 0, sizeof(double) * 2 * n_prob, s);
    if (e != cudaSuccess) return e;
    const bool vec = NB % 2 == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0;
    const unsigned bx = (unsigned)std::min<long>((NB + 255) / 256, 64);
    if (vec)
        k_clip_sums<true><<<dim3(bx, (unsigned)n_prob), 256, 0, s>>>(V, NB, N, d_sums);
    else
        k_clip_sums<false><<<dim3(bx, (unsigned)n_prob), 256, 0, s>>>(V, NB, N, d_sums);
    g_launches++;
    double *thr = d_sums + 2 * n_prob;
    float *thr_f = reinterpret_cast<float *>(thr + n_prob);
    k_clip_thr<<<(unsigned)((n_prob + 255) / 256), 256, 0, s>>>(d_sums, n_prob, (long)N * (N - 1) / 2, k1 * k1, thr,
                                                               thr_f);
    g_launches++;
    const dim3 fgrid((unsigned)((NB + 127) / 128), (unsigned)n_sb);
    if (C <= 64)
        k_clip_flags<64><<<fgrid, 128, 0, s>>>(V, NB, N, C, thr, thr_f, k2 * k2, flags);
    else
        k_clip_flags<256><<<fgrid, 128, 0, s>>>(V, NB, N, C, thr, thr_f, k2 * k2, flags);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_weights(const unsigned char *mask, long n_blocks, int N, long spb, uint32_t *d_bits, long long *W,
                           cudaStream_t s)
{
    const long n_words = (n_blocks + 31) / 32;
    k_pack_mask<<<dim3((unsigned)((N + 127) / 128), (unsigned)n_words), 128, 0, s>>>(mask, n_blocks, N, n_words, d_bits);
    g_launches++;
    const int nt = (N + 31) / 32;
    k_weights<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(d_bits, N, n_words, spb, W);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_reweight(float2 *V, const long long *W, long n_total, int n_prob, int N, cudaStream_t s)
{
    const long NB = n_bl(N);
    const unsigned gy = (unsigned)std::min<long>(n_prob, 16);
    k_reweight<<<dim3((unsigned)((NB + 255) / 256), gy), 256, 0, s>>>(V, W, NB, (long)n_prob, (double)n_total);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace acf

// ---------------------------------------------------------------------------
// C ABI (stateless entry points; see include/acf.h)
// ---------------------------------------------------------------------------
using namespace acf;

namespace {
bool dev_ptr_ok(const void *p) { return p != nullptr; }
size_t up16(size_t b) { return (b + 15) / 16 * 16; }
}  // namespace

extern "C" {

acf_status acf_delay_compensate(void *V, int n_subbands, int n_channels, int n_inputs, const double *delays,
                                const double *f_centre, double sample_rate, acf_stream_t stream)
{
    if (!dev_ptr_ok(V) || !delays || !f_centre || n_subbands < 1 || n_channels < 1 || n_inputs < 1 ||
        !(sample_rate > 0.0) || !std::isfinite(sample_rate))
        return ACF_EINVAL;
    if (n_subbands > 65535 || (long)n_subbands * n_channels > 65535) return ACF_EINVAL;
    for (int i = 0; i < n_inputs; ++i)
        if (!std::isfinite(delays[i])) return ACF_EINVAL;
    for (int k = 0; k < n_subbands; ++k)
        if (!std::isfinite(f_centre[k])) return ACF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const long n_prob = (long)n_subbands * n_channels;
    const size_t b_d = up16(sizeof(double) * n_inputs), b_f = up16(sizeof(double) * n_subbands);
    const size_t b_t = sizeof(float2) * (size_t)n_prob * n_inputs;
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, b_d + b_f + b_t, s) != cudaSuccess) return ACF_ENOMEM;
    double *dd = static_cast<double *>(buf);
    double *dfc = reinterpret_cast<double *>(static_cast<char *>(buf) + b_d);
    float2 *tab = reinterpret_cast<float2 *>(static_cast<char *>(buf) + b_d + b_f);
    cudaError_t e = cudaMemcpyAsync(dd, delays, sizeof(double) * n_inputs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dfc, f_centre, sizeof(double) * n_subbands, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_delay_table(dd, dfc, sample_rate, n_subbands, n_channels, n_inputs, tab, s);
    if (e == cudaSuccess) e = launch_delay_apply(static_cast<float2 *>(V), tab, n_prob, n_inputs, s);
    cudaFreeAsync(buf, s);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_integrate_channels(const void *V_in, void *V_out, int n_subbands, int n_channels, int n_inputs,
                                  int group, int vis_int64, acf_stream_t stream)
{
    if (!V_in || !V_out || V_in == V_out || n_subbands < 1 || n_channels < 1 || n_inputs < 1 || group < 1)
        return ACF_EINVAL;
    if (n_channels % group != 0) return ACF_EINVAL;
    if (group != n_channels && (n_channels / 2) % group != 0) return ACF_EINVAL;
    if (n_subbands > 65535 || n_channels / group > 65535) return ACF_EINVAL;
    cudaError_t e = launch_integrate(V_in, V_out, n_subbands, n_channels, n_inputs, group, vis_int64 ? 1 : 0,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_sigma_clip(const void *V, unsigned char *flags, int n_subbands, int n_channels, int n_inputs,
                          double k_chan, double k_vis, acf_stream_t stream)
{
    if (!V || !flags || n_subbands < 1 || n_channels < 1 || n_inputs < 1) return ACF_EINVAL;
    if (!(k_chan > 0.0) || !(k_vis > 0.0) || !std::isfinite(k_chan) || !std::isfinite(k_vis)) return ACF_EINVAL;
    if (n_channels > 256) return ACF_EINVAL;
    if (n_subbands > 65535 || (long)n_subbands * n_channels > 65535) return ACF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const long n_prob = (long)n_subbands * n_channels;
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, sizeof(double) * 4 * n_prob, s) != cudaSuccess) return ACF_ENOMEM;
    cudaError_t e = launch_sigma_clip(static_cast<const float2 *>(V), n_subbands, n_channels, n_inputs, k_chan, k_vis,
                                      static_cast<double *>(buf), flags, s);
    cudaFreeAsync(buf, s);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_lost_sample_weights(const unsigned char *mask, long n_blocks, int n_inputs, long samples_per_block,
                                   long long *W, acf_stream_t stream)
{
    if (!mask || !W || n_blocks < 1 || n_inputs < 1 || samples_per_block < 1) return ACF_EINVAL;
    const long n_words = (n_blocks + 31) / 32;
    if (n_words > 65535) return ACF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, sizeof(uint32_t) * (size_t)n_inputs * n_words, s) != cudaSuccess) return ACF_ENOMEM;
    cudaError_t e = launch_weights(mask, n_blocks, n_inputs, samples_per_block, static_cast<uint32_t *>(buf), W, s);
    cudaFreeAsync(buf, s);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_reweight(void *V, const long long *W, long n_total, int n_problems, int n_inputs, acf_stream_t stream)
{
    if (!V || !W || n_total < 0 || n_problems < 1 || n_problems > 65535 || n_inputs < 1) return ACF_EINVAL;
    cudaError_t e = launch_reweight(static_cast<float2 *>(V), W, n_total, n_problems, n_inputs, (cudaStream_t)stream);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

}  // extern "C"
