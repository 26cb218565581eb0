// Plain fp32 CUDA-core X-engine (Sec. 4.2.5): the comparison path.
//
// The paper's design divides each channel's covariance triangle into squares
// of 32x32 receivers, one work-group each, every thread holding a 2x2
// receiver tile in registers across the time loop.  Here a 128-thread block
// owns a 64x64 square of complex inputs and each thread an 8x4 tile (rows
// 2ty + 16a + {0, 1}, columns tx + 16b), so every operand value a thread
// loads from shared memory feeds 4 (row) or 8 (column) complex MACs.  The
// packed fp32x2 FMAs run over pairs of adjacent rows i0, i1: for V_ij +=
// x_i conj(y_j),
//   Re += (xr0, xr1) * (yr, yr) + (xi0, xi1) * (yi, yi)
//   Im += (xi0, xi1) * (yr, yr) - (xr0, xr1) * (yi, yi),
// so the row operand is read as (xr0, xr1) and (xi0, xi1) from separate real
// and imaginary planes and only the column value is duplicated in registers.
// The stages hold each operand value once (8 bytes a complex value): 3 bytes
// of shared-memory reads per complex MAC, 96 of the SM's 128 B/clk at the
// full FMA rate.
// Stages of 16 spectra are double buffered: the next stage's global loads
// (four lanes per 64-byte row piece) are in flight while the current one is
// multiplied.  Partial sums are flushed to
// V with atomic adds every CHUNK spectra (V is zeroed by the caller), which
// keeps the rounding error of long raw-subband integrations near
// sqrt(T / CHUNK) * 2^-24 relative.
#include "acf_internal.h"

namespace acf {
namespace {

constexpr int BT = 64;          // complex inputs per tile side
constexpr int KT = 16;          // spectra per stage
constexpr int NTH = 128;        // threads per block
constexpr int CHUNK = 4096;     // spectra per partial sum
constexpr size_t SMEM_SIMT = 2ull * 2 * KT * BT * sizeof(float2);   // A and B, two buffers: 32 KB

__device__ __forceinline__ void tri_decode(int k, int &bi, int &bj) {
    int b = (int)((sqrtf(8.f * (float)k + 1.f) - 1.f) * 0.5f);
    while ((b + 1) * (b + 2) / 2 <= k) ++b;
    while (b * (b + 1) / 2 > k) --b;
    bi = b;
    bj = k - b * (b + 1) / 2;
}

// Four spectra t .. t + 3 of one operand row; zeros past n_time.
__device__ __forceinline__ float4 row4(const float *src, long t, long n_time) {
    if (t + 3 < n_time) return __ldg(reinterpret_cast<const float4 *>(src + t));
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t + 0 < n_time) v.x = __ldg(src + t);
    if (t + 1 < n_time) v.y = __ldg(src + t + 1);
    if (t + 2 < n_time) v.z = __ldg(src + t + 2);
    return v;
}

__global__ void __launch_bounds__(NTH, 3)
k_xeng_simt(const float *__restrict__ x, int N, long n_time, long t_stride, float vscale, float2 *__restrict__ V)
{
    extern __shared__ __align__(16) float2 sm[];
    float (*Ar)[KT][BT] = reinterpret_cast<float (*)[KT][BT]>(sm);                   // [buf][t][i], real parts
    float (*Ai)[KT][BT] = reinterpret_cast<float (*)[KT][BT]>(sm + KT * BT);         // imaginary parts
    float2 (*Bs)[KT][BT] = reinterpret_cast<float2 (*)[KT][BT]>(sm + 2 * KT * BT);  // [buf][t][j], (re, im)
    int bi, bj;
    tri_decode(blockIdx.x, bi, bj);
    const long p = blockIdx.y;
    const float *xp = x + p * 2L * N * t_stride;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int i0 = bi * BT, j0 = bj * BT;

    // staging: threads 0-63 stage the A rows, 64-127 the B rows.  A thread
    // covers (4-spectrum group tg, input il) for il = il0 + 16 q: four lanes
    // read one row's 16 spectra (64 contiguous bytes), a warp 8 rows.  The
    // stage column of (t, i) is i ^ sw(t): for the 4-byte planes of A
    // sw(t) = 8 * ((t >> 2) & 3), for the 8-byte (re, im) values of B
    // sw(t) = 4 * ((t >> 2) & 3); either keeps the transposing stores of a
    // warp on distinct banks (and adjacent A rows adjacent); the MAC loads
    // apply the same swizzles.
    const int se = tid & 63, tg = se & 3, il0 = se >> 2;
    const bool stage_b = tid >= 64;
    const int nbase = stage_b ? j0 : i0;
    float4 pre[4][2];            // (q, re | im): 4 spectra each

    auto fetch = [&](long t0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = nbase + il0 + 16 * q;
            if (n < N) {
                const float *re_row = xp + 2L * n * t_stride;
                pre[q][0] = row4(re_row, t0 + 4 * tg, n_time);
                pre[q][1] = row4(re_row + t_stride, t0 + 4 * tg, n_time);
            } else {
                pre[q][0] = pre[q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    auto deposit = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float r[4] = {pre[q][0].x, pre[q][0].y, pre[q][0].z, pre[q][0].w};
            const float m[4] = {pre[q][1].x, pre[q][1].y, pre[q][1].z, pre[q][1].w};
            if (stage_b) {
                const int col = (il0 + 16 * q) ^ (4 * tg);
#pragma unroll
                for (int k = 0; k < 4; ++k) Bs[buf][4 * tg + k][col] = make_float2(r[k], m[k]);
            } else {
                const int col = (il0 + 16 * q) ^ (8 * tg);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    Ar[buf][4 * tg + k][col] = r[k];
                    Ai[buf][4 * tg + k][col] = m[k];
                }
            }
        }
    };

    // accR[a][b] = (Re V, Re V) and accI[a][b] = (Im V, Im V) of rows
    // 2ty + 16a and 2ty + 16a + 1 against column tx + 16b
    float2 accR[4][4], accI[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accR[a][b] = accI[a][b] = make_float2(0.f, 0.f);

    const long NB = (long)N * (N + 1) / 2;
    auto flush = [&]() {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = i0 + 2 * ty + 16 * a, j = j0 + tx + 16 * b;
                if (i < N && j <= i)
                    atomicAdd(&V[p * NB + (long)i * (i + 1) / 2 + j], make_float2(accR[a][b].x * vscale, accI[a][b].x * vscale));
                if (i + 1 < N && j <= i + 1)
                    atomicAdd(&V[p * NB + (long)(i + 1) * (i + 2) / 2 + j],
                              make_float2(accR[a][b].y * vscale, accI[a][b].y * vscale));
                accR[a][b] = accI[a][b] = make_float2(0.f, 0.f);
            }
    };

    fetch(0);
    deposit(0);
    __syncthreads();
    int buf = 0;
    long since = 0;
    for (long t0 = 0; t0 < n_time; t0 += KT) {
        const bool more = t0 + KT < n_time;
        if (more) fetch(t0 + KT);            // in flight during this stage's MACs
#pragma unroll 2
        for (int tt = 0; tt < KT; ++tt) {
            const int swa = 8 * ((tt >> 2) & 3), swb = 4 * ((tt >> 2) & 3);
            float2 xr[4], xi[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                xr[a] = *reinterpret_cast<const float2 *>(&Ar[buf][tt][(2 * ty + 16 * a) ^ swa]);
                xi[a] = *reinterpret_cast<const float2 *>(&Ai[buf][tt][(2 * ty + 16 * a) ^ swa]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[buf][tt][(tx + 16 * b) ^ swb];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float2 yr = make_float2(bv[b].x, bv[b].x), yi = make_float2(bv[b].y, bv[b].y);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    accR[a][b] = __ffma2_rn(xr[a], yr, accR[a][b]);
                    accR[a][b] = __ffma2_rn(xi[a], yi, accR[a][b]);
                    accI[a][b] = __ffma2_rn(xi[a], yr, accI[a][b]);
                    accI[a][b] = __ffma2_rn(make_float2(-xr[a].x, -xr[a].y), yi, accI[a][b]);
                }
            }
        }
        since += KT;
        if (since >= CHUNK && more) {
            flush();
            since = 0;
        }
        if (more) deposit(buf ^ 1);          // the other buffer: last read before the previous barrier
        __syncthreads();
        buf ^= 1;
    }
    flush();
}

}  // namespace

cudaError_t launch_xeng_simt(const float *x, int n_problems, int N, long n_time, long t_stride,
                             float vscale, float2 *V, cudaStream_t s)
{
    if (n_problems <= 0 || N <= 0 || n_time <= 0) return cudaSuccess;
    if (n_problems > 65535) return cudaErrorInvalidValue;
    const int nt = (N + BT - 1) / BT;
    cudaError_t e = cudaFuncSetAttribute(k_xeng_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_SIMT);
    if (e != cudaSuccess) return e;
    dim3 grid(nt * (nt + 1) / 2, n_problems);
    k_xeng_simt<<<grid, NTH, SMEM_SIMT, s>>>(x, N, n_time, t_stride, vscale, V);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace acf
