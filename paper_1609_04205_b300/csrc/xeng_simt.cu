// Plain fp32 CUDA-core X-engine (Sec. 4.2.5): the comparison path.
//
// The paper's design divides each channel's covariance triangle into
// squares of 32x32 receivers, one work-group each, every thread holding a
// 2x2 receiver tile in registers across the time loop.  Here the square is
// 64x64 complex inputs per 256-thread block and each thread keeps a 4x4 tile
// (four loads per complex MAC pair instead of two), staged through shared
// memory 32 spectra at a time.  Accumulation is two-level: fp32 partial sums
// over chunks of 4096 spectra are folded into fp32 totals, which keeps the
// rounding error of long raw-subband integrations near sqrt(T)*2^-24 relative.
#include "acf_internal.h"

namespace acf {
namespace {

constexpr int TILE = 64, KT = 32, CHUNK = 4096;

__device__ __forceinline__ void tri_decode(int k, int &bi, int &bj) {
    int b = (int)((sqrtf(8.f * (float)k + 1.f) - 1.f) * 0.5f);
    while ((b + 1) * (b + 2) / 2 <= k) ++b;
    while (b * (b + 1) / 2 > k) --b;
    bi = b;
    bj = k - b * (b + 1) / 2;
}

__global__ void __launch_bounds__(256)
k_xeng_simt(const float *__restrict__ x, int N, long n_time, long t_stride, float vscale,
            float2 *__restrict__ V)
{
    __shared__ float As[KT][2][TILE + 4];
    __shared__ float Bs[KT][2][TILE + 4];
    int bi, bj;
    tri_decode(blockIdx.x, bi, bj);
    const long p = blockIdx.y;
    const float *xp = x + p * 2L * N * t_stride;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int i0 = bi * TILE, j0 = bj * TILE;

    float ar[4][4], ai[4][4], tr[4][4], ti[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = tr[a][b] = ti[a][b] = 0.f;

    long since = 0;
    for (long t0 = 0; t0 < n_time; t0 += KT) {
        // stage 64 inputs x (re, im) x 32 spectra for both row blocks
        for (int e = tid; e < 2 * TILE * 2 * (KT / 4); e += 256) {
            const int which = e / (TILE * 2 * (KT / 4));        // 0 = A rows, 1 = B rows
            const int r = (e / (KT / 4)) % (TILE * 2);          // local real row
            const int seg = e % (KT / 4);
            const int n = (which ? j0 : i0) + (r >> 1);
            const int comp = r & 1;
            const long t = t0 + seg * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n < N) {
                const float *src = xp + (2L * n + comp) * t_stride + t;
                if (t + 3 < n_time) {
                    v = *reinterpret_cast<const float4 *>(src);
                } else {
                    if (t + 0 < n_time) v.x = src[0];
                    if (t + 1 < n_time) v.y = src[1];
                    if (t + 2 < n_time) v.z = src[2];
                }
            }
            float (*S)[2][TILE + 4] = which ? Bs : As;
            S[seg * 4 + 0][comp][r >> 1] = v.x;
            S[seg * 4 + 1][comp][r >> 1] = v.y;
            S[seg * 4 + 2][comp][r >> 1] = v.z;
            S[seg * 4 + 3][comp][r >> 1] = v.w;
        }
        __syncthreads();
#pragma unroll 4
        for (int tt = 0; tt < KT; ++tt) {
            float xr[4], xi[4], yr[4], yi[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                xr[a] = As[tt][0][ty + 16 * a];
                xi[a] = As[tt][1][ty + 16 * a];
                yr[a] = Bs[tt][0][tx + 16 * a];
                yi[a] = Bs[tt][1][tx + 16 * a];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // x_i conj(y_j)
                    ar[a][b] = fmaf(xr[a], yr[b], ar[a][b]);
                    ar[a][b] = fmaf(xi[a], yi[b], ar[a][b]);
                    ai[a][b] = fmaf(xi[a], yr[b], ai[a][b]);
                    ai[a][b] = fmaf(-xr[a], yi[b], ai[a][b]);
                }
        }
        __syncthreads();
        since += KT;
        if (since >= CHUNK) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    tr[a][b] += ar[a][b];
                    ti[a][b] += ai[a][b];
                    ar[a][b] = ai[a][b] = 0.f;
                }
            since = 0;
        }
    }
    const long NB = (long)N * (N + 1) / 2;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < N && j <= i) {
                const float re = (tr[a][b] + ar[a][b]) * vscale;
                const float im = (ti[a][b] + ai[a][b]) * vscale;
                atomicAdd(&V[p * NB + (long)i * (i + 1) / 2 + j], make_float2(re, im));
            }
        }
}

}  // namespace

cudaError_t launch_xeng_simt(const float *x, int n_problems, int N, long n_time, long t_stride,
                             float vscale, float2 *V, cudaStream_t s)
{
    if (n_problems <= 0 || N <= 0 || n_time <= 0) return cudaSuccess;
    const int nt = (N + TILE - 1) / TILE;
    dim3 grid(nt * (nt + 1) / 2, n_problems);
    k_xeng_simt<<<grid, 256, 0, s>>>(x, N, n_time, t_stride, vscale, V);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace acf
