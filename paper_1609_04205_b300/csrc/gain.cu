// Gain-corrupted correlation M = G R G^H, its squared-Frobenius loss against
// observed visibilities and the adjoint (gradient) with respect to the
// per-input complex gains -- the calibration-facing form of the correlator
// output (Sec. 5 fits per-dipole gains to the visibilities).
//
// One pass over the packed lower triangles of R and V: a block owns a 64x64
// tile of one channel's triangle, forms E = g_i R_ij conj(g_j) - V_ij per
// element, adds w|E|^2 (w = 2 off the diagonal: the upper triangle is the
// conjugate) to a per-block partial, and accumulates the gradient rows
//   grad_i += 4 E_ij conj(R_ij) g_j      and, for i != j,
//   grad_j += 4 conj(E_ij) R_ij g_i      (= 4 E_ji conj(R_ji) g_i).
// Row sums are warp-reduced; each lane keeps the column sums of its two tile
// columns in registers, the warps' sums are combined once per tile in shared
// memory, and one global atomic per (tile row/column) lands in grad.  The per-block
// loss partials are summed by a second, single-block kernel in a fixed order,
// so the loss is deterministic.
#include <mutex>

#include "acf_internal.h"

namespace acf {
namespace {

constexpr int GT = 64;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ void tri_decode_g(int k, int &bi, int &bj) {
    int b = (int)((sqrtf(8.f * (float)k + 1.f) - 1.f) * 0.5f);
    while ((b + 1) * (b + 2) / 2 <= k) ++b;
    while (b * (b + 1) / 2 > k) --b;
    bi = b;
    bj = k - b * (b + 1) / 2;
}

__global__ void __launch_bounds__(256)
k_gain(const float2 *__restrict__ R, const float2 *__restrict__ V, const float2 *__restrict__ g,
       int N, float *__restrict__ partials, float2 *__restrict__ grad)
{
    __shared__ float2 gi_s[GT], gj_s[GT];
    __shared__ float2 colred[8][GT];
    __shared__ float red[8];
    int bi, bj;
    tri_decode_g(blockIdx.x, bi, bj);
    const int c = blockIdx.y;
    const int i0 = bi * GT, j0 = bj * GT;
    const long NB = (long)N * (N + 1) / 2;
    const float2 *Rc = R + (long)c * NB;
    const float2 *Vc = V + (long)c * NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < GT) {
        gi_s[tid] = (i0 + tid < N) ? g[i0 + tid] : make_float2(0.f, 0.f);
        gj_s[tid] = (j0 + tid < N) ? g[j0 + tid] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // lane owns tile columns jj = lane and lane + 32: its g_j, and the column
    // sums of the rows its warp walks, stay in registers
    const float2 gj[2] = {gj_s[lane], gj_s[lane + 32]};
    float2 col[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float loss = 0.f;
    // the warp's 8 rows (ii = warp + 8k): all 32 loads first, then the
    // arithmetic; elements outside the triangle load as zero, so E = 0 there
    // and they add nothing
    float2 rr[8][2], vv[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = i0 + warp + 8 * k;
        const long base = (long)i * (i + 1) / 2;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + lane + 32 * h;
            const bool in = i < N && j <= i;
            rr[k][h] = in ? __ldg(Rc + base + j) : make_float2(0.f, 0.f);
            vv[k][h] = in ? __ldg(Vc + base + j) : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int ii = warp + 8 * k, i = i0 + ii;
        const float2 gi = gi_s[ii];
        float2 rowsum = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + lane + 32 * h;
            const float2 r = rr[k][h], v = vv[k][h];
            const float2 m = cmulf(cmulf(gi, r), conjf2(gj[h]));
            const float2 e = make_float2(m.x - v.x, m.y - v.y);
            const float w = (i == j) ? 1.f : 2.f;
            loss = fmaf(w, e.x * e.x + e.y * e.y, loss);
            if (grad) {
                const float2 t = cmulf(cmulf(e, conjf2(r)), gj[h]);
                rowsum.x += t.x;
                rowsum.y += t.y;
                if (i != j) {
                    const float2 u = cmulf(cmulf(conjf2(e), r), gi);
                    col[h].x += u.x;
                    col[h].y += u.y;
                }
            }
        }
        if (grad) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                rowsum.x += __shfl_xor_sync(0xffffffffu, rowsum.x, o);
                rowsum.y += __shfl_xor_sync(0xffffffffu, rowsum.y, o);
            }
            if (lane == 0 && i < N) atomicAdd(&grad[i], make_float2(4.f * rowsum.x, 4.f * rowsum.y));
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) red[warp] = loss;
    if (grad) {
        colred[warp][lane] = col[0];
        colred[warp][lane + 32] = col[1];
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        partials[(long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
    if (grad && tid < GT && j0 + tid < N) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            v.x += colred[w][tid].x;
            v.y += colred[w][tid].y;
        }
        if (v.x != 0.f || v.y != 0.f) atomicAdd(&grad[j0 + tid], make_float2(4.f * v.x, 4.f * v.y));
    }
}

// Fixed-order pairwise reduction of the partials into *loss.
__global__ void __launch_bounds__(1024) k_reduce(const float *__restrict__ part, long long n, float *loss)
{
    __shared__ float s[1024];
    float acc = 0.f;
    for (long long k = threadIdx.x; k < n; k += 1024) acc += part[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w >= 1; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s[0];
}

}  // namespace

long long gain_partials_needed(int N, int C)
{
    // 64-bit throughout: for millions of inputs the tile count alone passes 2^31
    const long long nt = ((long long)N + GT - 1) / GT;
    return nt * (nt + 1) / 2 * (long long)C;
}

cudaError_t launch_gain(const float2 *R, const float2 *V, const float2 *g, int N, int C,
                        float *loss, float2 *grad, float *partials, long long n_partials_cap,
                        cudaStream_t s)
{
    const long long nt = ((long long)N + GT - 1) / GT;
    const long long tiles = nt * (nt + 1) / 2;
    // grid x holds the tiles of one channel, grid y the channels
    if (N < 1 || C < 1 || C > 65535 || tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (tiles * C > n_partials_cap) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (grad) {
        e = cudaMemsetAsync(grad, 0, sizeof(float2) * N, s);
        if (e != cudaSuccess) return e;
    }
    k_gain<<<dim3((unsigned)tiles, (unsigned)C), 256, 0, s>>>(R, V, g, N, partials, grad);
    g_launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (loss) {
        k_reduce<<<1, 1024, 0, s>>>(partials, tiles * C, loss);
        g_launches++;
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace acf

// ---------------------------------------------------------------------------
// Allocation-free variant of acf_gain_forward for callers that cannot call
// cudaMalloc while they run: processes whose device memory is reserved up
// front, real-time loops that must not block in the allocator, and plug-ins of
// a framework that owns every allocation.  The loss partials live in a fixed
// array in this library's device image instead of a buffer the library
// allocates.  Every GPU that loads the library holds the array
// (kGainStaticPartials floats) until the process exits.
// ---------------------------------------------------------------------------
namespace acf {
namespace {
constexpr int kGainStaticPartials = 65536;          // 256 KiB of loss partials
static __device__ __align__(256) float g_gain_static_partials[kGainStaticPartials];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
float *g_static_ptr[kMaxDevices] = {nullptr};        // device address per device, set once

// Device address of the static array for the current device, looked up on the
// first call on that device and kept.  Host code may not use the symbol itself
// (it is a host-side stand-in, not a device pointer).  cudaDeviceReset unloads
// the module, so an address kept from before a reset would be stale: the
// entry point's contract forbids resetting the device between calls.
cudaError_t static_partials(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gain_static_partials);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}
}  // namespace
}  // namespace acf

extern "C" acf_status acf_gain_forward_noalloc(const void *R, const void *V, const void *g, int n_inputs,
                                               int n_channels, float *loss, void *grad, acf_stream_t stream)
{
    using namespace acf;
    if (!R || !V || !g || n_inputs < 1 || n_channels < 1 || n_channels > 65535 || (!loss && !grad))
        return ACF_EINVAL;
    // checked before any CUDA call: a size beyond the fixed scratch never launches
    const long long need = gain_partials_needed(n_inputs, n_channels);
    if (need > kGainStaticPartials) return ACF_EINVAL;
    float *part = nullptr;
    if (static_partials(&part) != cudaSuccess) return ACF_ECUDA;
    cudaError_t e = launch_gain(static_cast<const float2 *>(R), static_cast<const float2 *>(V),
                                static_cast<const float2 *>(g), n_inputs, n_channels, loss,
                                static_cast<float2 *>(grad), part, kGainStaticPartials, (cudaStream_t)stream);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

