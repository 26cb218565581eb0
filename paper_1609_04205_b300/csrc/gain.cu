// Gain-corrupted correlation M = G R G^H, its squared-Frobenius loss against
// observed visibilities and the adjoint (gradient) with respect to the
// per-input complex gains -- the calibration-facing form of the correlator
// output (Sec. 5 fits per-dipole gains to the visibilities).
//
// Per element of the packed lower triangles of channel c:
//   E_ij = w_ij R_ij - V_ij,   w_ij = g_i conj(g_j),
//   loss += s_ij |E_ij|^2      (s = 2 off the diagonal: the upper triangle is
//                               the conjugate, 1 on it),
//   grad_i += 4 z_ij g_j        and, for i != j,  grad_j += 4 conj(z_ij) g_i,
// with z_ij = E_ij conj(R_ij) (conj(z_ij) g_i = conj(E_ij) R_ij g_i is the
// upper-triangle term E_ji conj(R_ji) g_i).  The gradient terms are linear in
// z, so a block that covers the same tile for several channels sums z over
// them and multiplies by g once: per element and channel that leaves w R,
// the residual, |E|^2 and z.
//
// A block owns a 16-row x 64-column tile for KCH = 8 consecutive channels
// (lane: two columns; warp: two rows), computes w_ij once, keeps the loads of
// two channels in flight ahead of the arithmetic, then reduces: row sums by
// a warp butterfly over the four (row, re/im) values, column sums across the
// warps in shared memory, one global atomic per tile row and column.  Each
// block writes one loss partial; a single-block kernel adds them in a fixed
// order, so the loss is deterministic.  The zeroing of grad before, and the
// loss reduction after, overlap k_gain through programmatic dependent launch,
// so the three launches cost little more than k_gain alone.
#include <mutex>

#include "acf_internal.h"

namespace acf {
namespace {

constexpr int KCH = 8;            // channels per block
constexpr int TR = 16, TC = 64;   // tile rows, columns

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while the kernel before it runs;
// dep_wait() returns once that kernel has completed and its writes are
// visible, dep_release() lets the next kernel start early.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Tile k -> (row block, column block).  Super-row sr (64 rows) holds four
// row blocks of sr + 1 column blocks each, so 2 sr (sr + 1) tiles precede it.
__device__ __forceinline__ void tile_decode(int k, int &rb, int &cb) {
    int sr = (int)((sqrtf(2.f * (float)k + 1.f) - 1.f) * 0.5f);
    while (2 * (sr + 1) * (sr + 2) <= k) ++sr;
    while (sr > 0 && 2 * sr * (sr + 1) > k) --sr;
    const int rem = k - 2 * sr * (sr + 1);
    rb = 4 * sr + rem / (sr + 1);
    cb = rem % (sr + 1);
}

__global__ void __launch_bounds__(256, 2)
k_gain(const float2 *__restrict__ R, const float2 *__restrict__ V, const float2 *__restrict__ g,
       int N, int C, float *__restrict__ partials, float2 *__restrict__ grad)
{
    __shared__ float2 colred[8][TC];
    __shared__ float red[8];
    int rb, cb;
    tile_decode(blockIdx.x, rb, cb);
    const int i0 = TR * rb, j0 = TC * cb;
    const long NB = (long)N * (N + 1) / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.y * KCH, nc = min(KCH, C - c0);

    // the thread's 2 x 2 elements: rows i0 + 2 warp + a, columns j0 + lane + 32 b
    int ii[2], jj[2], off[2][2];
    float2 gi[2], gj[2], w[2][2], zacc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        ii[a] = i0 + 2 * warp + a;
        jj[a] = j0 + lane + 32 * a;
        gi[a] = ii[a] < N ? __ldg(g + ii[a]) : make_float2(0.f, 0.f);
        gj[a] = jj[a] < N ? __ldg(g + jj[a]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const bool in = ii[a] < N && jj[b] <= ii[a];    // outside: zeros, adding nothing
            off[a][b] = in ? (int)((long)ii[a] * (ii[a] + 1) / 2 + jj[b]) : -1;
            w[a][b] = in ? cmulf(gi[a], conjf2(gj[b])) : make_float2(0.f, 0.f);
            zacc[a][b] = make_float2(0.f, 0.f);
        }
    const float2 *Rb = R + (long)c0 * NB, *Vb = V + (long)c0 * NB;
    float loss = 0.f;
    auto load = [&](float2 (&r)[2][2], float2 (&v)[2][2], int cc) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int o = cc < nc ? off[a][b] : -1;
                r[a][b] = o >= 0 ? __ldcs(Rb + (long)cc * NB + o) : make_float2(0.f, 0.f);
                v[a][b] = o >= 0 ? __ldcs(Vb + (long)cc * NB + o) : make_float2(0.f, 0.f);
            }
    };
    auto accumulate = [&](const float2 (&r)[2][2], const float2 (&v)[2][2]) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float2 m = cmulf(w[a][b], r[a][b]);
                const float2 e = make_float2(m.x - v[a][b].x, m.y - v[a][b].y);
                const float s = ii[a] == jj[b] ? 1.f : 2.f;
                loss = fmaf(s, fmaf(e.x, e.x, e.y * e.y), loss);
                const float2 z = cmulf(e, conjf2(r[a][b]));
                zacc[a][b].x += z.x;
                zacc[a][b].y += z.y;
            }
    };
    // two channels in flight ahead of the arithmetic (three rotating buffers)
    float2 rbuf[3][2][2], vbuf[3][2][2];
#pragma unroll
    for (int k = 0; k < 3 && k < KCH; ++k) load(rbuf[k], vbuf[k], k);
#pragma unroll
    for (int cc = 0; cc < KCH; ++cc) {
        accumulate(rbuf[cc % 3], vbuf[cc % 3]);
        if (cc + 3 < KCH) load(rbuf[cc % 3], vbuf[cc % 3], cc + 3);
    }

    // grad was zeroed by the kernel before this one, which may still be running
    dep_wait();
    dep_release();
    // row sums z g_j: the lane's two columns, then the warp's four (row, re/im)
    // values by a butterfly that halves the set per step; afterwards lanes
    // 8q .. 8q + 7 hold value q = 2 (row) + (re/im)
    float rs[4];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float2 t0 = cmulf(zacc[a][0], gj[0]), t1 = cmulf(zacc[a][1], gj[1]);
        rs[2 * a] = t0.x + t1.x;
        rs[2 * a + 1] = t0.y + t1.y;
    }
    {
        const bool up16 = lane & 16;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float snd = up16 ? rs[q] : rs[q + 2], kp = up16 ? rs[q + 2] : rs[q];
            rs[q] = kp + __shfl_xor_sync(0xffffffffu, snd, 16);
        }
        const bool up8 = lane & 8;
        const float snd = up8 ? rs[0] : rs[1], kp = up8 ? rs[1] : rs[0];
        rs[0] = kp + __shfl_xor_sync(0xffffffffu, snd, 8);
        rs[0] += __shfl_xor_sync(0xffffffffu, rs[0], 4);
        rs[0] += __shfl_xor_sync(0xffffffffu, rs[0], 2);
        rs[0] += __shfl_xor_sync(0xffffffffu, rs[0], 1);
        if ((lane & 7) == 0) {
            const int q = lane >> 3, a = q >> 1;
            if (grad && ii[a] < N && rs[0] != 0.f) atomicAdd(reinterpret_cast<float *>(grad + ii[a]) + (q & 1), 4.f * rs[0]);
        }
    }
    // column sums conj(z) g_i over the thread's two rows, diagonal excluded
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        float2 cs = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float2 u = cmulf(conjf2(zacc[a][b]), gi[a]);
            if (ii[a] != jj[b]) {
                cs.x += u.x;
                cs.y += u.y;
            }
        }
        colred[warp][lane + 32 * b] = cs;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) red[warp] = loss;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int q = 0; q < 8; ++q) s += red[q];
        partials[(long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
    if (grad && tid < TC && j0 + tid < N) {
        float2 cs = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            cs.x += colred[q][tid].x;
            cs.y += colred[q][tid].y;
        }
        if (cs.x != 0.f || cs.y != 0.f) atomicAdd(&grad[j0 + tid], make_float2(4.f * cs.x, 4.f * cs.y));
    }
}

// Zeroes grad ahead of k_gain's atomics, letting k_gain start at once.
__global__ void k_zero(float2 *__restrict__ grad, int N)
{
    dep_release();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
        grad[k] = make_float2(0.f, 0.f);
}

// Fixed-order reduction of the partials into *loss: each thread adds a fixed
// strided subset (four loads in flight), then warp butterflies and one warp
// over the warp sums.  Launched to overlap k_gain; reads after it completes.
__global__ void __launch_bounds__(1024) k_reduce(const float *__restrict__ part, long long n, float *loss)
{
    __shared__ float ws[32];
    dep_wait();
    float acc = 0.f;
#pragma unroll 4
    for (long long k = threadIdx.x; k < n; k += 1024) acc += part[k];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = ws[threadIdx.x];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *loss = acc;
    }
}

long long n_tiles(int N)
{
    const long long nsr = ((long long)N + 63) / 64;
    return 2 * nsr * (nsr + 1);
}

}  // namespace

long long gain_partials_needed(int N, int C)
{
    // 64-bit throughout: for millions of inputs the tile count alone passes 2^31
    return n_tiles(N) * (((long long)C + KCH - 1) / KCH);
}

cudaError_t launch_gain(const float2 *R, const float2 *V, const float2 *g, int N, int C,
                        float *loss, float2 *grad, float *partials, long long n_partials_cap,
                        cudaStream_t s)
{
    const long long tiles = n_tiles(N);
    const long long groups = ((long long)C + KCH - 1) / KCH;
    // grid x holds the tiles of the triangle, grid y the channel groups; the
    // element offsets within a channel are 32-bit
    if (N < 1 || C < 1 || C > 65535 || tiles > 0x7fffffffLL || (long long)N * (N + 1) / 2 > 0x7fffffffLL)
        return cudaErrorInvalidValue;
    if (tiles * groups > n_partials_cap) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    if (grad) {
        // grad is accumulated with atomics: k_zero clears it and k_gain, which
        // reads only R, V and g before its dep_wait(), overlaps k_zero.  k_zero
        // itself starts after all earlier work on the stream.
        k_zero<<<(N + 255) / 256 < 64 ? (N + 255) / 256 : 64, 256, 0, s>>>(grad, N);
        g_launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tiles, (unsigned)groups);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cfg.attrs = pdl;
    cfg.numAttrs = grad ? 1 : 0;     // without k_zero, k_gain waits for the earlier work in full
    e = cudaLaunchKernelEx(&cfg, k_gain, R, V, g, N, C, partials, grad);
    g_launches++;
    if (e != cudaSuccess) return e;
    if (loss) {
        cudaLaunchConfig_t rc = {};
        rc.gridDim = dim3(1);
        rc.blockDim = dim3(1024);
        rc.stream = s;
        rc.attrs = pdl;
        rc.numAttrs = 1;
        e = cudaLaunchKernelEx(&rc, k_reduce, (const float *)partials, tiles * groups, loss);
        g_launches++;
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

