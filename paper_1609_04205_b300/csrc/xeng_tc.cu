// Tensor-core X-engine for sm_103a (Sec. 4.2.5 on 5th-generation tensor cores).
//
// The complex rank-k update V = sum_t x_t x_t^H is computed as one REAL
// product D = Y Y^T, where Y holds each complex input as two real rows
// (2n = Re x_n, 2n+1 = Im x_n) with time along the row.  Every 2x2 block of D
// gives one visibility:
//     Re V_ij = D[2i][2j] + D[2i+1][2j+1],   Im V_ij = D[2i+1][2j] - D[2i][2j+1].
// No negated or swapped operand copy is needed and the work equals the
// complex product's 4 real MACs per baseline and sample.  Only tiles that
// touch the lower triangle (i >= j) are computed; the epilogue masks the rest.
//
// Kernel structure (one persistent CTA per SM, 10 warps):
//   warp 0     TMA producer: 64-sample K steps of a 128-row A tile and an
//              NT-row B tile (SW128, K-major) into a ring of four 48 KB slots;
//   warp 1     owns the TMEM allocation (2 x 256 fp32 columns = two
//              accumulators) and one lane issues tcgen05.mma (M=128, N=NT,
//              K=16, fp16 x fp16 -> fp32), committing each slot back to the
//              producer and each finished chunk to the epilogue;
//   warps 2-9  epilogue: tcgen05.ld the finished accumulator chunk, fold it
//              into per-thread register masters (fp32, or int32 for the exact
//              mode), and at the end of a work item combine the 2x2 blocks
//              and store (or, when a tile has several writers, atomically
//              add) the visibilities into the packed triangle.
// Modes: FP16 (one product per K step), FP16x3 (hi*hi + hi*lo + lo*hi, the
// lo operands in a second slot), INT8 (fp16 holding integers |x| <= 127:
// products are exact and each 512-sample chunk sum stays below 2^24, so the
// fp32 tensor-core accumulation is exact; chunks are folded into int32
// masters and work items never exceed 32,768 samples, so the masters stay
// below 2^29 and their 2x2 combine below 2^31; the output is int64).
// Every mbarrier wait is bounded; on timeout the CTA records an error word,
// drains its own TMA copies and MMAs, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "acf_internal.h"

namespace acf {
namespace {

constexpr int kMaxJobs = 64;
constexpr int kSlots = 4;
constexpr int kSlotBytes = 48 * 1024;          // A 16 KB + B up to 32 KB
constexpr int kSlots2 = 6;                      // two-SM kernel: ring slots per CTA
constexpr int kSlotBytes2 = 32 * 1024;          // own 128 A rows + own 128 B rows
constexpr int kBM = 128, kBK = 64;
constexpr int kThreadsTc = 320;
constexpr int kEpiWarps = 8;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitLimit = 1LL << 22;   // drain waits: polls x 256 ns back-off, about one second
constexpr long long kWaitCycles = 1LL << 31;  // pipeline waits: about one second of SM clock
// INT8 work items span at most 2^15 samples: int32 register sums of |x| <= 128
// products stay below 2^29, so masters and their 2x2 combine are exact.
constexpr long kInt8ItemMax = 32768;

struct JobDev {
    void *V;
    int N, n_problems, mode, nt;
    long n_time;
    int k_split, tiles_pp, mb, item_begin;
    float vscale;
    int store;            // 1: each visibility written once with plain stores; 0: atomically added
    const float2 *rot;    // delay compensation a[p][i] (V_ij *= a_i conj(a_j)), or nullptr
};

struct TcParams {
    CUtensorMap maps[kMaxJobs][2];
    JobDev jobs[kMaxJobs];
    int n_jobs;
    int n_items;
    int *err;
    const int *perm;      // work position -> item (interleaved order), or nullptr
};

struct Item {
    int job, p, bi, bj;
    long k0, k1;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about 20 us pass, instead of returning at once and
// spinning on issue slots the other roles need (A-12 X-engine 6% faster,
// A-6 INT8 step 4%).
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false on abort/timeout.  It
// polls the hinted try_wait without software sleeps, so a waiter resumes as
// soon as its data lands; every 256 polls (at most about 5 ms) it checks the
// CTA's abort flag and a clock-based limit of kWaitCycles (~1 s).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          int *err, int code) {
    if (mbar_try_wait_hint(bar, parity)) return true;
    const long long t0 = clock64();
    for (int it = 1;; ++it) {
        if (mbar_try_wait_hint(bar, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitCycles) {
                *abort_flag = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)(16u >> 4) << 16;                  // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                // SBO: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}

__device__ __forceinline__ uint32_t idesc_f16(int nt) {
    // D fp32, A/B fp16, both K-major, N = nt, M = 128
    return (1u << 4) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mma_f16_pair(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
                 "h"((uint16_t)0x3)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Lower-triangle tiles of one problem, bj-major: tile count and decode.
__host__ __device__ __forceinline__ int bi_min(int bj, int nt) {
    const int v = (nt / 2) * bj - 63;
    return v <= 0 ? 0 : (v + 63) / 64;
}
__host__ __device__ inline int tiles_per_problem(int N, int nt) {
    const int mb = (2 * N + kBM - 1) / kBM;
    const int nb = (2 * N + nt - 1) / nt;
    int t = 0;
    for (int bj = 0; bj < nb; ++bj) t += max(0, mb - bi_min(bj, nt));
    return t;
}

// PERM: the work position is mapped through the plan's interleaved order (a
// separate instantiation, so the plain order's kernels carry no extra load).
template <bool PERM>
__device__ __forceinline__ bool decode_item(const TcParams &P, int item, Item &it) {
    if (PERM) item = __ldg(P.perm + item);
    int j = 0;
    while (j + 1 < P.n_jobs && item >= P.jobs[j + 1].item_begin) ++j;
    const JobDev &J = P.jobs[j];
    int local = item - J.item_begin;
    const int per_p = J.tiles_pp * J.k_split;
    it.job = j;
    it.p = local / per_p;
    int rem = local - it.p * per_p;
    int tile = rem / J.k_split;
    const int s = rem - tile * J.k_split;
    int bj = 0;
    for (;; ++bj) {
        const int cnt = J.mb - bi_min(bj, J.nt);
        if (tile < cnt) break;
        tile -= cnt;
    }
    it.bj = bj;
    it.bi = bi_min(bj, J.nt) + tile;
    const long K64 = (J.n_time + 63) / 64 * 64;
    const long per = ((K64 + J.k_split - 1) / J.k_split + 63) / 64 * 64;
    it.k0 = (long)s * per;
    it.k1 = min(K64, it.k0 + per);
    return it.k0 < it.k1;
}

// The TMEM accumulator is drained into register sums every few K steps.  INT8
// needs 512-sample chunks for exactness (partial sums < 2^23).  The tensor
// core's fp32 accumulation rounds toward zero, so short chunks folded into
// round-to-nearest register sums bound the float modes' bias: 512 samples
// (32 MMAs, <= 2^-18 relative) for split FP16, 1024 samples (<= 2^-17) for
// plain FP16, whose operand rounding (2^-11) dominates anyway.
__device__ __forceinline__ int chunk_steps(int mode) { return mode == ACF_X_FP16 ? 16 : 8; }
// ---------------------------------------------------------------------------
// MMA issue for the K steps [s0, s1) of one accumulator chunk.  SPK is the
// number of ring slots per K step (1: one fp16 operand; 2: split FP16 hi and
// lo, issuing hi*hi, hi*lo and lo*hi).  The count is a template parameter so
// that the slot indices stay in registers and the unrolled issue sequence has
// no branches: a runtime count with the split-FP16 MMAs behind a branch inside
// the K loop ran the whole X-engine ~1.7x slower in FP16 mode.  PAIR selects
// the two-SM form (cta_group::2 MMAs and multicast commits, issued by the
// leader CTA).  Returns false when a wait gave up (abort or timeout).
template <int SPK, bool PAIR>
__device__ __forceinline__ bool issue_steps(uint32_t ring, uint64_t *full_bar, uint64_t *empty_bar, long &pos, long s0,
                                            long s1, uint32_t dt, uint32_t idesc, volatile int *abort_flag, int *err)
{
    constexpr int kRing = PAIR ? kSlots2 : kSlots;
    constexpr uint32_t kStride = PAIR ? kSlotBytes2 : kSlotBytes;
    for (long s = s0; s < s1; ++s) {
        int slot[SPK];
#pragma unroll
        for (int h = 0; h < SPK; ++h) {
            slot[h] = (int)(pos % kRing);
            if (!mbar_wait(smem_u32(&full_bar[slot[h]]), (uint32_t)((pos / kRing) & 1), abort_flag, err, PAIR ? 13 : 3))
                return false;
            ++pos;
        }
        tc_fence_after();
        const uint32_t a_hi = ring + (uint32_t)slot[0] * kStride;
        const uint64_t dah = desc_sw128(a_hi), dbh = desc_sw128(a_hi + kBM * kBK * 2);
        uint64_t dal = 0, dbl = 0;
        if constexpr (SPK == 2) {
            const uint32_t a_lo = ring + (uint32_t)slot[1] * kStride;
            dal = desc_sw128(a_lo);
            dbl = desc_sw128(a_lo + kBM * kBK * 2);
        }
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint32_t acc = (s > s0 || kk > 0) ? 1u : 0u;
            if constexpr (PAIR) {
                mma_f16_pair(dt, dah + 2 * kk, dbh + 2 * kk, idesc, acc);
                if constexpr (SPK == 2) {
                    mma_f16_pair(dt, dah + 2 * kk, dbl + 2 * kk, idesc, 1u);
                    mma_f16_pair(dt, dal + 2 * kk, dbh + 2 * kk, idesc, 1u);
                }
            } else {
                mma_f16(dt, dah + 2 * kk, dbh + 2 * kk, idesc, acc);
                if constexpr (SPK == 2) {
                    mma_f16(dt, dah + 2 * kk, dbl + 2 * kk, idesc, 1u);
                    mma_f16(dt, dal + 2 * kk, dbh + 2 * kk, idesc, 1u);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < SPK; ++h) {
            if constexpr (PAIR) mma_commit_pair(smem_u32(&empty_bar[slot[h]]));
            else mma_commit(smem_u32(&empty_bar[slot[h]]));
        }
    }
    return true;
}

// Flush one epilogue thread's register sums of a finished tile: combine each
// 2x2 real block into a complex visibility (in place: afterwards m[2k], m[2k+1]
// hold Re, Im of V[i][jbase + k]) and write the lane's run of up to 32
// consecutive visibilities of row i with 16-byte stores (or atomics).
__device__ __forceinline__ void flush_tile(const JobDev &J, int p, int i, int jbase, int odd, bool exact,
                                           uint32_t (&m)[128])
{
    // flush: combine 2x2 real blocks into complex visibilities, in place:
    // after iteration k, m[2k], m[2k+1] hold (Re, Im) of V[i][jbase + k]
    const long NB = (long)J.N * (J.N + 1) / 2;
    const long prow = (long)p * NB + (long)i * (i + 1) / 2;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const uint32_t s0v = odd ? m[2 * k] : m[64 + 2 * k];
        const uint32_t s1v = odd ? m[2 * k + 1] : m[65 + 2 * k];
        const uint32_t r0 = __shfl_xor_sync(0xffffffffu, s0v, 1);
        const uint32_t r1 = __shfl_xor_sync(0xffffffffu, s1v, 1);
        const uint32_t own0 = odd ? m[64 + 2 * k] : m[2 * k];
        const uint32_t own1 = odd ? m[65 + 2 * k] : m[2 * k + 1];
        // even lane: a = own0, b = own1, c = r0, d = r1; odd lane: c, d own, a, b received
        const uint32_t a = odd ? r0 : own0, bq = odd ? r1 : own1;
        const uint32_t c = odd ? own0 : r0, d = odd ? own1 : r1;
        if (exact) {
            // exact in int32: items span <= 32,768 samples, so |D| <= 128^2 * 2^15 = 2^29
            m[2 * k] = (uint32_t)((int)a + (int)d);
            m[2 * k + 1] = (uint32_t)((int)c - (int)bq);
        } else {
            m[2 * k] = __float_as_uint((__uint_as_float(a) + __uint_as_float(d)) * J.vscale);
            m[2 * k + 1] = __float_as_uint((__uint_as_float(c) - __uint_as_float(bq)) * J.vscale);
        }
    }
    // valid run of this lane: j in [jbase, min(jbase + 32, i + 1)), row i < N
    const int nval = (i < J.N) ? max(0, min(32, i + 1 - jbase)) : 0;
    if (!exact && J.rot && nval > 0) {
        // delay compensation (Sec. 4.2.4) folded into the flush: V_ij *= a_i conj(a_j)
        const float2 *ap = J.rot + (long)p * J.N;
        const float2 ai = __ldg(ap + i);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (k < nval) {
                const float2 aj = __ldg(ap + jbase + k);
                const float wr = ai.x * aj.x + ai.y * aj.y, wi = ai.y * aj.x - ai.x * aj.y;
                const float vr = __uint_as_float(m[2 * k]), vi = __uint_as_float(m[2 * k + 1]);
                m[2 * k] = __float_as_uint(vr * wr - vi * wi);
                m[2 * k + 1] = __float_as_uint(vr * wi + vi * wr);
            }
        }
    }
    if (nval > 0) {
        if (exact) {
            long long *dst = static_cast<long long *>(J.V) + 2 * (prow + jbase);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                if (k < nval) {
                    const long long re = (int)m[2 * k], im = (int)m[2 * k + 1];
                    if (J.store) {
                        *reinterpret_cast<longlong2 *>(dst + 2 * k) = make_longlong2(re, im);
                    } else {
                        atomicAdd(reinterpret_cast<unsigned long long *>(dst + 2 * k), (unsigned long long)re);
                        atomicAdd(reinterpret_cast<unsigned long long *>(dst + 2 * k + 1), (unsigned long long)im);
                    }
                }
            }
        } else if (J.store && nval == 32) {
            // a whole run (every tile off the diagonal): 16-byte stores, with a
            // single at each end when the run starts at an odd element
            float2 *dst = static_cast<float2 *>(J.V) + (prow + jbase);
            const auto mf = [&](int k) { return __uint_as_float(m[k]); };
            if (((prow + jbase) & 1) == 0) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    *reinterpret_cast<float4 *>(dst + 2 * k) = make_float4(mf(4 * k), mf(4 * k + 1), mf(4 * k + 2), mf(4 * k + 3));
            } else {
                dst[0] = make_float2(mf(0), mf(1));
#pragma unroll
                for (int k = 0; k < 15; ++k)
                    *reinterpret_cast<float4 *>(dst + 2 * k + 1) =
                        make_float4(mf(4 * k + 2), mf(4 * k + 3), mf(4 * k + 4), mf(4 * k + 5));
                dst[31] = make_float2(mf(62), mf(63));
            }
        } else {
            float2 *dst = static_cast<float2 *>(J.V) + (prow + jbase);
            // pair elements on 16-byte boundaries: a leading single when the run starts odd
            const int lead = (int)((prow + jbase) & 1);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float2 v0 = make_float2(__uint_as_float(m[2 * k]), __uint_as_float(m[2 * k + 1]));
                const bool single = (k == 0 && lead) || (k + 1 == nval && ((k - lead) & 1) == 0);
                const bool pair_start = !single && ((k - lead) & 1) == 0 && k + 1 < nval;
                if (k < nval && single) {
                    if (J.store) dst[k] = v0;
                    else atomicAdd(dst + k, v0);
                } else if (k < 31 && k < nval && pair_start) {
                    const float4 v = make_float4(v0.x, v0.y, __uint_as_float(m[2 * k + 2]), __uint_as_float(m[2 * k + 3]));
                    if (J.store) *reinterpret_cast<float4 *>(dst + k) = v;
                    else atomicAdd(reinterpret_cast<float4 *>(dst + k), v);
                }
            }
        }
    }
}

template <bool PERM>
__global__ void __launch_bounds__(kThreadsTc, 1) k_xeng_tc(const __grid_constant__ TcParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the SW128 tiles
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[kSlots], empty_bar[kSlots], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            for (int j = 0; j < P.n_jobs; ++j) {
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.maps[j][0])) : "memory");
            }
            long pos = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
                Item it;
                if (!decode_item<PERM>(P, item, it)) continue;
                const JobDev &J = P.jobs[it.job];
                const int spk = J.mode == ACF_X_FP16x3 ? 2 : 1;
                const int rowA = it.p * 2 * J.N + it.bi * kBM;
                const int rowB = it.p * 2 * J.N + it.bj * J.nt;
                const uint32_t bytes = (uint32_t)(kBM + J.nt) * kBK * 2;
                for (long k = it.k0; k < it.k1 && ok; k += kBK) {
                    for (int h = 0; h < spk && ok; ++h) {
                        const int slot = (int)(pos % kSlots);
                        const uint32_t ph = (uint32_t)((pos / kSlots) & 1);
                        ok = mbar_wait(smem_u32(&empty_bar[slot]), ph ^ 1, &abort_flag, P.err, 1);
                        if (!ok) break;
                        const uint32_t fb = smem_u32(&full_bar[slot]);
                        mbar_expect_tx(fb, bytes);
                        const uint32_t base = smem_u32(smem + slot * kSlotBytes);
                        const CUtensorMap *map = &P.maps[it.job][h];
                        tma_load_2d(base, map, fb, (int)k, rowA);
                        for (int q = 0; q < J.nt / kBM; ++q)
                            tma_load_2d(base + (kBM + q * kBM) * kBK * 2, map, fb, (int)k, rowB + q * kBM);
                        ++pos;
                    }
                }
            }
            if (!ok) {
                // drain our own copies still in flight before the CTA exits
                for (long q = pos - 1; q >= 0 && q >= pos - kSlots; --q) {
                    const int slot = (int)(q % kSlots);
                    for (long long it = 0; it < kWaitLimit && !mbar_try_wait(smem_u32(&full_bar[slot]), (uint32_t)((q / kSlots) & 1)); ++it)
                        __nanosleep(256);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            long pos = 0, cc = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
                Item it;
                if (!decode_item<PERM>(P, item, it)) continue;
                const JobDev &J = P.jobs[it.job];
                const int spk = J.mode == ACF_X_FP16x3 ? 2 : 1;
                const uint32_t idesc = idesc_f16(J.nt);
                const uint32_t ring = smem_u32(smem);
                const long steps = (it.k1 - it.k0) / kBK;
                const long csteps = chunk_steps(J.mode);
                for (long s0 = 0; s0 < steps && ok; s0 += csteps) {
                    const int b = (int)(cc & 1);
                    ok = mbar_wait(smem_u32(&acce_bar[b]), (uint32_t)(((cc >> 1) & 1) ^ 1), &abort_flag, P.err, 2);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)(b * 256);
                    const long s1 = min(steps, s0 + csteps);
                    ok = spk == 2 ? issue_steps<2, false>(ring, full_bar, empty_bar, pos, s0, s1, dt, idesc, &abort_flag, P.err)
                                  : issue_steps<1, false>(ring, full_bar, empty_bar, pos, s0, s1, dt, idesc, &abort_flag, P.err);
                    if (!ok) break;
                    mma_commit(smem_u32(&accf_bar[b]));
                    ++cc;
                }
            }
            // all MMAs issued by this thread complete before TMEM is released
            mma_commit(smem_u32(&done_bar));
            for (long long it = 0; it < kWaitLimit && !mbar_try_wait(smem_u32(&done_bar), 0); ++it) __nanosleep(256);
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int q = warp & 3;                 // TMEM lane quadrant
        const int half = (warp - 2) >> 2;       // column half
        const int odd = lane & 1;
        uint32_t m[128];
#pragma unroll
        for (int k = 0; k < 128; ++k) m[k] = 0u;
        long cc = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < P.n_items && ok; item += gridDim.x) {
            Item it;
            if (!decode_item<PERM>(P, item, it)) continue;
            const JobDev &J = P.jobs[it.job];
            const bool exact = J.mode == ACF_X_INT8;
            const bool active = half * 128 < J.nt;
            const long steps = (it.k1 - it.k0) / kBK;
            const long csteps = chunk_steps(J.mode);
            for (long s0 = 0; s0 < steps; s0 += csteps) {
                const int b = (int)(cc & 1);
                // one lane waits; the warp follows its verdict (keeps .sync.aligned loads converged)
                int w_ok = 0;
                if (lane == 0) w_ok = mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)((cc >> 1) & 1), &abort_flag, P.err, 4);
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                if (active) {
                    const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 256 + half * 128);
#pragma unroll
                    for (int piece = 0; piece < 4; ++piece) {
                        uint32_t r[32];
                        tmem_ld32(tbase + piece * 32, r);
                        tmem_wait_ld();
                        if (exact) {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                m[piece * 32 + k] = (uint32_t)((int)m[piece * 32 + k] + __float2int_rn(__uint_as_float(r[k])));
                        } else {
#pragma unroll
                            for (int k = 0; k < 32; ++k)
                                m[piece * 32 + k] = __float_as_uint(__uint_as_float(m[piece * 32 + k]) + __uint_as_float(r[k]));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acce_bar[b]));
                ++cc;
            }
            if (!ok) break;
            if (!active) continue;
            flush_tile(J, it.p, it.bi * 64 + 16 * q + (lane >> 1), (J.nt * it.bj + 128 * half) / 2 + 32 * odd, odd,
                       exact, m);
#pragma unroll
            for (int k = 0; k < 128; ++k) m[k] = 0u;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Two-SM variant: a cluster of two CTAs computes one 256x256 real tile with
// tcgen05.mma.cta_group::2 (M = 256 split across the pair, N = 256 split in the
// operand load).  Each CTA loads only its 128 A rows and its 128 B rows per K
// step (32 KB instead of 48 KB), so six slots fit in shared memory and each SM
// lands a third fewer operand bytes per MMA.  CTA rank 0 (the leader) issues
// the MMAs; both CTAs' TMA loads complete on the leader's slot barrier, and the
// leader's commits are multicast to both CTAs' slot and accumulator barriers.
// Each CTA keeps two 256-column accumulators (its 128 rows of the tile) so the
// epilogue drains one chunk while the next accumulates; epilogue warps of both
// CTAs report a drained chunk to the leader.  The pair allocation is collective
// (both CTAs receive the same TMEM base, which the kernel checks).
// ---------------------------------------------------------------------------
constexpr uint32_t kTmemCols2 = 512;            // two 256-column accumulators per CTA
constexpr int kBM2 = 256;                       // real rows per tile side

__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Load into this CTA's shared memory, completing on the pair leader's barrier.
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ uint32_t idesc_f16_pair() {
    // D fp32, A/B fp16, both K-major, N = 256, M = 256 (across the CTA pair)
    return (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

// Square 256x256 tiles of the lower triangle, row-major in bi >= bj.
__host__ __device__ inline int sq_tiles_per_problem(int N) {
    const int nb = (2 * N + kBM2 - 1) / kBM2;
    return nb * (nb + 1) / 2;
}

template <bool PERM>
__device__ __forceinline__ bool decode_item2(const TcParams &P, int item, Item &it) {
    if (PERM) item = __ldg(P.perm + item);
    int j = 0;
    while (j + 1 < P.n_jobs && item >= P.jobs[j + 1].item_begin) ++j;
    const JobDev &J = P.jobs[j];
    int local = item - J.item_begin;
    const int per_p = J.tiles_pp * J.k_split;
    it.job = j;
    it.p = local / per_p;
    int rem = local - it.p * per_p;
    int tile = rem / J.k_split;
    const int s = rem - tile * J.k_split;
    int bi = 0;
    while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
    it.bi = bi;
    it.bj = tile - bi * (bi + 1) / 2;
    const long K64 = (J.n_time + 63) / 64 * 64;
    const long per = ((K64 + J.k_split - 1) / J.k_split + 63) / 64 * 64;
    it.k0 = (long)s * per;
    it.k1 = min(K64, it.k0 + per);
    return it.k0 < it.k1;
}

template <bool PERM>
__global__ void __launch_bounds__(kThreadsTc, 1) k_xeng_tc2(const __grid_constant__ TcParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[kSlots2], empty_bar[kSlots2], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots2; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);      // leader's: its producer's expect_tx for both CTAs' bytes
            mbar_init(smem_u32(&empty_bar[s]), 1);     // the leader's multicast commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), 2 * kEpiWarps);  // leader's: every epilogue warp of both CTAs
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(kTmemCols2)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();
    const uint32_t tmem = tmem_base_s;
    // the pair must see one accumulator address; otherwise record an error and do no work
    if (threadIdx.x == 0) {
        const uint32_t peer = ld_cluster_u32(mapa_u32(smem_u32(&tmem_base_s), rank ^ 1u));
        if (peer != tmem) {
            abort_flag = 1;
            atomicCAS(P.err, 0, 9);
        }
    }
    __syncthreads();
    const bool run = !abort_flag;
    cluster_sync();   // both CTAs decided before either starts
    const uint32_t full_leader0 = mapa_u32(smem_u32(&full_bar[0]), 0);
    const uint32_t acce_leader0 = mapa_u32(smem_u32(&acce_bar[0]), 0);

    if (!run) {
        // nothing issued: fall through to the common exit
    } else if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            for (int j = 0; j < P.n_jobs; ++j)
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.maps[j][0])) : "memory");
            long pos = 0;
            bool ok = true;
            for (int item = cid; item < P.n_items && ok; item += ncl) {
                Item it;
                if (!decode_item2<PERM>(P, item, it)) continue;
                const JobDev &J = P.jobs[it.job];
                const int spk = J.mode == ACF_X_FP16x3 ? 2 : 1;
                const int rowA = it.p * 2 * J.N + it.bi * kBM2 + (int)rank * kBM;
                const int rowB = it.p * 2 * J.N + it.bj * kBM2 + (int)rank * kBM;
                for (long k = it.k0; k < it.k1 && ok; k += kBK) {
                    for (int h = 0; h < spk && ok; ++h) {
                        const int slot = (int)(pos % kSlots2);
                        const uint32_t ph = (uint32_t)((pos / kSlots2) & 1);
                        ok = mbar_wait(smem_u32(&empty_bar[slot]), ph ^ 1, &abort_flag, P.err, 11);
                        if (!ok) break;
                        const uint32_t fb = full_leader0 + (uint32_t)(slot * sizeof(uint64_t));
                        // Only the leader arrives, locally, expecting both CTAs' bytes; the
                        // peer's copies just complete their bytes on the leader's barrier (a
                        // transaction count may run ahead of its expect_tx).  A remote
                        // release-cluster arrive per slot from the peer was slow enough to
                        // starve the MMA.
                        if (leader) mbar_expect_tx(smem_u32(&full_bar[slot]), 2u * (uint32_t)kSlotBytes2);
                        const uint32_t base = smem_u32(smem + slot * kSlotBytes2);
                        const CUtensorMap *map = &P.maps[it.job][h];
                        tma_load_2d_pair(base, map, fb, (int)k, rowA);
                        tma_load_2d_pair(base + kBM * kBK * 2, map, fb, (int)k, rowB);
                        ++pos;
                    }
                }
            }
            // before the CTA may exit: the leader's MMAs have consumed every fill
            for (long q = pos - 1; q >= 0 && q >= pos - kSlots2; --q) {
                const int slot = (int)(q % kSlots2);
                for (long long it = 0; it < kWaitLimit && !mbar_try_wait(smem_u32(&empty_bar[slot]), (uint32_t)((q / kSlots2) & 1)); ++it) {
                    if (abort_flag) break;
                    __nanosleep(256);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (leader only) ----------------
        if (lane == 0 && leader) {
            long pos = 0, cc = 0;
            bool ok = true;
            const uint32_t idesc = idesc_f16_pair();
            const uint32_t ring = smem_u32(smem);
            for (int item = cid; item < P.n_items && ok; item += ncl) {
                Item it;
                if (!decode_item2<PERM>(P, item, it)) continue;
                const JobDev &J = P.jobs[it.job];
                const int spk = J.mode == ACF_X_FP16x3 ? 2 : 1;
                const long steps = (it.k1 - it.k0) / kBK;
                const long csteps = chunk_steps(J.mode);
                for (long s0 = 0; s0 < steps && ok; s0 += csteps) {
                    // accumulator b is free once both CTAs drained the chunk it last held
                    const int b = (int)(cc & 1);
                    ok = mbar_wait(smem_u32(&acce_bar[b]), (uint32_t)(((cc >> 1) & 1) ^ 1), &abort_flag, P.err, 12);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)(b * 256);
                    const long s1 = min(steps, s0 + csteps);
                    ok = spk == 2 ? issue_steps<2, true>(ring, full_bar, empty_bar, pos, s0, s1, dt, idesc, &abort_flag, P.err)
                                  : issue_steps<1, true>(ring, full_bar, empty_bar, pos, s0, s1, dt, idesc, &abort_flag, P.err);
                    if (!ok) break;
                    mma_commit_pair(smem_u32(&accf_bar[b]));
                    ++cc;
                }
            }
            mma_commit_pair(smem_u32(&done_bar));
            for (long long it = 0; it < kWaitLimit && !mbar_try_wait(smem_u32(&done_bar), 0); ++it) __nanosleep(256);
        }
    } else {
        // ---------------- epilogue (warps 2..9, both CTAs) ----------------
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const int odd = lane & 1;
        uint32_t m[128];
#pragma unroll
        for (int k = 0; k < 128; ++k) m[k] = 0u;
        long cc = 0;
        bool ok = true;
        for (int item = cid; item < P.n_items && ok; item += ncl) {
            Item it;
            if (!decode_item2<PERM>(P, item, it)) continue;
            const JobDev &J = P.jobs[it.job];
            const bool exact = J.mode == ACF_X_INT8;
            const long steps = (it.k1 - it.k0) / kBK;
            const long csteps = chunk_steps(J.mode);
            for (long s0 = 0; s0 < steps; s0 += csteps) {
                const int b = (int)(cc & 1);
                int w_ok = 0;
                if (lane == 0) w_ok = mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)((cc >> 1) & 1), &abort_flag, P.err, 14);
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 256 + half * 128);
#pragma unroll
                for (int piece = 0; piece < 4; ++piece) {
                    uint32_t r[32];
                    tmem_ld32(tbase + piece * 32, r);
                    tmem_wait_ld();
                    if (exact) {
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            m[piece * 32 + k] = (uint32_t)((int)m[piece * 32 + k] + __float2int_rn(__uint_as_float(r[k])));
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            m[piece * 32 + k] = __float_as_uint(__uint_as_float(m[piece * 32 + k]) + __uint_as_float(r[k]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acce_leader0 + (uint32_t)(b * sizeof(uint64_t)));
                ++cc;
            }
            if (!ok) break;
            // this CTA holds real rows [256 bi + 128 rank, +128) of the tile
            flush_tile(J, it.p, it.bi * 128 + 64 * (int)rank + 16 * q + (lane >> 1), it.bj * 128 + 64 * half + 32 * odd,
                       odd, exact, m);
#pragma unroll
            for (int k = 0; k < 128; ++k) m[k] = 0u;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols2) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
}

}  // namespace

void *tensor_map_encoder()
{
    static void *fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = p;
    });
    return fn;
}

struct TcPlan {
    TcParams params;
    int slot_of[kMaxJobs];   // caller's job index -> position in the work list
    int grid = 0;
    size_t smem = 0;
    bool pair = false;       // two-SM kernel (CTA pairs, cta_group::2)
    int *d_perm = nullptr;   // device copy of params.perm (interleaved order)
};

// Interleaved work order: items whose K range spans at most four K steps
// (short-K jobs, e.g. 256 channels of a 0.25 s integration) are flush-bound,
// the rest MMA-bound.  The persistent kernels hand work position w to worker
// w mod W (W = CTAs or CTA pairs), so alternating chunks of W long items with
// the proportional number of W-item chunks of short ones gives every worker
// a mix: the TMEM double buffer then overlaps a short item's flush with a
// long item's MMAs.  Returns an empty vector when either class is empty.
static std::vector<int> interleave_items(const TcParams &P, int workers)
{
    std::vector<int> sh, lg;
    for (int jj = 0; jj < P.n_jobs; ++jj) {
        const JobDev &D = P.jobs[jj];
        const long K64 = round_up(D.n_time, 64);
        const long per = round_up((K64 + D.k_split - 1) / D.k_split, 64);
        std::vector<int> &v = per <= 4 * kBK ? sh : lg;
        const int cnt = D.tiles_pp * D.k_split * D.n_problems;
        for (int k = 0; k < cnt; ++k) v.push_back(D.item_begin + k);
    }
    std::vector<int> perm;
    if (sh.empty() || lg.empty() || workers < 1) return perm;
    perm.reserve(sh.size() + lg.size());
    const double ratio = (double)sh.size() / (double)lg.size();   // short chunks per long chunk
    size_t si = 0, li = 0;
    double credit = 0.0;
    while (li < lg.size()) {
        for (int k = 0; k < workers && li < lg.size(); ++k) perm.push_back(lg[li++]);
        credit += ratio;
        for (; credit >= 1.0 && si < sh.size(); credit -= 1.0)
            for (int k = 0; k < workers && si < sh.size(); ++k) perm.push_back(sh[si++]);
    }
    while (si < sh.size()) perm.push_back(sh[si++]);
    return perm;
}

bool tc_supported(int device)
{
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) return false;
    return major == 10 && minor == 3;
}

cudaError_t tc_plan_create(const TcJob *jobs, int n_jobs, const TcTuning &tun, TcPlan **out, std::string *err)
{
    *out = nullptr;
    if (n_jobs < 1 || n_jobs > kMaxJobs) {
        if (err) *err = "tensor-core plan: 1..64 jobs";
        return cudaErrorInvalidValue;
    }
    auto enc = encode_fn();
    if (!enc) {
        if (err) *err = "cuTensorMapEncodeTiled unavailable";
        return cudaErrorNotSupported;
    }
    TcPlan *p = new TcPlan();
    std::memset(&p->params, 0, sizeof(p->params));
    // longest-first order when requested (items of a job are contiguous)
    std::vector<int> order(n_jobs);
    for (int j = 0; j < n_jobs; ++j) order[j] = j;
    auto cost = [&](int j) {
        return (double)jobs[j].N * jobs[j].N * jobs[j].n_time * (jobs[j].mode == ACF_X_FP16x3 ? 3 : 1);
    };
    if (tun.order >= 1) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    int items = 0;
    for (int jj = 0; jj < n_jobs; ++jj) {
        const TcJob &J = jobs[order[jj]];
        JobDev &D = p->params.jobs[jj];
        if (J.t_stride % 64 != 0 || J.N < 1 || J.n_problems < 1 || J.n_time < 0 ||
            (long)J.n_problems * 2 * J.N >= (1L << 31) || J.t_stride >= (1L << 31)) {
            delete p;
            if (err) *err = "tensor-core plan: bad job geometry";
            return cudaErrorInvalidValue;
        }
        D.V = J.V;
        D.N = J.N;
        D.n_problems = J.n_problems;
        D.mode = J.mode;
        D.nt = (tun.n_tile == 128 && !tun.pair) ? 128 : 256;
        D.n_time = J.n_time;
        const long K64 = round_up(J.n_time, 64);
        int ks = std::max(1, tun.k_split);
        if (J.mode == ACF_X_INT8) ks = std::max<long>(ks, (K64 + kInt8ItemMax - 1) / kInt8ItemMax);
        D.k_split = ks;
        D.mb = (2 * J.N + kBM - 1) / kBM;
        D.tiles_pp = tun.pair ? sq_tiles_per_problem(J.N) : tiles_per_problem(J.N, D.nt);
        D.item_begin = items;
        D.vscale = J.vscale;
        D.store = (J.store && ks == 1) ? 1 : 0;
        D.rot = J.rot;
        p->slot_of[order[jj]] = jj;
        items += D.tiles_pp * ks * J.n_problems;
        for (int h = 0; h < 2; ++h) {
            const void *base = (h == 0 || !J.x_lo) ? (const void *)J.x : (const void *)J.x_lo;
            cuuint64_t dims[2] = {(cuuint64_t)J.t_stride, (cuuint64_t)J.n_problems * 2 * J.N};
            cuuint64_t strides[1] = {(cuuint64_t)J.t_stride * 2};
            cuuint32_t box[2] = {64, 128};
            cuuint32_t es[2] = {1, 1};
            CUresult r = enc(&p->params.maps[jj][h], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims,
                             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                delete p;
                if (err) *err = "cuTensorMapEncodeTiled failed (alignment or size)";
                return cudaErrorInvalidValue;
            }
        }
    }
    p->params.n_jobs = n_jobs;
    p->params.n_items = items;
    p->pair = tun.pair != 0;
    p->params.err = device_error_word();
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->smem = (size_t)kSlots * kSlotBytes + 1024;
    static_assert(kSlots * kSlotBytes == kSlots2 * kSlotBytes2, "both kernels use the same shared memory");
    cudaError_t e = cudaSuccess;
    for (auto fn : {k_xeng_tc2<false>, k_xeng_tc2<true>, k_xeng_tc<false>, k_xeng_tc<true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    if (e != cudaSuccess) {
        delete p;
        if (err) *err = "cudaFuncSetAttribute(max dynamic smem) failed";
        return e;
    }
    if (!p->pair) {
        p->grid = std::max(1, std::min(items, sms));
    } else {
        // CTA pairs must be co-resident: as many as fit at once, at most one per work item
        int clusters = sms / 2;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * clusters);
        cfg.blockDim = dim3(kThreadsTc);
        cfg.dynamicSmemBytes = p->smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_xeng_tc2<false>, &cfg) == cudaSuccess && n > 0)
            clusters = std::min(clusters, n);
        cudaGetLastError();
        p->grid = 2 * std::max(1, std::min(items, clusters));
    }
    if (tun.order == 2) {
        const std::vector<int> perm = interleave_items(p->params, p->pair ? p->grid / 2 : p->grid);
        if (!perm.empty()) {
            // a permutation of the work items, each exactly once
            std::vector<char> seen(items, 0);
            bool okp = (int)perm.size() == items;
            for (int v : perm) okp = okp && v >= 0 && v < items && !seen[v]++;
            if (!okp) {
                delete p;
                if (err) *err = "tensor-core plan: bad interleaved order";
                return cudaErrorUnknown;
            }
            if ((e = cudaMalloc(&p->d_perm, perm.size() * sizeof(int))) != cudaSuccess ||
                (e = cudaMemcpy(p->d_perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
                    cudaSuccess) {
                cudaFree(p->d_perm);
                delete p;
                if (err) *err = "tensor-core plan: work order copy failed";
                return e;
            }
            p->params.perm = p->d_perm;
        }
    }
    *out = p;
    return cudaSuccess;
}

cudaError_t tc_plan_set_job(TcPlan *p, int job, long n_time, float vscale, int store)
{
    if (job < 0 || job >= p->params.n_jobs) return cudaErrorInvalidValue;
    JobDev &D = p->params.jobs[p->slot_of[job]];
    const long K64 = round_up(n_time, 64);
    // the time split was sized for the planned length; refuse a longer one
    if (D.mode == ACF_X_INT8 && (K64 + D.k_split - 1) / D.k_split > kInt8ItemMax) return cudaErrorInvalidValue;
    D.n_time = n_time;
    D.vscale = vscale;
    D.store = (store && D.k_split == 1) ? 1 : 0;
    return cudaSuccess;
}

cudaError_t tc_plan_set_rot(TcPlan *p, int job, const float2 *rot)
{
    if (job < 0 || job >= p->params.n_jobs) return cudaErrorInvalidValue;
    p->params.jobs[p->slot_of[job]].rot = rot;
    return cudaSuccess;
}

int tc_plan_job_stores(const TcPlan *p, int job) { return p->params.jobs[p->slot_of[job]].store; }
int tc_plan_job_split(const TcPlan *p, int job) { return p->params.jobs[p->slot_of[job]].k_split; }

cudaError_t tc_plan_launch(const TcPlan *p, cudaStream_t s)
{
    if (p->params.n_items == 0) return cudaSuccess;
    if (!p->pair) {
        if (p->params.perm) k_xeng_tc<true><<<p->grid, kThreadsTc, p->smem, s>>>(p->params);
        else k_xeng_tc<false><<<p->grid, kThreadsTc, p->smem, s>>>(p->params);
        g_launches++;
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p->grid);
    cfg.blockDim = dim3(kThreadsTc);
    cfg.dynamicSmemBytes = p->smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = p->params.perm ? cudaLaunchKernelEx(&cfg, k_xeng_tc2<true>, p->params)
                                   : cudaLaunchKernelEx(&cfg, k_xeng_tc2<false>, p->params);
    g_launches++;
    return e != cudaSuccess ? e : cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tensor-pipe ceiling probe: every SM runs one CTA whose elected thread issues
// back-to-back kind::f16 MMAs (M = 128, N = 256, K = 16) on A (128 x 64) and
// B (256 x 64) fp16 tiles resident in shared memory, accumulating in TMEM, so
// no operand traffic limits the rate.  The operands hold small non-zero
// values (the power drawn, and so the clock, depends on the data).  One
// commit at the end; the wait for it is bounded (kWaitCycles), a timeout sets
// *err.  One lane reads the accumulator back so the work stays observable.
namespace {
constexpr int kProbeThreads = 128;
constexpr uint32_t kProbeCols = 256;

__global__ void __launch_bounds__(kProbeThreads, 1) k_probe_mma(long k_steps, int *err, float *sink)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __half *ab = reinterpret_cast<__half *>(smem);
    constexpr int kElems = (kBM + 256) * kBK;            // A then B, one K step of 64
    for (int i = threadIdx.x; i < kElems; i += kProbeThreads) {
        const uint32_t hsh = (uint32_t)(i + 1) * 2654435761u;
        ab[i] = __float2half(((float)((hsh >> 20) & 63) - 31.5f) * (1.f / 64.f));
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(kProbeCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_s;
    if (threadIdx.x == 0) {
        const uint32_t a = smem_u32(smem);
        const uint64_t da = desc_sw128(a), db = desc_sw128(a + kBM * kBK * 2);
        const uint32_t idesc = idesc_f16(256);
        for (long s = 0; s < k_steps; ++s) {
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                mma_f16(tmem, da + 2 * kk, db + 2 * kk, idesc, (s > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(&done));
        const long long t0 = clock64();
        bool ok = true;
        while (!mbar_try_wait(smem_u32(&done), 0)) {
            if (clock64() - t0 > kWaitCycles) {
                atomicCAS(err, 0, 21);
                ok = false;
                break;
            }
        }
        (void)ok;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        uint32_t r[32];
        tmem_ld32(tmem, r);
        tmem_wait_ld();
        if (lane == 0) sink[blockIdx.x] = __uint_as_float(r[0]);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kProbeCols) : "memory");
    }
}
}  // namespace

cudaError_t probe_tensor_peak(long k_steps, double *tflops, float *ms_out)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!tc_supported(dev)) return cudaErrorInvalidDevice;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)(kBM + 256) * kBK * 2 + 1024;
    if ((e = cudaFuncSetAttribute(k_probe_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    float *sink = nullptr;
    int *err = device_error_word();
    if (!err) return cudaErrorMemoryAllocation;
    if ((e = cudaMalloc(&sink, sizeof(float) * sms)) != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe_mma<<<sms, kProbeThreads, smem>>>(std::max<long>(1, k_steps / 8), err, sink);   // warm-up
    g_launches++;
    cudaEventRecord(e0);
    k_probe_mma<<<sms, kProbeThreads, smem>>>(k_steps, err, sink);
    g_launches++;
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kBM * 256 * 16 * (kBK / 16) * (double)k_steps * sms;
    if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return cudaSuccess;
}

int tc_plan_items(const TcPlan *p) { return p->params.n_items; }
void tc_plan_destroy(TcPlan *p)
{
    if (p && p->d_perm) cudaFree(p->d_perm);
    delete p;
}

}  // namespace acf
