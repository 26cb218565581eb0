// Internal declarations shared by the libacf translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <atomic>
#include <string>
#include <vector>

#include "acf.h"

namespace acf {

// Host-side count of kernel launches (graph replays add their node count).
extern std::atomic<long long> g_launches;

// Device-side error word written by bounded waits (0 = fine).  One per
// device, allocated on first use by the runtime.
int *device_error_word();

enum OutKind { OUT_F32 = 0, OUT_F16 = 1, OUT_F16X3 = 2 };

inline int in_elem_bytes(acf_in_dtype d) { return d == ACF_IN_CI8 ? 2 : d == ACF_IN_CI16 ? 4 : 8; }
inline long round_up(long a, long b) { return (a + b - 1) / b * b; }
inline long n_baselines(long n) { return n * (n + 1) / 2; }

// Filter-bank prototype (Sec. 4.2.3): Hann-windowed sinc of length P*C, unit
// sum, evaluated in double and rounded to float (runtime.cu).
void prototype_host(int P, int C, std::vector<float> &h);

// ---- channeliser (chan_ppf.cu) -------------------------------------------
// Twiddle table exp(-2 pi i k / C), k < C, float2, device.
cudaError_t make_twiddles(int C, float2 **d_tw);
// scratch: an optional device buffer the 256-channel path may use for its
// corner turn (chan256_scratch_bytes); other geometries ignore it.
cudaError_t launch_channelise(const void *hist, long n_hist, const void *samples, long n_samples,
                              acf_in_dtype dt, int n_sb, int N, int C, int P, const float *h,
                              const float *bandpass, const float2 *tw, int out_kind, void *out,
                              void *out_lo, long t_stride, float scale, long T,
                              cudaStream_t s, void *scratch = nullptr, size_t scratch_bytes = 0);
// General kernel (any supported C, P, dtype); launch_channelise picks the fast path when it applies.
cudaError_t launch_channelise_generic(const void *hist, long n_hist, const void *samples, long n_samples,
                                      acf_in_dtype dt, int n_sb, int N, int C, int P, const float *h,
                                      const float *bandpass, const float2 *tw, int out_kind, void *out,
                                      void *out_lo, long t_stride, float scale, long T, cudaStream_t s);
// Fast path (chan_fast.cu): 16 taps, 16 or 64 channels, ci8 / ci16 input.
bool chan_fast_supported(acf_in_dtype dt, int C, int P);
cudaError_t launch_chan_fast(const void *hist, long n_hist, const void *samples, long n_samples, acf_in_dtype dt,
                             int n_sb, int N, int C, const float *h, const float *bp, const float2 *tw, int out_kind,
                             void *out, void *out_lo, long t_stride, float scale, long T, cudaStream_t s);
// 256-channel, 16-tap channeliser (chan256.cu): ci8 / ci16 input, history
// included, operand rows padded to a multiple of 16 spectra.
// With a scratch buffer of chan256_scratch_bytes() it first corner-turns the
// stream into input-major rows, so that the per-phase sample loads are
// contiguous; without one it reads the [time][input] stream directly.
bool chan256_supported(acf_in_dtype dt, int C, int P, long t_stride);
long chan256_row_pitch(long n_hist, long n_samples);
size_t chan256_scratch_bytes(acf_in_dtype dt, int n_sb, int N, long n_hist, long n_samples);
cudaError_t launch_chan256(const void *hist, long n_hist, const void *samples, long n_samples, acf_in_dtype dt,
                           int n_sb, int N, const float *h, const float *bp, const float2 *tw, int out_kind,
                           void *out, void *out_lo, long t_stride, float scale, long T, cudaStream_t s,
                           void *scratch = nullptr, size_t scratch_bytes = 0);
// Warp-specialised 64-channel, 16-tap channeliser (chan_ws.cu): ci8 / ci16
// input read through a TMA tensor map (N a multiple of 16 bytes' worth of
// inputs, 16-byte aligned samples).  It produces spectra
// [chan_ws_begin(...), roundup(T, 64)); the spectra before that reach into
// the history and are left to the generic kernel.  The tensor-core variant
// (fp16 and split fp16 output) reads a history shorter than one window itself
// and begins at spectrum 0; otherwise the range begins at
// chan_ws_first_spectrum(n_hist).
bool chan_ws_supported(acf_in_dtype dt, int C, int P, int N, const void *samples, long n_samples);
long chan_ws_first_spectrum(long n_hist);
long chan_ws_begin(acf_in_dtype dt, int out_kind, int N, long t_stride, const void *out, const void *out_lo,
                   const void *hist, long n_hist);
cudaError_t launch_chan_ws(const void *hist, const void *samples, long n_samples, long n_hist, acf_in_dtype dt,
                           int n_sb, int N, const float *h, const float *bp, float scale, int out_kind, void *out,
                           void *out_lo, long t_stride, long T, cudaStream_t s);
// Generic kernel restricted to spectra [0, m_head) (m_head a multiple of 16).
cudaError_t launch_channelise_head(const void *hist, long n_hist, const void *samples, long n_samples,
                                   acf_in_dtype dt, int n_sb, int N, int C, int P, const float *h,
                                   const float *bandpass, const float2 *tw, int out_kind, void *out,
                                   void *out_lo, long t_stride, float scale, long T, long m_head, cudaStream_t s);
// cuTensorMapEncodeTiled through the runtime's driver entry point (NULL when
// unavailable); returned untyped so this header needs no driver types.
void *tensor_map_encoder();
cudaError_t launch_transpose_raw(const void *samples, long n_samples, acf_in_dtype dt, int n_sb,
                                 int N, int out_kind, void *out, void *out_lo, long t_stride,
                                 float scale, cudaStream_t s);
// Copy stream samples [from, from + count) of (hist ++ samples) into dst
// ([n_sb][count][N]); used to carry the filter-bank history across pushes.
cudaError_t launch_history(const void *hist, long n_hist, const void *samples, long n_samples,
                           acf_in_dtype dt, int n_sb, int N, long from, long count, void *dst,
                           long dst_cap, cudaStream_t s);

// ---- X-engines --------------------------------------------------------------
cudaError_t launch_xeng_simt(const float *x, int n_problems, int N, long n_time, long t_stride,
                             float vscale, float2 *V, cudaStream_t s);

// One job of the tensor-core X-engine work list.
struct TcJob {
    const __half *x;      // operand (hi), [n_problems][2N][t_stride]
    const __half *x_lo;   // lo part (FP16x3) or nullptr
    void *V;              // accumulator, [n_problems][NB] complex float or int64
    int N;                // complex inputs
    int n_problems;       // subbands * channels
    long n_time;          // valid spectra (K extent; zero padded to 64)
    long t_stride;        // row stride in elements
    int mode;             // ACF_X_FP16, ACF_X_FP16x3 or ACF_X_INT8
    float vscale;
    int store = 0;        // 1: overwrite V (allowed only when one work item owns each tile)
    const float2 *rot = nullptr;   // delay compensation a[problem][input] applied in the flush, or nullptr
};
struct TcPlan;            // opaque: tensor maps + work list on the device
struct TcTuning {
    int n_tile = 256;     // real rows per N tile: 128 or 256
    int k_split = 1;      // time split factor per tile (atomically reduced)
    int order = 0;        // 0: problem-major, 1: longest-first, 2: longest-first with short-K items interleaved
    int pair = 0;         // 1: two-SM kernel (256x256 tiles on CTA pairs, cta_group::2)
};
cudaError_t tc_plan_create(const TcJob *jobs, int n_jobs, const TcTuning &tun, TcPlan **out,
                           std::string *err);
cudaError_t tc_plan_launch(const TcPlan *p, cudaStream_t s);
// Per-launch job parameters: valid spectra, the fp result scale, and whether
// the launch may overwrite V (granted only when the job has no time split).
cudaError_t tc_plan_set_job(TcPlan *p, int job, long n_time, float vscale, int store);
// Delay compensation for a job's float results from now on (nullptr: off):
// every visibility the flush writes becomes V_ij a_i conj(a_j), a[p][i] from
// launch_delay_table.
cudaError_t tc_plan_set_rot(TcPlan *p, int job, const float2 *rot);
int tc_plan_job_stores(const TcPlan *p, int job);   // 1 when the job overwrites V
int tc_plan_job_split(const TcPlan *p, int job);
int tc_plan_items(const TcPlan *p);
void tc_plan_destroy(TcPlan *p);
// Tensor-pipe ceiling with resident operands (xeng_tc.cu): kind::f16 MMAs
// M = 128, N = 256 on every SM for k_steps K steps of 64; TFLOP/s and ms.
cudaError_t probe_tensor_peak(long k_steps, double *tflops, float *ms);
bool tc_supported(int device);

// ---- gain (gain.cu) ---------------------------------------------------------
cudaError_t launch_gain(const float2 *R, const float2 *V, const float2 *g, int N, int C,
                        float *loss, float2 *grad, float *partials, long long n_partials_cap,
                        cudaStream_t s);
// Loss partials a gain launch needs (64-bit): one per block, a block covering a
// 16 x 64 tile of the triangle for 4 channels: 2 m (m + 1) * ceil(C / 4), m = ceil(N / 64).
long long gain_partials_needed(int N, int C);

// ---- post-correlation steps (post.cu) ------------------------------------------
cudaError_t launch_delay_table(const double *d_delays, const double *d_fc, double fs, int n_sb, int C, int N,
                               float2 *d_tab, cudaStream_t s);
cudaError_t launch_delay_apply(float2 *V, const float2 *d_tab, long n_prob, int N, cudaStream_t s);
cudaError_t launch_integrate(const void *in, void *out, int n_sb, int C, int N, int G, int int64, cudaStream_t s);
cudaError_t launch_sigma_clip(const float2 *V, int n_sb, int C, int N, double k1, double k2, double *d_sums,
                              unsigned char *flags, cudaStream_t s);
cudaError_t launch_weights(const unsigned char *mask, long n_blocks, int N, long spb, uint32_t *d_bits, long long *W,
                           cudaStream_t s);
cudaError_t launch_reweight(float2 *V, const long long *W, long n_total, int n_prob, int N, cudaStream_t s);

}  // namespace acf
