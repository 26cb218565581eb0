/*
 * acf.h -- C ABI of libacf, a B300 (sm_103a) implementation of the AARTFAAC
 * correlator stage (Prasad et al., arXiv 1609.04205, Sec. 4): a polyphase
 * filter-bank channeliser (FIR + FFT, Sec. 4.2.3), bandpass correction and
 * transpose (Sec. 4.2.4), and an X-engine that integrates one triangle of the
 * Hermitian covariance matrix per channel (Sec. 4.2.5).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Complex numbers are (re, im) pairs, re first.
 *  - Input samples are laid out [subband][time][input] (inputs contiguous),
 *    the order the data router delivers after its transpose (Sec. 3.3).
 *    Input index = 2 * antenna + polarisation.
 *  - Filter bank (Sec. 4.2.3): prototype h = Hann-windowed sinc of length
 *    L = n_taps * n_channels with sum(h) = 1; spectrum m uses stream samples
 *    [m*C, m*C + L): y_m[n] = sum_k h[k*C + n] x[m*C + k*C + n], then
 *    X_c[m] = w_c * sum_n y_m[n] exp(-2 pi i c n / C) (natural channel order).
 *    The stream is continuous across pushes: a push emits every spectrum
 *    whose window completes inside it; the first push of S samples emits
 *    floor((S - (P-1) C) / C) spectra.
 *  - n_channels == 1 selects raw-subband correlation: no filter bank, the
 *    subband samples are correlated directly (n_taps must be 1).
 *  - Visibilities (Sec. 4.2.5): V_c[i][j] = sum_t x_i,c[t] conj(x_j,c[t]) for
 *    i >= j, packed lower-triangular at bl = i*(i+1)/2 + j, laid out
 *    [subband][channel][bl].  Element type: complex float32 (8 bytes) for the
 *    FP32, FP16 and FP16x3 modes; complex int64 (16 bytes) for INT8 mode.
 *  - Pointers marked "device" must be CUDA device (or managed) memory of the
 *    current device; "host" pointers are ordinary or pinned host memory.
 *    Callers own every buffer they pass; the library never frees them.
 *    All work is enqueued on the given stream (0 = legacy default stream);
 *    a call returns once its work is enqueued, not when it completes.
 *  - Errors: every entry point returns an acf_status.  Argument checks run
 *    on the host before anything is enqueued; a failing check leaves the
 *    context unchanged.  acf_last_error() gives a one-line reason.
 *    No entry point throws, aborts or traps.
 */
#ifndef ACF_H
#define ACF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *acf_stream_t;   /* same type as cudaStream_t */
typedef struct acf_ctx acf_ctx;             /* opaque, owned by the library */
typedef struct acf_batch acf_batch;         /* opaque, owned by the library */

typedef enum {
    ACF_OK = 0,
    ACF_EINVAL = 1,        /* bad argument (shape, pointer, enum value)        */
    ACF_ENOMEM = 2,        /* device or host allocation failed                 */
    ACF_ECUDA = 3,         /* a CUDA runtime / driver call failed              */
    ACF_ESTATE = 4,        /* call not valid in the context's current state    */
    ACF_ETIMEOUT = 5,      /* a bounded device-side wait gave up               */
    ACF_EUNSUPPORTED = 6   /* valid request the build / device cannot run      */
} acf_status;

typedef enum { ACF_IN_CI8 = 0, ACF_IN_CI16 = 1, ACF_IN_CF32 = 2 } acf_in_dtype;

/* X-engine arithmetic (the "precision forms").
 *   FP32    -- plain fp32 CUDA-core FMA path (the comparison path).
 *   FP16    -- fp16 operands on tcgen05 tensor cores, fp32 accumulation.
 *   FP16x3  -- split fp16 hi + lo operands, three tensor-core products
 *              (hi*hi + hi*lo + lo*hi), fp32 accumulation: fp32-class accuracy.
 *   INT8    -- raw complex int8 subband samples (n_channels == 1,
 *              ACF_IN_CI8 only), exact integer sums, int64 output.  Runs on
 *              the fp16 tensor path: int8 values and their products are exact
 *              there, and partial sums are drained to integers before they can
 *              reach 2^24. */
typedef enum { ACF_X_FP32 = 0, ACF_X_FP16 = 1, ACF_X_FP16x3 = 2, ACF_X_INT8 = 3 } acf_xmode;

/* ---- streaming correlator (Sec. 4.2) ------------------------------------- */

/* Create a correlator for n_inputs inputs (dual-pol antennas x 2), n_subbands
 * independent subbands, n_channels in {1, 16, 64, 256} (1 = raw subband),
 * n_taps in [1, 32] (must be 1 when n_channels == 1), n_integrate >= 1 pushes
 * per integration, and pushes of at most max_samples samples per subband.
 * Allocates all device memory up front (history, channelised operand,
 * accumulators) on the current device.
 * Errors: EINVAL for any out-of-range value or a NULL `out`; EUNSUPPORTED for
 * INT8 mode with n_channels != 1 or dtype != CI8, or for tensor-core modes on
 * a device that is not sm_103; ENOMEM / ECUDA on allocation failure. */
acf_status acf_create(acf_ctx **out, int n_inputs, int n_subbands, int n_channels,
                      int n_taps, int n_integrate, acf_xmode mode, acf_in_dtype dtype,
                      long max_samples);

/* Per-channel real bandpass weights w_c (Sec. 4.2.4), `w` host, n_channels
 * floats, copied.  Default all ones.  EINVAL for NULL or non-finite values. */
acf_status acf_set_bandpass(acf_ctx *ctx, const float *w);

/* Power-of-two scale s applied to the channelised data before fp16 rounding
 * (FP16 and FP16x3 modes); visibilities are divided by s^2, exactly.  The
 * default keeps the filter-bank output of a full-scale input below the fp16
 * maximum.  EINVAL unless s is a positive power of two; ESTATE in other modes. */
acf_status acf_set_input_scale(acf_ctx *ctx, float s);

/* Push n_samples new samples per subband: `samples` device,
 * [n_subbands][n_samples][n_inputs] complex of the context's dtype.  The
 * samples are consumed in stream order on `stream`; the buffer may be reused
 * once that work completes.  1 <= n_samples <= max_samples; n_samples need
 * not be a multiple of n_channels (a one-second subband block holds 195,313
 * samples): samples past the last complete spectrum stay in the filter
 * history and open the next push's first spectrum.
 * Errors: EINVAL (NULL, size), ESTATE when the previous integration is
 * complete and has not been read, ETIMEOUT / ECUDA from the device. */
acf_status acf_push_block(acf_ctx *ctx, const void *samples, long n_samples,
                          acf_stream_t stream);

/* Same as acf_push_block but `samples` is HOST memory (pinned for best
 * speed).  Subbands are copied host->device into a device staging area on a
 * private copy stream, each subband's channeliser waiting only for its own
 * copy (Sec. 4.2, "asynchronous host to device transfers overlapping with
 * compute").  A push's copies wait only for the previous host push's kernels
 * that read the staging, so they also overlap the previous push's X-engine
 * and a visibility read-back enqueued after it.  The call returns once the
 * work is enqueued; the host buffer must stay valid and unchanged until
 * `stream` reaches this point. */
acf_status acf_push_block_host(acf_ctx *ctx, const void *samples, long n_samples,
                               acf_stream_t stream);

/* Copy out the completed integration: `out` device or host,
 * [n_subbands][n_channels][n_inputs*(n_inputs+1)/2] complex (float32, or
 * int64 in INT8 mode).  *n_ready is set to 1 when an integration was copied
 * (the copy is enqueued on `stream`) and 0 when none is complete (nothing is
 * copied).  Reading re-arms the context for the next integration. */
acf_status acf_get_visibilities(acf_ctx *ctx, void *out, int *n_ready, acf_stream_t stream);

/* Device pointer of the accumulator (same layout as acf_get_visibilities);
 * valid until acf_destroy.  The content is only meaningful once an
 * integration is complete. */
acf_status acf_visibilities_device(acf_ctx *ctx, const void **dev_ptr);

/* Zero-copy alternative to acf_get_visibilities: finishes the completed
 * integration in place (on `stream`) and re-arms the context without
 * copying it.  The visibilities stay in the accumulator (acf_visibilities_device)
 * until the next push's X-engine overwrites them; work that reads them must
 * be ordered before that push (the same stream, or an event).  *n_ready as
 * for acf_get_visibilities. */
acf_status acf_release_visibilities(acf_ctx *ctx, int *n_ready, acf_stream_t stream);

/* Spectra produced by the most recent push (per channel), the padded time
 * stride of the channelised operand, and the scale in use. */
acf_status acf_query(acf_ctx *ctx, long *last_spectra, long *t_stride, float *scale);

/* Per-push stage timing (profiling aid).  When enabled, CUDA events bracket
 * the channeliser stage (filter bank or raw transpose, plus the history
 * update) and the X-engine stage of every push, on the push's stream.
 * acf_last_timing waits for the last push's events and returns the two stage
 * durations in milliseconds (either pointer may be NULL); ESTATE when timing
 * is off or nothing was pushed since it was enabled. */
acf_status acf_enable_timing(acf_ctx *ctx, int on);
acf_status acf_last_timing(acf_ctx *ctx, float *chan_ms, float *xeng_ms);

/* Tensor-core X-engine variant for this context: 0 = one SM per 128x256 tile,
 * 1 = SM pairs (clusters of two CTAs) per 256x256 tile, each SM loading half
 * of both operands.  acf_create picks 1 in the FP16 modes with 512 or more
 * inputs, else 0.
 * Rebuilds the launch plan; only between integrations.  EINVAL for other
 * values, ESTATE mid-integration or in FP32 mode. */
acf_status acf_set_xengine_variant(acf_ctx *ctx, int variant);

/* Autotune the tensor-core X-engine on this context's geometry: times every
 * candidate launch shape (variant 0 or 1, N tile 128 or 256 real rows, time
 * split 1, 2 or 4) on the context's full launch (its first subband's
 * problems when the scratch for all of them cannot be had), writing a
 * temporary visibility buffer (allocated and freed here), and rebuilds the
 * launch plan with the fastest.  The candidates run on the operand buffer as
 * it stands: zeros before the first push, the last push's operands after an
 * integration.  Tensor-core power, and so the clock under the power cap,
 * depends on the data, so tuning after one integration of live samples ranks
 * the shapes as the pushes will run them.  Only between integrations (ESTATE
 * otherwise, and in FP32 mode); ENOMEM when the scratch cannot be had.
 * Synchronises the device. */
acf_status acf_tune(acf_ctx *ctx);

/* Measurement aid with no counterpart in the paper: the tensor pipe's rate
 * with operands resident in shared memory.  Every SM runs one CTA issuing
 * k_steps x 4 back-to-back kind::f16 MMAs (M = 128, N = 256, K = 16, fp32
 * accumulation in TMEM) on fixed tiles; no global memory is read.  Writes the
 * achieved TFLOP/s (2 M N K per MMA) and the launch time in ms (host
 * pointers, either may be NULL).  k_steps in [1, 2^22]; EUNSUPPORTED without
 * an sm_103 device.  Allocates a few bytes; synchronises the device. */
acf_status acf_probe_tensor_peak(long k_steps, double *tflops, float *ms);

/* The X-engine launch shape in use: variant (0 / 1), N tile, time split, and
 * whether acf_tune chose it (1) or the creation rule did (0).  Any pointer
 * may be NULL. */
acf_status acf_query_xengine(const acf_ctx *ctx, int *variant, int *n_tile, int *k_split, int *tuned);

/* Release every resource.  Synchronises the device first.  NULL is a no-op. */
acf_status acf_destroy(acf_ctx *ctx);

/* One-line description of the last error on `ctx` (or of the last failed
 * acf_create when ctx is NULL).  Never NULL; owned by the library. */
const char *acf_last_error(const acf_ctx *ctx);
const char *acf_status_string(acf_status s);

/* ---- stateless building blocks (each one step of Sec. 4.2) ----------------
 * These run one step on caller-owned device buffers; the streaming context is
 * built from them.  They allocate nothing. */

/* Filter-bank prototype (Sec. 4.2.3), `h_out` host, n_taps * n_channels floats. */
acf_status acf_prototype(int n_taps, int n_channels, float *h_out);

/* Channelise one block (Sec. 4.2.3 FIR + FFT, Sec. 4.2.4 bandpass + transpose).
 *   hist     device [n_subbands][n_hist][n_inputs] complex dtype (may be NULL
 *            when n_hist == 0): stream samples preceding `samples`;
 *   samples  device [n_subbands][n_samples][n_inputs] complex dtype;
 *   h        device float[n_taps * n_channels]; bandpass device float[n_channels];
 *   out      device, [n_subbands][n_channels][2*n_inputs][t_stride] where row
 *            2n holds Re and row 2n+1 holds Im of input n, spectra along the
 *            row; element float32 (out_kind 0), fp16 (1) or fp16 hi with the
 *            fp16 residual in `out_lo` (2).  Values are scaled by `scale`
 *            before fp16 rounding.  Spectra [T, roundup(T, 64)) are zeroed.
 *            Precision: float32 and split output carry the fp32 FFT.  fp16
 *            output with 64 channels, 16 taps, ci8/ci16 input and a multiple
 *            of 8 inputs computes the DFT on the tensor cores with the FIR
 *            outputs and the twiddles rounded to fp16 (fp32 accumulation);
 *            the extra error is at most (2^-10 + 2^-14) ||z||_2 per value,
 *            ||z||_2 the spectrum's norm over the 64 unweighted channels,
 *            times the channel's weight and `scale`. 
 *   *n_spectra_out (host) receives T = floor((n_hist + n_samples - (P-1) C) / C)
 *   (0 when negative).  t_stride must be >= roundup(T, 64) and a multiple of 64.
 * n_channels in {16, 64, 256}; use acf_transpose_raw for n_channels == 1. */
acf_status acf_channelise(const void *hist, long n_hist, const void *samples, long n_samples,
                          acf_in_dtype dtype, int n_subbands, int n_inputs, int n_channels,
                          int n_taps, const float *h, const float *bandpass, int out_kind,
                          void *out, void *out_lo, long t_stride, float scale,
                          long *n_spectra_out, acf_stream_t stream);

/* Raw-subband operand (a "filter bank" of one channel): the transpose of
 * Sec. 4.2.4 alone, [n_subbands][n_samples][n_inputs] complex dtype ->
 * [n_subbands][2*n_inputs][t_stride] as in acf_channelise (out_kind 0/1/2),
 * tail [n_samples, roundup(n_samples, 64)) zeroed. */
acf_status acf_transpose_raw(const void *samples, long n_samples, acf_in_dtype dtype,
                             int n_subbands, int n_inputs, int out_kind, void *out,
                             void *out_lo, long t_stride, float scale, acf_stream_t stream);

/* X-engine (Sec. 4.2.5) on a channelised operand laid out as acf_channelise
 * writes it, for n_problems = n_subbands * n_channels independent matrices:
 *   V[p][bl] += sum_{t < n_time} x_i[t] conj(x_j[t])  (ACCUMULATES into V).
 * mode FP32: x float32 (x_lo NULL); FP16: fp16 (x_lo NULL); FP16x3: fp16 hi
 * in x, lo in x_lo; INT8: fp16 holding integers |v| <= 127, V is int64 and
 * exact.  `vscale` multiplies every FP result (1/scale^2 undoes the operand
 * scale; ignored for INT8).  V device, complex float32 or int64 per mode. */
acf_status acf_xengine(acf_xmode mode, const void *x, const void *x_lo, int n_problems,
                       int n_inputs, long n_time, long t_stride, float vscale, void *V,
                       acf_stream_t stream);

/* ---- post-correlation steps on the visibilities ----------------------------
 * V below is laid out as the correlator writes it: [n_subbands][n_channels][NB]
 * with NB = n_inputs*(n_inputs+1)/2, complex float32 unless stated.  All are
 * single passes over V (HBM-bound).  Scratch comes from the stream-ordered
 * allocator (cudaMallocAsync on `stream`) and is released on the stream.
 * Errors: EINVAL on the argument checks listed, ENOMEM when the scratch
 * allocation fails, ECUDA when a launch fails; nothing is enqueued on EINVAL. */

/* Delay compensation (Sec. 4.2.4: fixed cable delays applied as phase
 * rotations of the visibilities).  With d_i the delay of input i relative to
 * the reference (x_i(t) = r(t - d_i)):
 *     V_ij <- V_ij * exp(+2 pi i f (d_i - d_j)),
 * f = f_centre[s] + c' * sample_rate / n_channels, c' = c for 2c < n_channels
 * and c - n_channels otherwise (the natural channel order of the filter bank;
 * a raw subband, n_channels == 1, sits at f_centre).  Phases are reduced to
 * turns in fp64 before the sine; the rotation is applied in fp32.
 *   V        device, modified in place;
 *   delays   host, n_inputs doubles (seconds), copied before return;
 *   f_centre host, n_subbands doubles (Hz), copied before return.
 * EINVAL: NULL pointer, a count < 1, n_subbands * n_channels > 65535,
 * sample_rate not finite and > 0, a delay or frequency not finite. */
acf_status acf_delay_compensate(void *V, int n_subbands, int n_channels, int n_inputs, const double *delays,
                                const double *f_centre, double sample_rate, acf_stream_t stream);

/* Apply the same delay compensation to every integration this context hands
 * out through acf_get_visibilities (FP modes; the INT8 path keeps exact
 * integers and gives EUNSUPPORTED).  The phase table is built on the device
 * now (n_subbands * n_channels * n_inputs complex float32, owned by the
 * context); delays == NULL switches compensation off again.  Only between
 * integrations (ESTATE otherwise). */
acf_status acf_set_delays(acf_ctx *ctx, const double *delays, const double *f_centre, double sample_rate);

/* Channel integration to a coarser resolution (Sec. 4.2.4): output channel k
 * of subband s is the sum of input channels k*group .. k*group + group - 1.
 * `group` must divide n_channels and either equal it or divide n_channels/2,
 * so that each group is contiguous in frequency in the natural channel
 * order.  vis_int64 = 1 sums complex int64 visibilities (INT8 mode) exactly.
 *   V_in   device [n_subbands][n_channels][NB];
 *   V_out  device [n_subbands][n_channels/group][NB], written; must not
 *          alias V_in.
 * EINVAL: NULL or aliasing pointers, a count < 1, a group that breaks the
 * rule above, grid limits (n_subbands or n_channels/group > 65535). */
acf_status acf_integrate_channels(const void *V_in, void *V_out, int n_subbands, int n_channels, int n_inputs,
                                  int group, int vis_int64, acf_stream_t stream);

/* Two-stage sigma-clip flagging of visibility amplitudes (Sec. 4.3).
 * Stage 1, per channel: flag cross-correlation V_ij when
 *     |V_ij|^2 > k_chan^2 * mean over the channel's cross-correlations of |V|^2;
 * stage 2, per baseline across the channels of its subband: flag channel c
 * when |V_ij,c|^2 > k_vis^2 * mean of |V_ij|^2 over the channels stage 1
 * kept.  Squares, sums and comparisons in fp64.  Autocorrelations are never
 * used or flagged.
 *   V      device, complex float32 (not modified);
 *   flags  device uint8 [n_subbands][n_channels][NB], written (1 = flagged).
 * EINVAL: NULL pointer, a count < 1, n_channels > 256, k not finite and > 0,
 * more than 65535 subbands * channels. */
acf_status acf_sigma_clip(const void *V, unsigned char *flags, int n_subbands, int n_channels, int n_inputs,
                          double k_chan, double k_vis, acf_stream_t stream);

/* Weighting matrix for lost data (Sec. 4.2.1: lost station packets; the
 * weighting step of Sec. 4.3):  W_ij = samples_per_block * sum_b m_i[b] m_j[b]
 * with m_i[b] = (mask[b][i] != 0), i.e. the number of samples both inputs
 * delivered.  Computed as AND + popcount over bit-packed masks.
 *   mask  device uint8 [n_blocks][n_inputs] (time-major like the samples);
 *   W     device int64 [NB], written, packed like V.
 * EINVAL: NULL pointer, a count < 1, n_blocks > 65535 * 32. */
acf_status acf_lost_sample_weights(const unsigned char *mask, long n_blocks, int n_inputs, long samples_per_block,
                                   long long *W, acf_stream_t stream);

/* Re-weighting for lost data: V_ij <- V_ij * n_total / W_ij for every one of
 * n_problems triangles (0 where W_ij == 0).  V device complex float32
 * [n_problems][NB], in place; W device int64 [NB] as acf_lost_sample_weights
 * writes it.  EINVAL: NULL pointer, n_total < 0, a count < 1, n_problems > 65535. */
acf_status acf_reweight(void *V, const long long *W, long n_total, int n_problems, int n_inputs,
                        acf_stream_t stream);

/* ---- gain-corrupted correlation and its adjoint (calibration) ------------
 * Model M_c = G R_c G^H with G = diag(g); residual E_c = M_c - V_c;
 * loss L = sum_c ||E_c||_F^2 over the full Hermitian matrix;
 * gradient grad_k = dL/dRe g_k + i dL/dIm g_k = 4 sum_c sum_j E_kj conj(R_kj) g_j.
 *   R, V   device [n_channels][n_inputs*(n_inputs+1)/2] complex float32, packed
 *          lower triangles (the upper triangle is their conjugate);
 *   g      device [n_inputs] complex float32;
 *   loss   device float (written, not accumulated) or NULL;
 *   grad   device [n_inputs] complex float32 (written) or NULL.
 * Uses a library-owned reduction buffer per device, grown on demand (the
 * first call for a given size may allocate; calls on different streams must
 * not overlap).  fp32 throughout. */
acf_status acf_gain_forward(const void *R, const void *V, const void *g, int n_inputs,
                            int n_channels, float *loss, void *grad, acf_stream_t stream);
/* Gradient only (recomputes the residual from R, V, g). */
acf_status acf_gain_backward(const void *R, const void *V, const void *g, int n_inputs,
                             int n_channels, void *grad, acf_stream_t stream);

/* Same as acf_gain_forward, but allocates nothing: for callers that cannot
 * call cudaMalloc while they run (processes whose device memory is reserved
 * up front, real-time loops that must not block in the allocator, plug-ins of
 * a framework that owns every allocation).  This entry point has no
 * counterpart in the paper; it is a deployment convenience.
 *   - The per-block loss partials live in a fixed device array inside the
 *     library of 65,536 floats (256 KiB), held by every GPU that loads the
 *     library until the process exits.  Problems needing more partials than
 *     that -- m (m + 1) / 2 * 4 * ceil(n_channels / 8) > 65,536 with
 *     m = ceil(n_inputs / 64), counted in 64 bits (for a multiple of 8
 *     channels: m (m + 1) / 2 * n_channels / 2) -- are rejected with ACF_EINVAL
 *     before anything is enqueued; acf_gain_forward handles them.
 *   - The first call on a device looks up the array's device address (no
 *     allocation) and keeps it.  cudaDeviceReset unloads the library's
 *     device image and would leave the kept address stale: do not reset the
 *     device between calls.
 *   - All calls share the array, so calls that may overlap on the GPU (on
 *     different streams without ordering) race; serialise them.
 *   - Each call rewrites the partials it reads (the array keeps the last
 *     call's contents, none of which a later call depends on); `grad` is
 *     zeroed on `stream` before it is accumulated.  Arguments and results as
 *     acf_gain_forward; n_channels <= 65535. */
acf_status acf_gain_forward_noalloc(const void *R, const void *V, const void *g, int n_inputs,
                                    int n_channels, float *loss, void *grad, acf_stream_t stream);

/* ---- ragged batch: many independent arrays in one persistent launch ------ */

typedef struct {
    int n_inputs;        /* >= 1 */
    int n_channels;      /* 1 (raw, INT8 exact) or 16 / 64 / 256 (split FP16) */
    int n_taps;          /* 1 for raw jobs, else [1, 32] */
    long n_samples;      /* samples per push, one subband */
} acf_job;

/* Plan a batch of n_jobs independent correlators (one subband each).  Raw
 * jobs (n_channels == 1) take complex int8 input and run INT8-exact; the
 * others take complex int8 input and run the split-FP16 path.  All device
 * memory is allocated here.  `autotune` != 0 times candidate tile / split
 * settings on the device and keeps the fastest (slow: seconds). */
acf_status acf_batch_create(acf_batch **out, const acf_job *jobs, int n_jobs, int autotune);

/* Run the batch on `stream`: `inputs[k]` device [n_samples][n_inputs] complex
 * int8 of job k; `outputs[k]` device, job k's visibilities
 * [n_channels][n_inputs*(n_inputs+1)/2] (complex int64 for raw jobs, complex
 * float32 otherwise), overwritten.  The first call captures the whole batch
 * (channelisers, transposes and ONE persistent X-engine launch) in a CUDA
 * graph keyed on the pointer set; later calls with the same pointers replay
 * it.  Each run is a fresh, independent integration (no history). */
acf_status acf_batch_run(acf_batch *b, const void *const *inputs, void *const *outputs,
                         acf_stream_t stream);

/* Tile settings chosen by the planner/autotuner: n_tile (128 or 256 real rows)
 * and the time split factor. */
acf_status acf_batch_query(const acf_batch *b, int *n_tile, int *k_split, int *n_work_items);

/* The rest of the chosen plan: pair = 1 when CTA pairs share 256 x 256 tiles
 * (tcgen05 cta_group::2), 0 for one SM per 128-row tile; order = 0 (jobs as
 * given), 1 (largest job first) or 2 (largest first, with the items of
 * short-integration jobs interleaved among the others so that each SM's
 * flush-bound and MMA-bound tiles overlap).  NULL outputs are skipped. */
acf_status acf_batch_query_plan(const acf_batch *b, int *pair, int *order);

/* Choose the plan instead of the autotuner: pair 0 or 1 (pair = 1 needs
 * n_tile 256), n_tile 128 or 256, k_split 1, 2 or 4, order 0, 1 or 2 (as
 * acf_batch_query_plan reports them).  The call first waits until the device
 * is idle (a replay of the batch's graph may still run), then drops the
 * graph; the next acf_batch_run rebuilds the work list and re-captures it.
 * ACF_EINVAL for other values (the batch keeps its plan). */
acf_status acf_batch_set_plan(acf_batch *b, int pair, int n_tile, int k_split, int order);
acf_status acf_batch_destroy(acf_batch *b);
const char *acf_batch_last_error(const acf_batch *b);

/* ---- diagnostics ---------------------------------------------------------- */

/* Kernel launches issued by this process since load (host-side count of the
 * library's own kernels; a CUDA-graph replay counts its kernel nodes). */
long long acf_launch_count(void);

/* Synchronise the current device, then read and clear the library's device
 * error word: ETIMEOUT when a bounded device-side wait gave up since the last
 * call, ECUDA when the synchronisation itself failed, OK otherwise. */
acf_status acf_device_status(void);

/* Library version string. */
const char *acf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ACF_H */
