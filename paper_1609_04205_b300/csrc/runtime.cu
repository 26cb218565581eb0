// Host runtime behind the C ABI: the streaming correlator context (Sec. 4.2:
// per-integration push -> channelise -> correlate), the ragged batch planner
// with its CUDA-graph capture and autotuner, argument validation and error
// reporting.  No entry point throws; every CUDA failure becomes a status.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "acf_internal.h"

namespace acf {
std::atomic<long long> g_launches{0};



namespace {
std::mutex g_mu;
std::map<int, int *> g_err_words;          // device -> error word
std::map<int, std::pair<float *, long long>> g_gain_scratch;   // device -> (partials, capacity)
thread_local std::string g_create_err;
}  // namespace

int *device_error_word()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_err_words.find(dev);
    if (it != g_err_words.end()) return it->second;
    int *w = nullptr;
    if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(w, 0, sizeof(int));
    g_err_words[dev] = w;
    return w;
}

}  // namespace acf

using namespace acf;

struct acf_ctx {
    int N = 0, n_sb = 0, C = 0, P = 0, n_integrate = 1;
    acf_xmode mode = ACF_X_FP32;
    acf_in_dtype dt = ACF_IN_CI8;
    long max_samples = 0;
    int device = 0;
    float scale = 1.f;
    bool user_scale = false;
    std::vector<float> h_host, bp_host;
    float *d_h = nullptr, *d_bp = nullptr;
    float2 *d_tw = nullptr;
    void *d_hist[2] = {nullptr, nullptr};
    void *d_cturn = nullptr;      // 256-channel corner-turn scratch (optional)
    size_t cturn_bytes = 0;
    int hist_cur = 0;
    long H = 0;                   // samples of history per subband
    void *d_X = nullptr, *d_Xlo = nullptr;
    long t_stride = 0;
    void *d_V = nullptr;
    size_t v_bytes = 0;
    void *d_stage = nullptr;      // host-push staging [n_sb][max_samples][N]
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> ev_copied;
    cudaEvent_t ev_stage_free = nullptr;   // recorded after the last kernel that reads the staging
    bool stage_pending = false;
    TcPlan *plan = nullptr;
    int variant = 0;              // 0: one SM per 128x256 tile; 1: SM pairs per 256x256 tile
    TcTuning tun;                 // N tile, time split, order (pair mirrors `variant`)
    bool tuned = false;           // tun chosen by acf_tune
    int pushes = 0;
    bool ready = false;
    bool v_valid = false;         // V already holds this integration's partial sums
    long last_T = 0;
    bool timing = false, timed = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    float2 *d_delay_tab = nullptr;  // delay-compensation phases [n_sb * C][N], or NULL (off)
    std::string err;
};

static acf_status fail(acf_ctx *c, acf_status s, const std::string &m)
{
    if (c) c->err = m;
    else g_create_err = m;
    return s;
}
static acf_status cuda_fail(acf_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? ACF_ENOMEM : ACF_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}
static bool valid_channels(int c) { return c == 1 || c == 16 || c == 64 || c == 256; }

// Sec. 4.2.3 prototype in double, rounded to float (same reading as the oracle).
void acf::prototype_host(int P, int C, std::vector<float> &h)
{
    const long L = (long)P * C;
    h.assign(L, 0.f);
    if (L == 1) {
        h[0] = 1.f;
        return;
    }
    std::vector<double> d(L);
    double sum = 0;
    for (long n = 0; n < L; ++n) {
        const double w = 0.5 - 0.5 * std::cos(2.0 * M_PI * (double)n / (double)(L - 1));
        const double u = ((double)n - 0.5 * (double)(L - 1)) / (double)C;
        const double s = (u == 0.0) ? 1.0 : std::sin(M_PI * u) / (M_PI * u);
        d[n] = w * s;
        sum += d[n];
    }
    for (long n = 0; n < L; ++n) h[n] = (float)(d[n] / sum);
}

// Largest power-of-two scale keeping |scale * X| < 60000 for full-scale input.
static float default_scale(acf_in_dtype dt, int C, const std::vector<float> &h, const std::vector<float> &bp)
{
    if (dt == ACF_IN_CF32) return 1.f;
    const double maxabs = dt == ACF_IN_CI8 ? 128.0 : 32768.0;
    double sabs = 0;
    for (float v : h) sabs += std::fabs((double)v);
    double wmax = 0;
    for (float v : bp) wmax = std::max(wmax, (double)std::fabs(v));
    const double bound = (C == 1 ? 1.0 : 2.0) * sabs * wmax * maxabs;
    const int e = (int)std::floor(std::log2(60000.0 / bound));
    return std::ldexp(1.f, e);
}

static long spectra_for(long len, int P, int C)
{
    const long L = (long)P * C;
    return len < L ? 0 : (len - L) / C + 1;
}

static cudaError_t make_plan(acf_ctx *c, std::string *perr)
{
    if (c->plan) {
        tc_plan_destroy(c->plan);
        c->plan = nullptr;
    }
    const long L = (long)c->P * c->C;
    TcJob j;
    j.x = static_cast<const __half *>(c->d_X);
    j.x_lo = static_cast<const __half *>(c->d_Xlo);
    j.V = c->d_V;
    j.N = c->N;
    j.n_problems = c->n_sb * c->C;
    j.n_time = c->C == 1 ? c->max_samples : spectra_for(L - 1 + c->max_samples, c->P, c->C);
    j.t_stride = c->t_stride;
    j.mode = c->mode;
    j.vscale = 1.f / (c->scale * c->scale);
    j.rot = c->d_delay_tab;
    TcTuning tun = c->tun;
    tun.pair = c->variant;
    if (tun.pair) tun.n_tile = 256;     // the pair kernel always uses 256-row tiles
    return tc_plan_create(&j, 1, tun, &c->plan, perr);
}

// X-engine launch of the context's geometry restricted to its first
// n_problems problems, into scratch V: the autotuner's timing job.
static TcJob timing_job(const acf_ctx *c, int n_problems, void *V)
{
    const long L = (long)c->P * c->C;
    TcJob j;
    j.x = static_cast<const __half *>(c->d_X);
    j.x_lo = static_cast<const __half *>(c->d_Xlo);
    j.V = V;
    j.N = c->N;
    j.n_problems = n_problems;
    j.n_time = c->C == 1 ? c->max_samples : spectra_for(L - 1 + c->max_samples, c->P, c->C);
    j.t_stride = c->t_stride;
    j.mode = c->mode;
    j.vscale = 1.f / (c->scale * c->scale);
    return j;
}

extern "C" {

const char *acf_version(void) { return "acf 0.1 (sm_103a)"; }

acf_status acf_set_xengine_variant(acf_ctx *c, int variant)
{
    if (!c) return ACF_EINVAL;
    if (variant != 0 && variant != 1) return fail(c, ACF_EINVAL, "variant must be 0 or 1");
    if (c->mode == ACF_X_FP32) return fail(c, ACF_ESTATE, "the FP32 path has no tensor-core variant");
    if (c->pushes != 0) return fail(c, ACF_ESTATE, "variant can only change between integrations");
    if (variant == c->variant) return ACF_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    const int old = c->variant;
    c->variant = variant;
    std::string perr;
    if ((e = make_plan(c, &perr)) != cudaSuccess) {
        c->variant = old;
        make_plan(c, &perr);
        return fail(c, ACF_ECUDA, "tensor-core plan: " + perr);
    }
    return ACF_OK;
}

acf_status acf_tune(acf_ctx *c)
{
    if (!c) return ACF_EINVAL;
    if (c->mode == ACF_X_FP32) return fail(c, ACF_ESTATE, "the FP32 path has no tensor-core plan");
    if (c->pushes != 0) return fail(c, ACF_ESTATE, "tuning only between integrations");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    // time the context's whole launch (how its tiles spread over the SMs
    // decides between the shapes), writing a scratch V; when that does not
    // fit, the first subband's problems
    int n_prob = c->n_sb * c->C;
    void *V = nullptr;
    size_t vb = 0;
    for (;;) {
        vb = (size_t)n_prob * n_baselines(c->N) * (c->mode == ACF_X_INT8 ? 16 : 8);
        if ((e = cudaMalloc(&V, vb)) == cudaSuccess) break;
        cudaGetLastError();
        if (n_prob == c->C) return cuda_fail(c, e, "tuning scratch");
        n_prob = c->C;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    TcJob j = timing_job(c, n_prob, V);
    float best = 1e30f;
    TcTuning best_t = c->tun;
    best_t.pair = c->variant;
    for (int pair : {1, 0})
        for (int nt : {256, 128})
            for (int ks : {1, 2, 4}) {
                if (pair && nt == 128) continue;
                TcTuning t;
                t.pair = pair;
                t.n_tile = nt;
                t.k_split = ks;
                TcPlan *p = nullptr;
                std::string perr;
                if (tc_plan_create(&j, 1, t, &p, &perr) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                tc_plan_set_job(p, 0, j.n_time, j.vscale, ks == 1 ? 1 : 0);
                // a time split accumulates atomically, so a push must clear V
                // first: that clear is part of the candidate's cost
                const bool clears = !tc_plan_job_stores(p, 0);
                if (clears) cudaMemsetAsync(V, 0, vb, st);
                tc_plan_launch(p, st);                       // warm-up
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r) {
                    if (clears) cudaMemsetAsync(V, 0, vb, st);
                    tc_plan_launch(p, st);
                }
                cudaEventRecord(e1, st);
                float ms = 0.f;
                const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                tc_plan_destroy(p);
                if (!ok) {
                    cudaGetLastError();
                    continue;
                }
                if (ms < best) {
                    best = ms;
                    best_t = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(V);
    if (best >= 1e30f) return fail(c, ACF_ECUDA, "no X-engine candidate ran");
    c->tun = best_t;
    c->variant = best_t.pair;
    c->tuned = true;
    std::string perr;
    if ((e = make_plan(c, &perr)) != cudaSuccess) return fail(c, ACF_ECUDA, "tensor-core plan: " + perr);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(c, e, "tune");
    return ACF_OK;
}

acf_status acf_query_xengine(const acf_ctx *c, int *variant, int *n_tile, int *k_split, int *tuned)
{
    if (!c) return ACF_EINVAL;
    if (variant) *variant = c->variant;
    if (n_tile) *n_tile = c->variant ? 256 : c->tun.n_tile;
    if (k_split) *k_split = c->tun.k_split;
    if (tuned) *tuned = c->tuned ? 1 : 0;
    return ACF_OK;
}

acf_status acf_probe_tensor_peak(long k_steps, double *tflops, float *ms)
{
    if (k_steps < 1 || k_steps > (1L << 22)) return ACF_EINVAL;
    cudaError_t e = probe_tensor_peak(k_steps, tflops, ms);
    if (e == cudaErrorInvalidDevice) return ACF_EUNSUPPORTED;
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

long long acf_launch_count(void) { return g_launches.load(); }

const char *acf_status_string(acf_status s)
{
    switch (s) {
    case ACF_OK: return "ok";
    case ACF_EINVAL: return "invalid argument";
    case ACF_ENOMEM: return "out of memory";
    case ACF_ECUDA: return "CUDA error";
    case ACF_ESTATE: return "invalid state";
    case ACF_ETIMEOUT: return "device wait timed out";
    case ACF_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *acf_last_error(const acf_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

acf_status acf_prototype(int n_taps, int n_channels, float *h_out)
{
    if (n_taps < 1 || n_taps > 32 || !valid_channels(n_channels) || !h_out) return ACF_EINVAL;
    std::vector<float> h;
    prototype_host(n_taps, n_channels, h);
    std::memcpy(h_out, h.data(), sizeof(float) * h.size());
    return ACF_OK;
}

acf_status acf_device_status(void)
{
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return ACF_ECUDA;
    int *w = device_error_word();
    if (!w) return ACF_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ACF_ECUDA;
    if (v != 0) {
        cudaMemset(w, 0, sizeof(int));
        return ACF_ETIMEOUT;
    }
    return ACF_OK;
}

acf_status acf_create(acf_ctx **out, int n_inputs, int n_subbands, int n_channels, int n_taps,
                      int n_integrate, acf_xmode mode, acf_in_dtype dtype, long max_samples)
{
    if (!out) return fail(nullptr, ACF_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_inputs < 1 || n_inputs > 65536) return fail(nullptr, ACF_EINVAL, "n_inputs must be in [1, 65536]");
    if (n_subbands < 1 || n_subbands > 4096) return fail(nullptr, ACF_EINVAL, "n_subbands must be in [1, 4096]");
    if (!valid_channels(n_channels)) return fail(nullptr, ACF_EINVAL, "n_channels must be 1, 16, 64 or 256");
    if (n_taps < 1 || n_taps > 32) return fail(nullptr, ACF_EINVAL, "n_taps must be in [1, 32]");
    if (n_channels == 1 && n_taps != 1) return fail(nullptr, ACF_EINVAL, "raw mode (n_channels == 1) needs n_taps == 1");
    if (n_integrate < 1) return fail(nullptr, ACF_EINVAL, "n_integrate must be >= 1");
    if (mode < ACF_X_FP32 || mode > ACF_X_INT8) return fail(nullptr, ACF_EINVAL, "bad X-engine mode");
    if (dtype < ACF_IN_CI8 || dtype > ACF_IN_CF32) return fail(nullptr, ACF_EINVAL, "bad input dtype");
    if (max_samples < 1 || max_samples > (1L << 31)) return fail(nullptr, ACF_EINVAL, "max_samples must be in [1, 2^31]");
    if (mode == ACF_X_INT8 && (n_channels != 1 || dtype != ACF_IN_CI8))
        return fail(nullptr, ACF_EUNSUPPORTED, "INT8 mode needs raw subbands (n_channels == 1) of complex int8");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (mode != ACF_X_FP32 && !tc_supported(dev))
        return fail(nullptr, ACF_EUNSUPPORTED, "tensor-core modes need an sm_103 device");
    acf_ctx *c = new acf_ctx();
    c->N = n_inputs;
    // SM pairs move a third fewer operand bytes per MMA; their 256x256 tiles
    // pay off once the array fills several of them (FP16 and split FP16 on
    // 1152 inputs: 11-14% faster per subband than one SM per tile).  The INT8
    // path (576-input raw subbands) measured faster on one SM per tile.
    c->variant = (n_inputs >= 512 && (mode == ACF_X_FP16 || mode == ACF_X_FP16x3)) ? 1 : 0;
    c->n_sb = n_subbands;
    c->C = n_channels;
    c->P = n_taps;
    c->n_integrate = n_integrate;
    c->mode = mode;
    c->dt = dtype;
    c->max_samples = max_samples;
    c->device = dev;
    prototype_host(n_taps, n_channels, c->h_host);
    c->bp_host.assign(n_channels, 1.f);
    c->scale = (mode == ACF_X_FP16 || mode == ACF_X_FP16x3) ? default_scale(dtype, n_channels, c->h_host, c->bp_host) : 1.f;
    const long L = (long)n_taps * n_channels;
    const long Tmax = n_channels == 1 ? max_samples : spectra_for(L - 1 + max_samples, n_taps, n_channels);
    c->t_stride = round_up(std::max<long>(Tmax, 1), 64);
    const int elem = in_elem_bytes(dtype);
    const long rows = (long)n_subbands * n_channels * 2 * n_inputs;
    const size_t xelem = mode == ACF_X_FP32 ? 4 : 2;
    const long NB = n_baselines(n_inputs);
    c->v_bytes = (size_t)n_subbands * n_channels * NB * (mode == ACF_X_INT8 ? 16 : 8);
    auto A = [&](void **p, size_t bytes, const char *what) -> acf_status {
        cudaError_t r = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (r != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(nullptr, r, what);
        }
        return ACF_OK;
    };
    acf_status st = ACF_OK;
    if ((st = A((void **)&c->d_h, sizeof(float) * L, "alloc prototype")) ||
        (st = A((void **)&c->d_bp, sizeof(float) * n_channels, "alloc bandpass")) ||
        (st = A(&c->d_hist[0], (size_t)n_subbands * L * n_inputs * elem, "alloc history")) ||
        (st = A(&c->d_hist[1], (size_t)n_subbands * L * n_inputs * elem, "alloc history")) ||
        (st = A(&c->d_X, (size_t)rows * c->t_stride * xelem, "alloc channelised operand")) ||
        (mode == ACF_X_FP16x3 && (st = A(&c->d_Xlo, (size_t)rows * c->t_stride * xelem, "alloc lo operand"))) ||
        (st = A(&c->d_V, c->v_bytes, "alloc visibilities"))) {
        acf_destroy(c);
        return st;
    }
    if (chan256_supported(dtype, n_channels, n_taps, c->t_stride)) {
        // input-major copy of history + push for the 256-channel kernel; when
        // it cannot be had the kernel reads the [time][input] stream directly
        const size_t cb = chan256_scratch_bytes(dtype, n_subbands, n_inputs, L, max_samples);
        if (cudaMalloc(&c->d_cturn, cb) == cudaSuccess) {
            c->cturn_bytes = cb;
        } else {
            cudaGetLastError();
            c->d_cturn = nullptr;
        }
    }
    if (n_channels > 1 && (e = make_twiddles(n_channels, &c->d_tw)) != cudaSuccess) {
        acf_destroy(c);
        return cuda_fail(nullptr, e, "twiddles");
    }
    cudaMemcpy(c->d_h, c->h_host.data(), sizeof(float) * L, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_bp, c->bp_host.data(), sizeof(float) * n_channels, cudaMemcpyHostToDevice);
    // zero the operand once: rows of unused inputs / tails stay zero
    cudaMemset(c->d_X, 0, (size_t)rows * c->t_stride * xelem);
    if (c->d_Xlo) cudaMemset(c->d_Xlo, 0, (size_t)rows * c->t_stride * xelem);
    if (!device_error_word()) {
        acf_destroy(c);
        return fail(nullptr, ACF_ENOMEM, "device error word");
    }
    if (mode != ACF_X_FP32) {
        std::string perr;
        e = make_plan(c, &perr);
        if (e != cudaSuccess) {
            acf_destroy(c);
            return fail(nullptr, ACF_ECUDA, "tensor-core plan: " + perr);
        }
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        acf_destroy(c);
        return cuda_fail(nullptr, e, "create");
    }
    *out = c;
    return ACF_OK;
}

acf_status acf_set_bandpass(acf_ctx *c, const float *w)
{
    if (!c) return ACF_EINVAL;
    if (!w) return fail(c, ACF_EINVAL, "bandpass is NULL");
    for (int k = 0; k < c->C; ++k)
        if (!std::isfinite(w[k])) return fail(c, ACF_EINVAL, "bandpass weights must be finite");
    if (c->pushes != 0) return fail(c, ACF_ESTATE, "bandpass can only change between integrations");
    c->bp_host.assign(w, w + c->C);
    cudaError_t e = cudaMemcpy(c->d_bp, w, sizeof(float) * c->C, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "bandpass copy");
    if (!c->user_scale && (c->mode == ACF_X_FP16 || c->mode == ACF_X_FP16x3)) {
        c->scale = default_scale(c->dt, c->C, c->h_host, c->bp_host);
    }
    return ACF_OK;
}

acf_status acf_set_input_scale(acf_ctx *c, float s)
{
    if (!c) return ACF_EINVAL;
    if (c->mode != ACF_X_FP16 && c->mode != ACF_X_FP16x3) return fail(c, ACF_ESTATE, "scale applies to FP16 modes only");
    int ex = 0;
    const float m = std::frexp(s, &ex);
    if (!(s > 0.f) || !std::isfinite(s) || m != 0.5f) return fail(c, ACF_EINVAL, "scale must be a positive power of two");
    if (c->pushes != 0) return fail(c, ACF_ESTATE, "scale can only change between integrations");
    c->scale = s;
    c->user_scale = true;
    return ACF_OK;
}

// One push of n_samples per subband whose samples sit at `dev_samples`.
// With `per_subband_ready` the channeliser of subband sb waits on that event.
static acf_status push_common(acf_ctx *c, const void *dev_samples, long S, cudaStream_t s,
                              const std::vector<cudaEvent_t> *per_subband_ready)
{
    cudaError_t e;
    const int elem = in_elem_bytes(c->dt);
    const long L = (long)c->P * c->C;
    const int out_kind = c->mode == ACF_X_FP32 ? OUT_F32 : (c->mode == ACF_X_FP16x3 ? OUT_F16X3 : OUT_F16);
    const float scale = (c->mode == ACF_X_FP16 || c->mode == ACF_X_FP16x3) ? c->scale : 1.f;
    if (c->timing) cudaEventRecord(c->ev[0], s);
    long T;
    const size_t xelem = c->mode == ACF_X_FP32 ? 4 : 2;
    const size_t x_sb = (size_t)c->C * 2 * c->N * c->t_stride * xelem;   // bytes per subband of X
    if (c->C == 1) {
        T = S;
        for (int sb = 0; sb < c->n_sb; ++sb) {
            if (per_subband_ready && (e = cudaStreamWaitEvent(s, (*per_subband_ready)[sb], 0)) != cudaSuccess)
                return cuda_fail(c, e, "wait copy");
            if (!per_subband_ready && sb > 0) break;
            const int nsb = per_subband_ready ? 1 : c->n_sb;
            const char *src = static_cast<const char *>(dev_samples) + (size_t)sb * S * c->N * elem;
            e = launch_transpose_raw(src, S, c->dt, nsb, c->N, out_kind, static_cast<char *>(c->d_X) + sb * x_sb,
                                     c->d_Xlo ? static_cast<char *>(c->d_Xlo) + sb * x_sb : nullptr, c->t_stride, scale, s);
            if (e != cudaSuccess) return cuda_fail(c, e, "transpose");
        }
    } else {
        const long Hn = c->H;
        T = spectra_for(Hn + S, c->P, c->C);
        const long newH = Hn + S - T * c->C;
        void *hist = c->d_hist[c->hist_cur];
        void *next = c->d_hist[c->hist_cur ^ 1];
        const int groups = per_subband_ready ? c->n_sb : 1;
        const int nsb = per_subband_ready ? 1 : c->n_sb;
        for (int sb = 0; sb < groups; ++sb) {
            if (per_subband_ready && (e = cudaStreamWaitEvent(s, (*per_subband_ready)[sb], 0)) != cudaSuccess)
                return cuda_fail(c, e, "wait copy");
            const char *src = static_cast<const char *>(dev_samples) + (size_t)sb * S * c->N * elem;
            const char *hs = static_cast<const char *>(hist) + (size_t)sb * Hn * c->N * elem;
            char *hd = static_cast<char *>(next) + (size_t)sb * newH * c->N * elem;
            if (T > 0) {
                // the scratch holds all subbands; a per-subband call uses its share
                const size_t cshare = c->cturn_bytes / c->n_sb;
                e = launch_channelise(Hn ? hs : nullptr, Hn, src, S, c->dt, nsb, c->N, c->C, c->P, c->d_h, c->d_bp,
                                      c->d_tw, out_kind, static_cast<char *>(c->d_X) + sb * x_sb,
                                      c->d_Xlo ? static_cast<char *>(c->d_Xlo) + sb * x_sb : nullptr, c->t_stride,
                                      scale, T, s, c->d_cturn ? static_cast<char *>(c->d_cturn) + sb * cshare : nullptr,
                                      (size_t)nsb * cshare);
                if (e != cudaSuccess) return cuda_fail(c, e, "channelise");
            }
            e = launch_history(Hn ? hs : nullptr, Hn, src, S, c->dt, nsb, c->N, T * c->C, newH, hd, newH, s);
            if (e != cudaSuccess) return cuda_fail(c, e, "history");
        }
        c->hist_cur ^= 1;
        c->H = newH;
        (void)L;
    }
    if (per_subband_ready && c->ev_stage_free) {
        // the staging's readers (transposes or channelisers and the history
        // copies) are all enqueued: the next host push may refill it after them
        if ((e = cudaEventRecord(c->ev_stage_free, s)) != cudaSuccess) return cuda_fail(c, e, "record staging");
        c->stage_pending = true;
    }
    if (c->timing) cudaEventRecord(c->ev[1], s);
    if (T > 0) {
        // the first X-engine pass of an integration overwrites V when one work item owns
        // each tile; otherwise V is cleared and every pass adds atomically
        bool clear = !c->v_valid;
        if (c->mode != ACF_X_FP32) {
            if ((e = tc_plan_set_job(c->plan, 0, T, 1.f / (scale * scale), c->v_valid ? 0 : 1)) != cudaSuccess)
                return cuda_fail(c, e, "x-engine plan");
            if (tc_plan_job_stores(c->plan, 0)) clear = false;
        }
        if (clear && (e = cudaMemsetAsync(c->d_V, 0, c->v_bytes, s)) != cudaSuccess)
            return cuda_fail(c, e, "clear accumulator");
        c->v_valid = true;
        if (c->mode == ACF_X_FP32) {
            e = launch_xeng_simt(static_cast<const float *>(c->d_X), c->n_sb * c->C, c->N, T, c->t_stride, 1.f,
                                 static_cast<float2 *>(c->d_V), s);
        } else {
            e = tc_plan_launch(c->plan, s);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "x-engine");
    }
    if (c->timing) {
        cudaEventRecord(c->ev[2], s);
        c->timed = true;
    }
    c->last_T = T;
    if (++c->pushes == c->n_integrate) {
        c->pushes = 0;
        c->ready = true;
        if (!c->v_valid) {   // an integration without a single spectrum is all zeros
            if ((e = cudaMemsetAsync(c->d_V, 0, c->v_bytes, s)) != cudaSuccess) return cuda_fail(c, e, "clear");
            c->v_valid = true;
        }
    }
    return ACF_OK;
}

acf_status acf_push_block(acf_ctx *c, const void *samples, long n_samples, acf_stream_t stream)
{
    if (!c) return ACF_EINVAL;
    if (!samples) return fail(c, ACF_EINVAL, "samples is NULL");
    if (n_samples < 1 || n_samples > c->max_samples) return fail(c, ACF_EINVAL, "n_samples out of [1, max_samples]");
    if (c->ready) return fail(c, ACF_ESTATE, "previous integration complete but not read");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, samples) != cudaSuccess || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(c, ACF_EINVAL, "samples must be device memory (use acf_push_block_host for host buffers)");
    }
    return push_common(c, samples, n_samples, (cudaStream_t)stream, nullptr);
}

acf_status acf_push_block_host(acf_ctx *c, const void *samples, long n_samples, acf_stream_t stream)
{
    if (!c) return ACF_EINVAL;
    if (!samples) return fail(c, ACF_EINVAL, "samples is NULL");
    if (n_samples < 1 || n_samples > c->max_samples) return fail(c, ACF_EINVAL, "n_samples out of [1, max_samples]");
    if (c->ready) return fail(c, ACF_ESTATE, "previous integration complete but not read");
    cudaError_t e;
    const size_t per_sb = (size_t)n_samples * c->N * in_elem_bytes(c->dt);
    if (!c->d_stage) {
        if ((e = cudaMalloc(&c->d_stage, (size_t)c->max_samples * c->N * in_elem_bytes(c->dt) * c->n_sb)) != cudaSuccess)
            return cuda_fail(c, e, "staging alloc");
        if ((e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "copy stream");
        c->ev_copied.resize(c->n_sb);
        for (auto &ev : c->ev_copied)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(c, e, "event");
        if ((e = cudaEventCreateWithFlags(&c->ev_stage_free, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "event");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the copies must not overwrite staging that the previous host push's
    // kernels still read; they need not wait for anything else on `s` (the
    // previous X-engine, a visibility read-back), so this push's host-to-device
    // copies overlap that work
    if (c->stage_pending && (e = cudaStreamWaitEvent(c->copy_stream, c->ev_stage_free, 0)) != cudaSuccess)
        return cuda_fail(c, e, "wait staging");
    for (int sb = 0; sb < c->n_sb; ++sb) {
        e = cudaMemcpyAsync(static_cast<char *>(c->d_stage) + sb * per_sb, static_cast<const char *>(samples) + sb * per_sb,
                            per_sb, cudaMemcpyHostToDevice, c->copy_stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "H2D copy");
        cudaEventRecord(c->ev_copied[sb], c->copy_stream);
    }
    return push_common(c, c->d_stage, n_samples, s, &c->ev_copied);
}

// Hand out a completed integration: finish it in place (the FP32 path's
// delay rotation), copy it to `out` when given, and re-arm the context.
static acf_status finish_integration(acf_ctx *c, void *out, int *n_ready, cudaStream_t s)
{
    *n_ready = 0;
    if (!c->ready) return ACF_OK;
    cudaError_t e = cudaSuccess;
    if (c->d_delay_tab && c->mode == ACF_X_FP32) {
        // the fp32 CUDA-core path has no fused rotation: the accumulator is
        // reset when the next integration starts, so rotate it in place (the
        // tensor-core X-engine applies the table in its flush)
        e = launch_delay_apply(static_cast<float2 *>(c->d_V), c->d_delay_tab, (long)c->n_sb * c->C, c->N, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "delay compensation");
    }
    if (out) {
        e = cudaMemcpyAsync(out, c->d_V, c->v_bytes, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy visibilities");
    }
    *n_ready = 1;
    c->ready = false;
    c->v_valid = false;
    return ACF_OK;
}

acf_status acf_get_visibilities(acf_ctx *c, void *out, int *n_ready, acf_stream_t stream)
{
    if (!c) return ACF_EINVAL;
    if (!out || !n_ready) return fail(c, ACF_EINVAL, "out / n_ready is NULL");
    return finish_integration(c, out, n_ready, (cudaStream_t)stream);
}

acf_status acf_release_visibilities(acf_ctx *c, int *n_ready, acf_stream_t stream)
{
    if (!c) return ACF_EINVAL;
    if (!n_ready) return fail(c, ACF_EINVAL, "n_ready is NULL");
    return finish_integration(c, nullptr, n_ready, (cudaStream_t)stream);
}

acf_status acf_set_delays(acf_ctx *c, const double *delays, const double *f_centre, double sample_rate)
{
    if (!c) return ACF_EINVAL;
    if (c->pushes != 0) return fail(c, ACF_ESTATE, "delays can only change between integrations");
    if (!delays) {
        cudaError_t e = cudaDeviceSynchronize();
        if (c->plan) tc_plan_set_rot(c->plan, 0, nullptr);
        cudaFree(c->d_delay_tab);
        c->d_delay_tab = nullptr;
        return e == cudaSuccess ? ACF_OK : cuda_fail(c, e, "sync");
    }
    if (c->mode == ACF_X_INT8) return fail(c, ACF_EUNSUPPORTED, "INT8 visibilities stay exact integers");
    if (!f_centre || !(sample_rate > 0.0) || !std::isfinite(sample_rate))
        return fail(c, ACF_EINVAL, "f_centre is NULL or sample_rate is not finite and positive");
    for (int i = 0; i < c->N; ++i)
        if (!std::isfinite(delays[i])) return fail(c, ACF_EINVAL, "non-finite delay");
    for (int k = 0; k < c->n_sb; ++k)
        if (!std::isfinite(f_centre[k])) return fail(c, ACF_EINVAL, "non-finite centre frequency");
    const long n_prob = (long)c->n_sb * c->C;
    if (n_prob > 65535) return fail(c, ACF_EINVAL, "more than 65535 subbands x channels");
    double *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(double) * ((size_t)c->N + c->n_sb));
    if (e != cudaSuccess) return fail(c, ACF_ENOMEM, "delay staging");
    if (!c->d_delay_tab) {
        e = cudaMalloc(&c->d_delay_tab, sizeof(float2) * (size_t)n_prob * c->N);
        if (e != cudaSuccess) {
            c->d_delay_tab = nullptr;
            cudaFree(tmp);
            return fail(c, ACF_ENOMEM, "delay table");
        }
    }
    e = cudaMemcpy(tmp, delays, sizeof(double) * c->N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tmp + c->N, f_centre, sizeof(double) * c->n_sb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_delay_table(tmp, tmp + c->N, sample_rate, c->n_sb, c->C, c->N, c->d_delay_tab, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e == cudaSuccess && c->plan) e = tc_plan_set_rot(c->plan, 0, c->d_delay_tab);
    return e == cudaSuccess ? ACF_OK : cuda_fail(c, e, "delay table");
}

acf_status acf_visibilities_device(acf_ctx *c, const void **p)
{
    if (!c || !p) return ACF_EINVAL;
    *p = c->d_V;
    return ACF_OK;
}

acf_status acf_query(acf_ctx *c, long *last_spectra, long *t_stride, float *scale)
{
    if (!c) return ACF_EINVAL;
    if (last_spectra) *last_spectra = c->last_T;
    if (t_stride) *t_stride = c->t_stride;
    if (scale) *scale = c->scale;
    return ACF_OK;
}

acf_status acf_enable_timing(acf_ctx *c, int on)
{
    if (!c) return ACF_EINVAL;
    if (on && !c->ev[0]) {
        for (auto &e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(c, ACF_ECUDA, "event create");
    }
    c->timing = on != 0;
    c->timed = false;
    return ACF_OK;
}

acf_status acf_last_timing(acf_ctx *c, float *chan_ms, float *xeng_ms)
{
    if (!c) return ACF_EINVAL;
    if (!c->timing || !c->timed) return fail(c, ACF_ESTATE, "timing off or no push since it was enabled");
    cudaError_t e = cudaEventSynchronize(c->ev[2]);
    if (e != cudaSuccess) return cuda_fail(c, e, "timing sync");
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
    if (chan_ms) *chan_ms = a;
    if (xeng_ms) *xeng_ms = b;
    return ACF_OK;
}

acf_status acf_destroy(acf_ctx *c)
{
    if (!c) return ACF_OK;
    cudaDeviceSynchronize();
    for (auto ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(c->d_h);
    cudaFree(c->d_bp);
    cudaFree(c->d_tw);
    cudaFree(c->d_hist[0]);
    cudaFree(c->d_hist[1]);
    cudaFree(c->d_cturn);
    cudaFree(c->d_X);
    cudaFree(c->d_Xlo);
    cudaFree(c->d_V);
    cudaFree(c->d_stage);
    cudaFree(c->d_delay_tab);
    for (auto ev : c->ev_copied) cudaEventDestroy(ev);
    if (c->ev_stage_free) cudaEventDestroy(c->ev_stage_free);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->plan) tc_plan_destroy(c->plan);
    delete c;
    cudaGetLastError();
    return ACF_OK;
}

// ---- stateless building blocks ---------------------------------------------

acf_status acf_channelise(const void *hist, long n_hist, const void *samples, long n_samples, acf_in_dtype dtype,
                          int n_subbands, int n_inputs, int n_channels, int n_taps, const float *h,
                          const float *bandpass, int out_kind, void *out, void *out_lo, long t_stride, float scale,
                          long *n_spectra_out, acf_stream_t stream)
{
    if (!samples || !h || !bandpass || !out || n_samples < 0 || n_hist < 0 || (n_hist > 0 && !hist)) return ACF_EINVAL;
    if (n_channels != 16 && n_channels != 64 && n_channels != 256) return ACF_EINVAL;
    if (n_taps < 1 || n_taps > 32 || n_inputs < 1 || n_subbands < 1) return ACF_EINVAL;
    if (out_kind < 0 || out_kind > 2 || (out_kind == 2 && !out_lo)) return ACF_EINVAL;
    if (dtype < ACF_IN_CI8 || dtype > ACF_IN_CF32) return ACF_EINVAL;
    const long T = spectra_for(n_hist + n_samples, n_taps, n_channels);
    if (t_stride % 64 != 0 || t_stride < round_up(T, 64)) return ACF_EINVAL;
    if (n_spectra_out) *n_spectra_out = T;
    if (T == 0) return ACF_OK;
    float2 *tw = nullptr;
    {
        static std::mutex mu;
        static std::map<std::pair<int, int>, float2 *> cache;
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        auto key = std::make_pair(dev, n_channels);
        auto it = cache.find(key);
        if (it == cache.end()) {
            if (make_twiddles(n_channels, &tw) != cudaSuccess) return ACF_ECUDA;
            cache[key] = tw;
        } else {
            tw = it->second;
        }
    }
    cudaError_t e = launch_channelise(hist, n_hist, samples, n_samples, dtype, n_subbands, n_inputs, n_channels, n_taps, h,
                                      bandpass, tw, out_kind, out, out_lo, t_stride, scale, T, (cudaStream_t)stream);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_transpose_raw(const void *samples, long n_samples, acf_in_dtype dtype, int n_subbands, int n_inputs,
                             int out_kind, void *out, void *out_lo, long t_stride, float scale, acf_stream_t stream)
{
    if (!samples || !out || n_samples < 1 || n_subbands < 1 || n_inputs < 1) return ACF_EINVAL;
    if (out_kind < 0 || out_kind > 2 || (out_kind == 2 && !out_lo)) return ACF_EINVAL;
    if (dtype < ACF_IN_CI8 || dtype > ACF_IN_CF32) return ACF_EINVAL;
    if (t_stride % 64 != 0 || t_stride < round_up(n_samples, 64)) return ACF_EINVAL;
    cudaError_t e = launch_transpose_raw(samples, n_samples, dtype, n_subbands, n_inputs, out_kind, out, out_lo, t_stride,
                                         scale, (cudaStream_t)stream);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_xengine(acf_xmode mode, const void *x, const void *x_lo, int n_problems, int n_inputs, long n_time,
                       long t_stride, float vscale, void *V, acf_stream_t stream)
{
    if (!x || !V || n_problems < 1 || n_inputs < 1 || n_time < 0 || t_stride % 64 != 0 || t_stride < round_up(n_time, 64))
        return ACF_EINVAL;
    if (reinterpret_cast<uintptr_t>(V) % 16 != 0 || reinterpret_cast<uintptr_t>(x) % 16 != 0 ||
        (x_lo && reinterpret_cast<uintptr_t>(x_lo) % 16 != 0))
        return ACF_EINVAL;
    if (mode < ACF_X_FP32 || mode > ACF_X_INT8) return ACF_EINVAL;
    if (mode == ACF_X_FP16x3 && !x_lo) return ACF_EINVAL;
    if (n_time == 0) return ACF_OK;
    cudaError_t e;
    if (mode == ACF_X_FP32) {
        e = launch_xeng_simt(static_cast<const float *>(x), n_problems, n_inputs, n_time, t_stride, vscale,
                             static_cast<float2 *>(V), (cudaStream_t)stream);
        return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (!tc_supported(dev)) return ACF_EUNSUPPORTED;
    TcJob j;
    j.x = static_cast<const __half *>(x);
    j.x_lo = static_cast<const __half *>(x_lo);
    j.V = V;
    j.N = n_inputs;
    j.n_problems = n_problems;
    j.n_time = n_time;
    j.t_stride = t_stride;
    j.mode = mode;
    j.vscale = vscale;
    TcPlan *p = nullptr;
    TcTuning tun;
    std::string perr;
    if (tc_plan_create(&j, 1, tun, &p, &perr) != cudaSuccess) return ACF_EINVAL;
    e = tc_plan_launch(p, (cudaStream_t)stream);
    tc_plan_destroy(p);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

// ---- gain -------------------------------------------------------------------

static acf_status gain_common(const void *R, const void *V, const void *g, int N, int C, float *loss, void *grad,
                              cudaStream_t s)
{
    if (!R || !V || !g || N < 1 || C < 1 || C > 65535) return ACF_EINVAL;
    // element offsets within one channel's triangle are 32-bit (this also
    // bounds the tile count, which fills grid x)
    if ((long long)N * (N + 1) / 2 > 0x7fffffffLL) return ACF_EINVAL;
    const long long need = gain_partials_needed(N, C);
    float *part = nullptr;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(g_mu);
        auto &slot = g_gain_scratch[dev];
        if (slot.second < need) {
            if (slot.first) {
                cudaStreamSynchronize(s);
                cudaFree(slot.first);
            }
            slot.first = nullptr;
            slot.second = 0;
            if (cudaMalloc(&slot.first, sizeof(float) * need) != cudaSuccess) return ACF_ENOMEM;
            slot.second = need;
        }
        part = slot.first;
    }
    cudaError_t e = launch_gain(static_cast<const float2 *>(R), static_cast<const float2 *>(V),
                                static_cast<const float2 *>(g), N, C, loss, static_cast<float2 *>(grad), part, need, s);
    return e == cudaSuccess ? ACF_OK : ACF_ECUDA;
}

acf_status acf_gain_forward(const void *R, const void *V, const void *g, int n_inputs, int n_channels, float *loss,
                            void *grad, acf_stream_t stream)
{
    if (!loss && !grad) return ACF_EINVAL;
    return gain_common(R, V, g, n_inputs, n_channels, loss, grad, (cudaStream_t)stream);
}

acf_status acf_gain_backward(const void *R, const void *V, const void *g, int n_inputs, int n_channels, void *grad,
                             acf_stream_t stream)
{
    if (!grad) return ACF_EINVAL;
    return gain_common(R, V, g, n_inputs, n_channels, nullptr, grad, (cudaStream_t)stream);
}

}  // extern "C"
