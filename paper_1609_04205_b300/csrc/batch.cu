// Ragged batch: many independent arrays (different input and channel counts)
// correlated by one persistent tensor-core X-engine launch, with every step
// captured in a single CUDA graph (the paper spreads independent subbands
// over free GPUs, Sec. 4.2 "GPU processing"; on one B300 the independent
// problems share one persistent launch instead).
//
// Raw jobs (n_channels == 1) run INT8-exact; channelised jobs run the split
// fp16 path after the filter bank.  The autotuner times the X-engine launch
// for each candidate (N tile 128/256, time split 1/2/4, job order) on the
// real geometry and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "acf_internal.h"

namespace acf {
namespace {
thread_local std::string g_batch_create_err;

long spectra_of(long len, int P, int C)
{
    const long L = (long)P * C;
    return len < L ? 0 : (len - L) / C + 1;
}

}  // namespace
}  // namespace acf

using namespace acf;

static TcTuning default_tuning()
{
    TcTuning t;
    t.pair = 0;        // one SM per tile; the autotuner also tries SM pairs
    return t;
}

struct acf_batch {
    std::vector<acf_job> jobs;
    std::vector<long> T, t_stride;
    std::vector<void *> X, Xlo;
    std::vector<void *> cturn;          // per job: 256-channel corner-turn scratch (or null)
    std::vector<size_t> cturn_bytes;
    std::vector<size_t> v_bytes;
    std::vector<float> scale;
    std::map<long, float *> d_h;        // key P*1024 + C
    std::map<int, float2 *> d_tw;       // key C
    std::map<int, float *> d_bp;        // key C (all ones)
    TcTuning tun = default_tuning();
    TcPlan *plan = nullptr;
    cudaStream_t s_int = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // per-job preparation (channeliser or raw transpose) forks onto these
    // streams so that small jobs run side by side; the X-engine joins them
    static constexpr int kAux = 4;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t aux_done[kAux] = {};
    cudaEvent_t ev_fork = nullptr;
    std::vector<int> aux_of;           // job -> aux stream (longest work first, least loaded)
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void *> g_in;
    std::vector<void *> g_out;
    long long graph_kernels = 0;
    std::string err;
};

static acf_status bf(acf_batch *b, acf_status s, const std::string &m)
{
    if (b) b->err = m;
    else g_batch_create_err = m;
    return s;
}

static std::vector<TcJob> tc_jobs(const acf_batch *b, void *const *outputs)
{
    std::vector<TcJob> v(b->jobs.size());
    for (size_t k = 0; k < b->jobs.size(); ++k) {
        TcJob &j = v[k];
        const bool raw = b->jobs[k].n_channels == 1;
        j.x = static_cast<const __half *>(b->X[k]);
        j.x_lo = static_cast<const __half *>(b->Xlo[k]);
        j.V = outputs[k];
        j.N = b->jobs[k].n_inputs;
        j.n_problems = b->jobs[k].n_channels;
        j.n_time = b->T[k];
        j.t_stride = b->t_stride[k];
        j.mode = raw ? ACF_X_INT8 : ACF_X_FP16x3;
        j.vscale = raw ? 1.f : 1.f / (b->scale[k] * b->scale[k]);
        j.store = 1;      // each run is a fresh integration: overwrite when the tiles are unsplit
    }
    return v;
}

// Enqueue the whole batch on stream s: the jobs' preparation forks across the
// auxiliary streams (graph branches when captured), then one X-engine launch.
static cudaError_t enqueue_all(acf_batch *b, const void *const *inputs, void *const *outputs, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaEventRecord(b->ev_fork, s)) != cudaSuccess) return e;
    for (int a = 0; a < acf_batch::kAux; ++a)
        if ((e = cudaStreamWaitEvent(b->aux[a], b->ev_fork, 0)) != cudaSuccess) return e;
    for (size_t k = 0; k < b->jobs.size(); ++k) {
        const acf_job &J = b->jobs[k];
        cudaStream_t sk = b->aux[b->aux_of[k]];
        if (b->T[k] == 0 || !tc_plan_job_stores(b->plan, (int)k))
            if ((e = cudaMemsetAsync(outputs[k], 0, b->v_bytes[k], sk)) != cudaSuccess) return e;
        if (b->T[k] == 0) continue;
        if (J.n_channels == 1) {
            e = launch_transpose_raw(inputs[k], J.n_samples, ACF_IN_CI8, 1, J.n_inputs, OUT_F16, b->X[k], nullptr,
                                     b->t_stride[k], 1.f, sk);
        } else {
            e = launch_channelise(nullptr, 0, inputs[k], J.n_samples, ACF_IN_CI8, 1, J.n_inputs, J.n_channels, J.n_taps,
                                  b->d_h[(long)J.n_taps * 1024 + J.n_channels], b->d_bp[J.n_channels],
                                  b->d_tw[J.n_channels], OUT_F16X3, b->X[k], b->Xlo[k], b->t_stride[k], b->scale[k],
                                  b->T[k], sk, b->cturn[k], b->cturn_bytes[k]);
        }
        if (e != cudaSuccess) return e;
    }
    for (int a = 0; a < acf_batch::kAux; ++a) {
        if ((e = cudaEventRecord(b->aux_done[a], b->aux[a])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, b->aux_done[a], 0)) != cudaSuccess) return e;
    }
    return tc_plan_launch(b->plan, s);
}

// Jobs to auxiliary streams: longest preparation first onto the least-loaded
// stream (cost ~ samples x inputs, x4 for a filter bank).
static void assign_aux(acf_batch *b)
{
    const size_t n = b->jobs.size();
    std::vector<int> order(n);
    std::vector<double> cost(n);
    for (size_t k = 0; k < n; ++k) {
        order[k] = (int)k;
        cost[k] = (double)b->jobs[k].n_samples * b->jobs[k].n_inputs * (b->jobs[k].n_channels > 1 ? 4.0 : 1.0);
    }
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    double load[acf_batch::kAux] = {};
    b->aux_of.assign(n, 0);
    for (int k : order) {
        int best = 0;
        for (int a = 1; a < acf_batch::kAux; ++a)
            if (load[a] < load[best]) best = a;
        b->aux_of[k] = best;
        load[best] += cost[k];
    }
}

static cudaError_t rebuild_plan(acf_batch *b, void *const *outputs, const TcTuning &tun)
{
    if (b->plan) {
        tc_plan_destroy(b->plan);
        b->plan = nullptr;
    }
    std::vector<TcJob> js = tc_jobs(b, outputs);
    std::string perr;
    cudaError_t e = tc_plan_create(js.data(), (int)js.size(), tun, &b->plan, &perr);
    if (e != cudaSuccess) b->err = "tensor-core plan: " + perr;
    return e;
}

static void autotune(acf_batch *b)
{
    // scratch outputs for timing
    std::vector<void *> outs(b->jobs.size(), nullptr);
    for (size_t k = 0; k < outs.size(); ++k)
        if (cudaMalloc(&outs[k], b->v_bytes[k]) != cudaSuccess) {
            for (void *p : outs) cudaFree(p);
            cudaGetLastError();
            return;
        }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TcTuning best_t = b->tun;
    for (int pair : {1, 0})
    for (int nt : {256, 128})
        for (int ks : {1, 2, 4})
            for (int order : {2, 1, 0}) {
                if (pair && nt == 128) continue;   // the pair kernel always uses 256-row tiles
                TcTuning t;
                t.pair = pair;
                t.n_tile = nt;
                t.k_split = ks;
                t.order = order;
                if (rebuild_plan(b, outs.data(), t) != cudaSuccess) continue;
                tc_plan_launch(b->plan, b->s_int);   // warm-up
                cudaEventRecord(e0, b->s_int);
                for (int r = 0; r < 3; ++r) tc_plan_launch(b->plan, b->s_int);
                cudaEventRecord(e1, b->s_int);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_t = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tun = best_t;
    for (void *p : outs) cudaFree(p);
    if (b->plan) {
        tc_plan_destroy(b->plan);
        b->plan = nullptr;
    }
}

extern "C" {

acf_status acf_batch_create(acf_batch **out, const acf_job *jobs, int n_jobs, int tune)
{
    if (!out) return bf(nullptr, ACF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!jobs || n_jobs < 1 || n_jobs > 64) return bf(nullptr, ACF_EINVAL, "need 1..64 jobs");
    for (int k = 0; k < n_jobs; ++k) {
        const acf_job &J = jobs[k];
        const bool cok = J.n_channels == 1 || J.n_channels == 16 || J.n_channels == 64 || J.n_channels == 256;
        if (J.n_inputs < 1 || J.n_inputs > 65536 || !cok || J.n_taps < 1 || J.n_taps > 32 ||
            (J.n_channels == 1 && J.n_taps != 1) || J.n_samples < 1 || J.n_samples > (1L << 30))
            return bf(nullptr, ACF_EINVAL, "job " + std::to_string(k) + ": bad geometry");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bf(nullptr, ACF_ECUDA, "cudaGetDevice failed");
    if (!tc_supported(dev)) return bf(nullptr, ACF_EUNSUPPORTED, "the batch runs on sm_103 tensor cores");
    acf_batch *b = new acf_batch();
    b->jobs.assign(jobs, jobs + n_jobs);
    cudaError_t e = cudaSuccess;
    auto cleanup = [&](acf_status s, const std::string &m) {
        acf_batch_destroy(b);
        return bf(nullptr, s, m);
    };
    for (int k = 0; k < n_jobs; ++k) {
        const acf_job &J = jobs[k];
        const bool raw = J.n_channels == 1;
        const long T = raw ? J.n_samples : spectra_of(J.n_samples, J.n_taps, J.n_channels);
        const long ts = round_up(std::max<long>(T, 1), 64);
        const size_t xb = (size_t)J.n_channels * 2 * J.n_inputs * ts * 2;
        void *x = nullptr, *xl = nullptr;
        if ((e = cudaMalloc(&x, xb)) != cudaSuccess) return cleanup(ACF_ENOMEM, "operand alloc");
        b->X.push_back(x);
        if (!raw) {
            if ((e = cudaMalloc(&xl, xb)) != cudaSuccess) return cleanup(ACF_ENOMEM, "operand alloc");
        }
        b->Xlo.push_back(xl);
        cudaMemset(x, 0, xb);
        if (xl) cudaMemset(xl, 0, xb);
        b->T.push_back(T);
        b->t_stride.push_back(ts);
        void *ct = nullptr;
        size_t ctb = 0;
        if (chan256_supported(ACF_IN_CI8, J.n_channels, J.n_taps, ts)) {
            ctb = chan256_scratch_bytes(ACF_IN_CI8, 1, J.n_inputs, 0, J.n_samples);
            if ((e = cudaMalloc(&ct, ctb)) != cudaSuccess) return cleanup(ACF_ENOMEM, "corner-turn scratch");
        }
        b->cturn.push_back(ct);
        b->cturn_bytes.push_back(ctb);
        b->v_bytes.push_back((size_t)J.n_channels * n_baselines(J.n_inputs) * (raw ? 16 : 8));
        float sc = 1.f;
        if (!raw) {
            const long key = (long)J.n_taps * 1024 + J.n_channels;
            std::vector<float> h;
            prototype_host(J.n_taps, J.n_channels, h);
            if (!b->d_h.count(key)) {
                float *d = nullptr;
                if ((e = cudaMalloc(&d, sizeof(float) * h.size())) != cudaSuccess) return cleanup(ACF_ENOMEM, "alloc");
                cudaMemcpy(d, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice);
                b->d_h[key] = d;
            }
            if (!b->d_tw.count(J.n_channels)) {
                float2 *tw = nullptr;
                if ((e = make_twiddles(J.n_channels, &tw)) != cudaSuccess) return cleanup(ACF_ENOMEM, "alloc");
                b->d_tw[J.n_channels] = tw;
                std::vector<float> ones(J.n_channels, 1.f);
                float *d = nullptr;
                if ((e = cudaMalloc(&d, sizeof(float) * J.n_channels)) != cudaSuccess) return cleanup(ACF_ENOMEM, "alloc");
                cudaMemcpy(d, ones.data(), sizeof(float) * J.n_channels, cudaMemcpyHostToDevice);
                b->d_bp[J.n_channels] = d;
            }
            double sabs = 0;
            for (float v : h) sabs += std::fabs((double)v);
            sc = std::ldexp(1.f, (int)std::floor(std::log2(60000.0 / (2.0 * sabs * 128.0))));
        }
        b->scale.push_back(sc);
    }
    if (!device_error_word()) return cleanup(ACF_ENOMEM, "device error word");
    if ((e = cudaStreamCreateWithFlags(&b->s_int, cudaStreamNonBlocking)) != cudaSuccess) return cleanup(ACF_ECUDA, "stream");
    cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (int a = 0; a < acf_batch::kAux; ++a) {
        if ((e = cudaStreamCreateWithFlags(&b->aux[a], cudaStreamNonBlocking)) != cudaSuccess)
            return cleanup(ACF_ECUDA, "aux stream");
        cudaEventCreateWithFlags(&b->aux_done[a], cudaEventDisableTiming);
    }
    assign_aux(b);
    if (tune) autotune(b);
    if (cudaDeviceSynchronize() != cudaSuccess) return cleanup(ACF_ECUDA, "device error during planning");
    *out = b;
    return ACF_OK;
}

acf_status acf_batch_run(acf_batch *b, const void *const *inputs, void *const *outputs, acf_stream_t stream)
{
    if (!b) return ACF_EINVAL;
    if (!inputs || !outputs) return bf(b, ACF_EINVAL, "inputs / outputs is NULL");
    const size_t n = b->jobs.size();
    for (size_t k = 0; k < n; ++k)
        if (!inputs[k] || !outputs[k]) return bf(b, ACF_EINVAL, "NULL input or output for job " + std::to_string(k));
    cudaError_t e;
    const bool same = b->gexec && std::equal(b->g_in.begin(), b->g_in.end(), inputs) &&
                      std::equal(b->g_out.begin(), b->g_out.end(), outputs);
    if (!same) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        if ((e = rebuild_plan(b, outputs, b->tun)) != cudaSuccess) return bf(b, ACF_ECUDA, b->err);
        cudaGraph_t g = nullptr;
        const long long before = g_launches.load();
        if ((e = cudaStreamBeginCapture(b->s_int, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bf(b, ACF_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        cudaError_t eq = enqueue_all(b, inputs, outputs, b->s_int);
        e = cudaStreamEndCapture(b->s_int, &g);
        b->graph_kernels = g_launches.load() - before;
        g_launches -= b->graph_kernels;   // captured, not launched
        if (eq != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return bf(b, ACF_ECUDA, std::string("capture: ") + cudaGetErrorString(eq != cudaSuccess ? eq : e));
        }
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bf(b, ACF_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        b->g_in.assign(inputs, inputs + n);
        b->g_out.assign(outputs, outputs + n);
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEventRecord(b->ev_in, s);
    cudaStreamWaitEvent(b->s_int, b->ev_in, 0);
    if ((e = cudaGraphLaunch(b->gexec, b->s_int)) != cudaSuccess)
        return bf(b, ACF_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    g_launches += b->graph_kernels;
    cudaEventRecord(b->ev_out, b->s_int);
    cudaStreamWaitEvent(s, b->ev_out, 0);
    return ACF_OK;
}

acf_status acf_batch_query(const acf_batch *b, int *n_tile, int *k_split, int *n_items)
{
    if (!b) return ACF_EINVAL;
    if (n_tile) *n_tile = b->tun.n_tile;
    if (k_split) *k_split = b->tun.k_split;
    if (n_items) *n_items = b->plan ? tc_plan_items(b->plan) : 0;
    return ACF_OK;
}

acf_status acf_batch_query_plan(const acf_batch *b, int *pair, int *order)
{
    if (!b) return ACF_EINVAL;
    if (pair) *pair = b->tun.pair;
    if (order) *order = b->tun.order;
    return ACF_OK;
}

acf_status acf_batch_set_plan(acf_batch *b, int pair, int n_tile, int k_split, int order)
{
    if (!b) return ACF_EINVAL;
    if ((pair != 0 && pair != 1) || (n_tile != 128 && n_tile != 256) || (pair && n_tile != 256) ||
        (k_split != 1 && k_split != 2 && k_split != 4) || order < 0 || order > 2)
        return bf(b, ACF_EINVAL, "plan: pair 0/1 (pair needs n_tile 256), n_tile 128/256, k_split 1/2/4, order 0..2");
    cudaDeviceSynchronize();
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->tun.pair = pair;
    b->tun.n_tile = n_tile;
    b->tun.k_split = k_split;
    b->tun.order = order;
    return ACF_OK;
}

acf_status acf_batch_destroy(acf_batch *b)
{
    if (!b) return ACF_OK;
    cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->plan) tc_plan_destroy(b->plan);
    for (void *p : b->X) cudaFree(p);
    for (void *p : b->Xlo) cudaFree(p);
    for (void *p : b->cturn) cudaFree(p);
    for (auto &kv : b->d_h) cudaFree(kv.second);
    for (auto &kv : b->d_tw) cudaFree(kv.second);
    for (auto &kv : b->d_bp) cudaFree(kv.second);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (int a = 0; a < acf_batch::kAux; ++a) {
        if (b->aux_done[a]) cudaEventDestroy(b->aux_done[a]);
        if (b->aux[a]) cudaStreamDestroy(b->aux[a]);
    }
    if (b->s_int) cudaStreamDestroy(b->s_int);
    delete b;
    cudaGetLastError();
    return ACF_OK;
}

const char *acf_batch_last_error(const acf_batch *b) { return b ? b->err.c_str() : g_batch_create_err.c_str(); }

}  // extern "C"
