// C ABI of libbigmeans (include/bigmeans.h): argument checks, workspace
// layout, and the launch sequence of Algorithm 1 (arXiv 2403.18766):
//
//   prepass(X)                  validate, largest |x| -> fixed-point grids
//   worker kernel (rounds)      one cluster per worker: Alg. 1 rounds
//   [full pass, incumbent]      optional, after every round
//   worker kernel (final eval)  common sample of size s_opt, f_hat_w for all w
//   full pass                   labels and f(C_best, X)
//
// Everything is enqueued on the caller's stream; each entry point
// synchronises that stream once before returning.
#include <algorithm>
#include <mutex>
#include <map>
#include <atomic>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_device.cuh"
#include "bm_sample.cuh"
#include "bm_worker.cuh"

namespace bm {
size_t worker_smem(int np, int k);
cudaError_t launch_worker(int np, const WorkerArgs& a, int clusters, cudaStream_t st);
size_t fullpass_smem_bytes(int np, int k, int n);
cudaError_t launch_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                            const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                            int incumbent, int grid, cudaStream_t st);
cudaError_t launch_prepass(const float* v, long long count, Globals* g, int grid, cudaStream_t st);
cudaError_t launch_pad(const float* src, long long rows, int n, int np, float* dst, cudaStream_t st);
cudaError_t launch_unpad(const float* src, long long rows, int n, int np, float* dst, cudaStream_t st);
cudaError_t launch_select_unpad(const float* Cw, const double* sel_f, int W, int k, int n, int np,
                                float* dst, cudaStream_t st);
cudaError_t launch_init_state(double* fhat, int W, unsigned char* deg, long long kdeg, Globals* g,
                              cudaStream_t st);
cudaError_t launch_globaltimer(unsigned long long* out, cudaStream_t st);
size_t tc_smem_bytes(int k);
cudaError_t launch_pack_bf16(const float* X, long long m, int n, long long m_pad, void* Xb, float* norms,
                             cudaStream_t st);
void set_fullpass_impl(int impl);
int last_fullpass_impl();
int fullpass_impl_setting();
bool tcx_eligible(const float* X, long long m, int n, int np, int k);
void set_tcx_wait_limit(unsigned polls, unsigned ns);
cudaError_t launch_tc_fullpass(const void* Xb, const float* xnorm, const float* Xf, long long m, int n,
                               const float* C, int k, float tau, int certify, int* labels, void* queue, Globals* g,
                               float gp2, int sms, cudaStream_t st);
}  // namespace bm

using namespace bm;

namespace {
thread_local std::string g_err;
}  // namespace

namespace bm {
// Record the thread-local message returned by bm_last_error (for other
// translation units of the library).
bm_status set_error(bm_status s, const char* msg) {
    g_err = msg;
    return s;
}
}  // namespace bm

namespace {

bm_status fail(bm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? BM_ENOMEM : BM_ECUDA,           \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

constexpr size_t kSmemLimit = 227 * 1024;
constexpr int kRowsPerCta = 1024;
constexpr int kMaxGroupWorkers = 64;     // workers of a fit that may form groups
constexpr int kGroupCs = 8;              // CTAs per cluster of a grouped launch

int padded_dim(int n) {
    if (n <= 4) return 4;
    if (n <= 8) return 8;
    if (n <= 16) return 16;
    if (n <= 32) return 32;
    return 64;
}

int sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// The library's own stream-ordered memory pool on the current device: freed
// memory stays in the pool (release threshold: never) and is reused by the
// next fit without being mapped again.  bm_trim_memory returns it.
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t lib_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) { *out = it->second; return cudaSuccess; }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    g_pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

// Test hook (bm_debug_fail_allocs): the next N device allocations of the
// library fail as if the device were out of memory.
std::atomic<int> g_fail_allocs{0};

cudaError_t lib_alloc(void** p, size_t bytes, cudaStream_t st) {
    for (int left = g_fail_allocs.load(); left > 0;)
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = lib_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// gamma_q = q u / (1 - q u), u = 2^-24, rounded up to float.
float gamma_up(int q) {
    const double u = std::ldexp(1.0, -24);
    const double gq = q * u / (1.0 - q * u);
    return std::nextafter((float)gq, INFINITY);
}
void cert_constants(int np, float& gB, float& gp2) {
    gB = std::nextafter(gamma_up(2 * np + 2) * (1.0f + 1e-6f), INFINITY);
    const double g2 = 2.0 * (1.0 + std::ldexp(1.0, -14)) * (double)gamma_up(np + 2);
    gp2 = std::nextafter((float)g2 * (1.0f + 1e-6f), INFINITY);
}

// Expected and safe number of bounded draws to collect s distinct values of m.
long long draw_cap(long long m, long long s) {
    double mean = 0.0, var = 0.0;
    if (s <= m / 2) {
        // each draw is new with probability >= 1/2: mean <= 2 s, tiny variance
        for (long long i = 0; i < s; i += 1 + s / 4096) {
            const double p = (double)(m - i) / (double)m;
            const long long cnt = std::min<long long>(1 + s / 4096, s - i);
            mean += cnt / p;
            var += cnt * (1.0 - p) / (p * p);
        }
    } else {
        for (long long i = 0; i < s; ++i) {
            const double p = (double)(m - i) / (double)m;
            mean += 1.0 / p;
            var += (1.0 - p) / (p * p);
        }
    }
    const double cap = mean + 8.0 * std::sqrt(var) + 1024.0 + 0.05 * mean;
    return (long long)std::ceil(cap);
}

// Target sample rows per CTA of a worker cluster (the tile the autotuner
// chooses; results do not depend on it: every reduction is exact).
std::atomic<int> g_rows_per_cta{kRowsPerCta};
// 1: workers whose cluster is at the size cap and still above the tile run
// with 512-thread CTAs (twice the warps per SM for the longest workers).
std::atomic<int> g_big_tpb{0};
std::atomic<int> g_sample_tables{0};
// 1: no groups (every worker is one cluster, as in a non-cooperative launch)
std::atomic<int> g_no_groups{0};
// Fits created on this thread may use groups (the serving runners turn it
// off: a cooperative launch sized for the whole device would wait for the
// other jobs' kernels to drain, which defeats running jobs side by side).
thread_local bool t_groups_ok = true;

// Most sample rows one worker CTA can take: kMaxRowsPerCta, and the label
// buckets of a Lloyd run (4 bytes per row) must fit beside the worker's
// shared memory.
long long rows_cap(int np, int k) {
    const long long room = ((long long)kSmemLimit - (long long)worker_smem(np, k)) / 4 - 16;
    return std::max<long long>(0, std::min<long long>(kMaxRowsPerCta, room));
}

// CTAs per worker cluster: about rows_per_cta sample rows per CTA, at most
// max_cs, and never more than `cap` rows per CTA (0 = impossible).
int cluster_size(long long s_cap, int max_cs, int rows_per_cta, long long cap) {
    const long long rpc = rows_per_cta > 0 ? rows_per_cta : g_rows_per_cta.load();
    long long cs = std::max<long long>(1, (s_cap + rpc - 1) / rpc);
    cs = std::min<long long>(cs, max_cs);
    while (cs < max_cs && (s_cap + cs - 1) / cs > cap) ++cs;
    if ((s_cap + cs - 1) / cs > cap) return 0;
    return (int)cs;
}

long long next_pow2(long long v) {
    long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

namespace bm {
void set_thread_groups(bool ok) { t_groups_ok = ok; }
}  // namespace bm

struct bm_fit_ctx {
    cudaStream_t st = nullptr;
    const float* X = nullptr;
    long long m = 0;
    int n = 0, k = 0, np = 0, cs = 1;
    bm_sample_policy pol{};
    bm_budget bud{};
    unsigned long long seed = 0;
    long long s_lo = 0, s_hi = 0, s_cap = 0, Tcap = 0, H = 0, L_cap = 0;
    size_t smem = 0;
    float gB = 0, gp2 = 0;
    int rounds_run = 0;
    unsigned long long t0_gpu = 0;
    std::chrono::steady_clock::time_point t0;
    // device buffers
    void* base = nullptr;
    Globals* glob = nullptr;
    int jobs = 0;                           // sample jobs per round: W * (P + 1)
    int prefetched = -1;                    // round whose samples were drawn ahead
    int rows_per_cta = 0;                   // cluster tile of this fit (fixed at create)
    long long L_sum0 = 0, L_len0 = 0;       // L at the start of the current round (exploit policy)
    int rounds_planned = 0x7fffffff;        // rounds the caller intends to run (T)
    cudaStream_t sst = nullptr;             // sampling stream (draws the next round ahead)
    cudaEvent_t ev_sdone = nullptr;
    unsigned int gen = 1;                   // next sampler-table generation
    float* S = nullptr; long long* idx = nullptr; unsigned int* draws = nullptr;
    unsigned long long* table = nullptr; int* job_s = nullptr; float* D2 = nullptr; int* lab = nullptr;
    float* Cw = nullptr; float* Cw_cta = nullptr; unsigned char* deg = nullptr;
    double* fhat = nullptr; double* f_final = nullptr; long long* L_buf = nullptr;
    unsigned long long* timer = nullptr;
    // group exchange of workers that span several clusters (null: no groups)
    long long* xpart = nullptr; int* xcnt = nullptr; unsigned long long* xobj = nullptr;
    unsigned* xbar = nullptr; float* xC = nullptr; int* xflag = nullptr;
    int max_cs = 8;
    cudaEvent_t ev_fork = nullptr;
    // phase timing: event pairs around each launch, summed when the stream syncs
    struct Span { cudaEvent_t a, b; int kind; cudaStream_t st; bool ended; };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> pool;
    double t_worker = 0, t_full = 0, t_sample = 0;
    long long n_worker = 0, n_full = 0;
    long long n_kernels = 0;                // kernels of this library launched so far
    int last_groups = 0;                    // clusters of the last grouped round launch (0: not grouped)
    bool groups_ok = true;                  // groups allowed for this fit (creating thread's setting)
    int w_lo = 0, w_hi = 0;                 // workers this context runs (a shard of a fit: [w_lo, w_hi))
};

namespace {

SizePolicy size_policy(const bm_fit_ctx* c) {
    SizePolicy p;
    memset(&p, 0, sizeof p);
    p.s_min = c->pol.s_min;
    p.s_hi = c->s_hi;
    for (int i = 0; i < 16; ++i) p.set[i] = c->pol.set[i];
    p.set_len = c->pol.set_len;
    p.kind = c->pol.kind;
    p.exploit = c->pol.exploit;
    p.L_sum = c->L_sum0;
    p.L_len = c->L_len0;
    return p;
}

WorkerArgs make_args(const bm_fit_ctx* c, int mode, int parity = 0) {
    WorkerArgs a;
    memset(&a, 0, sizeof a);
    a.X = c->X; a.m = c->m; a.n = c->n; a.k = c->k;
    a.s_min = c->pol.s_min; a.s_max = c->s_hi;
    for (int i = 0; i < 16; ++i) a.set[i] = c->pol.set[i];
    a.set_len = c->pol.set_len;
    a.W = c->pol.workers; a.P = c->pol.passes;
    a.max_lloyd = c->bud.max_lloyd; a.trials = c->bud.kpp_candidates; a.tol = c->bud.tol;
    a.seed = c->seed;
    a.mode = mode; a.cs = c->cs; a.glob = c->glob;
    a.S_stride = c->s_cap * c->np;
    a.S = c->S + (long long)parity * c->jobs * a.S_stride;
    a.job_s = c->job_s + (long long)parity * c->jobs;
    a.D2 = c->D2; a.D2_stride = c->s_cap; a.lab = c->lab;
    a.Cw = c->Cw; a.Cw_cta = c->Cw_cta; a.deg = c->deg; a.fhat = c->fhat;
    a.L_buf = c->L_buf; a.L_cap = c->L_cap; a.f_final = c->f_final;
    a.gB = c->gB; a.gp2 = c->gp2;
    a.xpart = c->xpart; a.xcnt = c->xcnt; a.xobj = c->xobj;
    a.xbar = c->xbar; a.xabort = c->xbar ? reinterpret_cast<int*>(c->xbar + c->pol.workers) : nullptr;
    a.xC = c->xC; a.xflag = c->xflag;
    return a;
}

SampleArgs make_sample_args(bm_fit_ctx* c, int mode, int jobs, int parity = 0) {
    SampleArgs a;
    memset(&a, 0, sizeof a);
    a.X = c->X; a.m = c->m; a.n = c->n; a.mode = mode; a.seed = c->seed;
    a.W = c->pol.workers; a.P = c->pol.passes;
    a.s_min = c->pol.s_min; a.s_max = c->s_hi;
    for (int i = 0; i < 16; ++i) a.set[i] = c->pol.set[i];
    a.set_len = c->pol.set_len;
    a.sp = size_policy(c);
    // first job of this buffer half, and of the context's first worker (a
    // shard draws only its own workers' samples, into their usual slots)
    const long long J = (long long)parity * c->jobs +
                        ((mode == kSampleRound) ? (long long)c->w_lo * (c->pol.passes + 1) : 0);
    a.worker_base = (mode == kSampleRound) ? c->w_lo : 0;
    a.S_stride = c->s_cap * c->np; a.S = c->S + J * a.S_stride;
    a.idx_stride = c->s_cap; a.idx = c->idx + J * a.idx_stride;
    a.draws_stride = c->Tcap; a.draws = c->draws + J * a.draws_stride; a.Tcap = c->Tcap;
    a.H = c->H; a.table_stride = c->H; a.table = c->table + J * a.table_stride;
    a.gen_base = c->gen;
    c->gen += (unsigned int)jobs;
    // shared-memory bitmap of the m values when it fits in one CTA
    const long long words = (c->m + 31) / 32;
    const size_t sb = sample_smem_bytes((int)std::min<long long>(words, 1 << 30));
    if (mode != kSampleGather && !g_sample_tables.load() && words <= (1 << 30) && sb <= 200 * 1024)
        a.bitmap_words = (int)words;
    a.job_s = c->job_s + J; a.glob = c->glob;
    return a;
}

cudaEvent_t take_event(bm_fit_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
// Record the start of a timed launch; returns the span index.
size_t span_begin(bm_fit_ctx* c, int kind, cudaStream_t st = nullptr) {
    if (!st) st = c->st;
    bm_fit_ctx::Span sp{take_event(c), take_event(c), kind, st, false};
    cudaEventRecord(sp.a, st);
    c->spans.push_back(sp);
    return c->spans.size() - 1;
}
void span_end(bm_fit_ctx* c, size_t i) {
    if (i >= c->spans.size()) return;
    cudaEventRecord(c->spans[i].b, c->spans[i].st);
    c->spans[i].ended = true;
}
// After a stream sync: fold the finished spans into the phase totals.
// Spans on other streams (the sampling stream) may still be running: those
// stay queued until they complete.
void collect_spans(bm_fit_ctx* c) {
    std::vector<bm_fit_ctx::Span> pending;
    for (auto& sp : c->spans) {
        if (!sp.ended) {                       // still open (its end is not recorded yet)
            pending.push_back(sp);
            continue;
        }
        float ms = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&ms, sp.a, sp.b);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            pending.push_back(sp);
            continue;
        }
        if (e != cudaSuccess) cudaGetLastError();   // a span that cannot be timed is dropped
        if (e == cudaSuccess) {
            if (sp.kind == 0) { c->t_worker += ms * 1e-3; c->n_worker++; }
            else if (sp.kind == 2) { c->t_sample += ms * 1e-3; }
            else { c->t_full += ms * 1e-3; c->n_full++; }
        }
        c->pool.push_back(sp.a);
        c->pool.push_back(sp.b);
    }
    c->spans.swap(pending);
}

// Carve one device allocation into the workspace: per sample job (W * (P+1)
// per round, two rounds' worth so the next round is drawn while this one
// runs) the padded sample, its indices, draws and sampler table; per worker
// the K-means++ D^2, labels, centroids and state.
// Device bytes of a fit's workspace (the layout of alloc_workspace).
// Bytes of the group exchange buffers, 0 when the fit cannot use groups
// (more workers than a cooperative launch can hold clusters, or too large).
size_t group_bytes(const bm_fit_ctx* c, int W) {
    if (W > kMaxGroupWorkers) return 0;
    const size_t part = (size_t)W * 2 * kMaxGroup * c->k * c->np * kAccWords * 8;
    if (part > ((size_t)256 << 20)) return 0;
    return part;
}

size_t workspace_bytes(const bm_fit_ctx* c, int W) {
    const long long k = c->k, np = c->np;
    const long long J = 2ll * W * (c->pol.passes + 1);
    size_t off = 0;
    auto take = [&](size_t bytes) { off += (bytes + 255) & ~(size_t)255; };
    if (const size_t gb = group_bytes(c, W)) {
        take(gb);
        take((size_t)W * 2 * kMaxGroup * k * 4);
        take((size_t)W * 2 * kMaxGroup * 4 * 8);
        take((size_t)W * 2 * 4);
        take((size_t)W * k * np * 4);
        take((size_t)W * 2 * 4);
    }
    take(sizeof(Globals));
    take((size_t)J * c->s_cap * np * 4);
    take((size_t)J * c->s_cap * 8);
    take((size_t)J * c->Tcap * 4);
    take((size_t)J * c->H * 8);
    take((size_t)J * 4);
    take((size_t)W * c->s_cap * 4);
    take((size_t)W * c->s_cap * 4);
    take((size_t)W * k * np * 4);
    take((size_t)W * kMaxCluster * k * np * 4);
    take((size_t)W * k);
    take((size_t)W * 8);
    take((size_t)W * 8);
    take((size_t)c->L_cap * 8);
    take(8);
    return off;
}

bm_status alloc_workspace(bm_fit_ctx* c, int W) {
    const long long k = c->k, np = c->np;
    c->jobs = W * (c->pol.passes + 1);
    const long long J = 2ll * c->jobs;                  // two halves: this round, next round
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t o_glob = take(sizeof(Globals));
    const size_t o_S = take((size_t)J * c->s_cap * np * 4);
    const size_t o_idx = take((size_t)J * c->s_cap * 8);
    const size_t o_draws = take((size_t)J * c->Tcap * 4);
    const size_t o_tab = take((size_t)J * c->H * 8);
    const size_t o_js = take((size_t)J * 4);
    const size_t o_D2 = take((size_t)W * c->s_cap * 4);
    const size_t o_lab = take((size_t)W * c->s_cap * 4);
    const size_t o_Cw = take((size_t)W * k * np * 4);
    const size_t o_Cwc = take((size_t)W * kMaxCluster * k * np * 4);
    const size_t o_deg = take((size_t)W * k);
    const size_t o_fhat = take((size_t)W * 8);
    const size_t o_ff = take((size_t)W * 8);
    const size_t o_L = take((size_t)c->L_cap * 8);
    const size_t o_t = take(8);
    const size_t gb = group_bytes(c, W);
    size_t o_xp = 0, o_xc = 0, o_xo = 0, o_xb = 0, o_xC = 0, o_xf = 0;
    if (gb) {
        o_xp = take(gb);
        o_xc = take((size_t)W * 2 * kMaxGroup * k * 4);
        o_xo = take((size_t)W * 2 * kMaxGroup * 4 * 8);
        o_xb = take((size_t)W * 2 * 4);
        o_xC = take((size_t)W * k * np * 4);
        o_xf = take((size_t)W * 2 * 4);
    }
    cudaError_t e = lib_alloc(&c->base, off, c->st);
    if (e != cudaSuccess) {
        c->base = nullptr;
        cudaGetLastError();
        return fail(BM_ENOMEM, "workspace of %zu bytes: %s", off, cudaGetErrorString(e));
    }
    char* b = (char*)c->base;
    c->glob = (Globals*)(b + o_glob);
    c->S = (float*)(b + o_S); c->idx = (long long*)(b + o_idx); c->draws = (unsigned int*)(b + o_draws);
    c->table = (unsigned long long*)(b + o_tab); c->job_s = (int*)(b + o_js);
    c->D2 = (float*)(b + o_D2); c->lab = (int*)(b + o_lab); c->Cw = (float*)(b + o_Cw); c->Cw_cta = (float*)(b + o_Cwc);
    c->deg = (unsigned char*)(b + o_deg); c->fhat = (double*)(b + o_fhat); c->f_final = (double*)(b + o_ff);
    c->L_buf = (long long*)(b + o_L); c->timer = (unsigned long long*)(b + o_t);
    if (gb) {
        c->xpart = (long long*)(b + o_xp); c->xcnt = (int*)(b + o_xc);
        c->xobj = (unsigned long long*)(b + o_xo); c->xbar = (unsigned*)(b + o_xb);
        c->xC = (float*)(b + o_xC); c->xflag = (int*)(b + o_xf);
    }
    CU(cudaMemsetAsync(c->glob, 0, sizeof(Globals), c->st));
    CU(cudaMemsetAsync(c->Cw, 0, (size_t)W * k * np * 4, c->st));
    CU(cudaMemsetAsync(c->table, 0, (size_t)J * c->H * 8, c->st));
    CU(cudaMemsetAsync(c->job_s, 0, (size_t)J * 4, c->st));
    return BM_OK;
}

bm_status check_ptr(const void* p, const char* what) {
    if (!p) return fail(BM_EINVAL, "%s is NULL", what);
    if (((uintptr_t)p) & 15) return fail(BM_EINVAL, "%s is not 16-byte aligned", what);
    return BM_OK;
}

// Size checks shared by the fit and the step entry points (the worker's
// shared-memory accumulators bound k * n unless only the full pass runs).
bm_status check_shape(long long m, int n, int k, bool worker = true) {
    if (m < 1 || m >= (1ll << 31)) return fail(BM_EINVAL, "m = %lld out of range [1, 2^31)", m);
    if (n < 1 || n > 64) return fail(BM_EINVAL, "n = %d out of range [1, 64]", n);
    if (k < 1) return fail(BM_EINVAL, "k = %d must be >= 1", k);
    if (!worker) return BM_OK;
    const size_t smem = worker_smem(padded_dim(n), k);
    if (smem > kSmemLimit)
        return fail(BM_EINVAL, "k = %d with n = %d needs %zu bytes of shared memory (limit %zu)", k, n,
                    smem, kSmemLimit);
    return BM_OK;
}

bm_status read_globals(bm_fit_ctx* c, Globals* h) {
    CU(cudaMemcpyAsync(h, c->glob, sizeof(Globals), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    collect_spans(c);
    return BM_OK;
}

void fill_report(const bm_fit_ctx* c, const Globals& h, bm_report* rep) {
    memset(rep, 0, sizeof *rep);
    rep->f_full = h.f_full;
    rep->f_incumbent = std::min(h.f_incumbent, h.f_full);
    rep->s_opt = h.s_opt;
    rep->best_worker = h.best_worker;
    rep->rounds_done = c->rounds_run;
    rep->passes_done = (int64_t)h.passes;
    rep->lloyd_iters = (int64_t)h.lloyd_iters;
    rep->assign_rows = (int64_t)h.assign_rows;
    rep->accepts = (int64_t)h.accepts;
    rep->L_sum = (int64_t)h.L_sum;
    rep->rescored_rows = (int64_t)h.rescored;
    rep->inexact_terms = (int64_t)h.inexact;
    rep->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - c->t0).count();
    rep->t_worker_s = c->t_worker;
    rep->t_fullpass_s = c->t_full;
    rep->kernel_launches = c->n_kernels;
    rep->fullpass_launches = c->n_full;
    rep->reseeded = (int64_t)h.reseeded;
    for (int i = 0; i < 16; ++i) rep->trace_cycles[i] = (int64_t)h.trace[i];
    rep->t_sample_s = c->t_sample;
}

}  // namespace

namespace bm {
// Status of a call from the device flags it left in its Globals record (also
// used by bm_assign_noalloc, so that both entry points report a failure alike).
bm_status status_from_flags(const Globals& h) {
    if (h.nonfinite) return fail(BM_EINVAL, "X contains %u non-finite values", h.nonfinite);
    if (h.maxbits >= 0x7e800000u)
        return fail(BM_EINVAL, "max |x| must be below 2^126");
    if (h.err & kErrSample) return fail(BM_EINTERNAL, "sampler needed more draws than its cap");
    if (h.err & kErrDigits) return fail(BM_EINTERNAL, "fixed-point accumulator range exceeded");
    if (h.err & kErrTimeout) return fail(BM_ETIMEOUT, "a bounded device wait gave up");
    if (h.err & kErrArgs) return fail(BM_EINVAL, "an index was outside [0, m) or a device consistency check failed");
    if (h.err) return fail(BM_EINTERNAL, "device error flags 0x%x", h.err);
    return BM_OK;
}
}  // namespace bm

namespace {

long long size_of(const bm_fit_ctx* c, int w, int t) {
    return policy_size(size_policy(c), c->seed, stream_k1(kPurposeSize, w, t, 0));
}

bm_status ensure_streams(bm_fit_ctx* c) {
    if (c->sst) return BM_OK;
    int lo_prio = 0, hi_prio = 0;
    CU(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    CU(cudaStreamCreateWithPriority(&c->sst, cudaStreamNonBlocking, lo_prio));
    CU(cudaEventCreateWithFlags(&c->ev_sdone, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    return BM_OK;
}

// The launch plan of one round: every worker of the fits in one launch.
//  * Groups (cooperative launch, clusters of 8 CTAs, or 4 when there are
//    more workers than resident clusters of 8): when every worker gets a
//    cluster and the whole grid can be resident at once, the clusters left
//    over go, one at a time, to the worker with the most sample rows per
//    CTA, so a large sample spreads over several clusters (up to kMaxGroup)
//    that add up their exact partial sums in global memory; rows per CTA
//    then stay about equal across workers.
//  * Otherwise (more workers than resident clusters, groups disabled or
//    unavailable, or 512-thread CTAs requested): one cluster per worker, all
//    of one size (for the largest sample), launched together; clusters that
//    do not fit at once start as others finish (they never wait on one
//    another).
// Clusters are ordered by decreasing sample size.  Returns the clusters.
struct PlanItem { int fit; int w; long long s; };

int plan_launch(const std::vector<bm_fit_ctx*>& fits, std::vector<PlanItem> items, WorkerArgs& a) {
    const int nw = (int)items.size();
    std::stable_sort(items.begin(), items.end(), [](const PlanItem& x, const PlanItem& y) { return x.s > y.s; });
    const bm_fit_ctx* c0 = fits[0];
    int kmax = 0;
    bool groups = !g_big_tpb.load() && !g_no_groups.load() && nw <= kMaxLaunchClusters;
    for (const bm_fit_ctx* c : fits) {
        kmax = std::max(kmax, c->k);
        groups = groups && c->xpart && c->groups_ok;
    }
    // Groups need a cooperative launch that keeps its cluster shape; a tool
    // that intercepts launches (Nsight Compute was seen to) may drop it, and
    // then every worker gets one cluster (the same results).
    groups = groups && cooperative_clusters_ok();
    const long long smax = items[0].s;
    const long long cap = rows_cap(c0->np, kmax);
    const size_t base = worker_smem(c0->np, kmax);
    a.k_smem = kmax;
    for (int gcs = kGroupCs; groups && gcs >= 4; gcs /= 2) {
        std::vector<int> G(nw, 1);
        int total = nw;
        auto rows_of = [&](int i) { return (items[i].s + (long long)G[i] * gcs - 1) / ((long long)G[i] * gcs); };
        // capacity with the bucket memory of the current plan (it only
        // shrinks as groups grow, so the capacity only grows)
        int capacity = 0;
        for (int pass = 0; pass < 3; ++pass) {
            long long rows = 0;
            for (int i = 0; i < nw; ++i) rows = std::max(rows, rows_of(i));
            capacity = std::min(worker_active_clusters(c0->np, gcs, base + bucket_smem_bytes((int)rows)),
                                kMaxLaunchClusters);
            while (total < capacity) {
                int best = -1;
                for (int i = 0; i < nw; ++i)
                    if (G[i] < kMaxGroup && (best < 0 || rows_of(i) > rows_of(best))) best = i;
                if (best < 0 || rows_of(best) <= 256) break;
                G[best]++;
                total++;
            }
        }
        long long rows = 0;
        for (int i = 0; i < nw; ++i) rows = std::max(rows, rows_of(i));
        if (nw <= capacity && total <= capacity && rows <= cap) {
            int ci = 0;
            for (int i = 0; i < nw; ++i)
                for (int q = 0; q < G[i]; ++q)
                    a.cmap[ci++] = (unsigned)items[i].w | ((unsigned)items[i].fit << 12) | ((unsigned)q << 16) |
                                   ((unsigned)G[i] << 24);
            a.ncl = ci;
            a.cs = gcs;
            // Under an Nsight tool (which runs one kernel at a time when it
            // profiles one, and was seen to drop the cluster shape of a
            // cooperative launch it profiles) the launch is not cooperative:
            // the grid is within what the device holds at once, so every CTA
            // is resident while nothing else runs.
            static const bool nsight = std::getenv("NV_NSIGHT_INJECTION_TRANSPORT_TYPE") != nullptr;
            a.coop = nsight ? 0 : 1;
            a.rows_cta = (int)rows;
            a.tpb = 256;
            return ci;
        }
    }
    a.cs = cluster_size(smax, c0->max_cs, c0->rows_per_cta, cap);
    a.rows_cta = (int)((smax + a.cs - 1) / a.cs);
    a.coop = 0;
    a.tpb = (fits.size() == 1 && g_big_tpb.load() && a.cs == c0->max_cs && smax > (long long)a.cs * c0->rows_per_cta)
                ? 512 : 256;
    if (nw <= kMaxLaunchClusters) {
        for (int i = 0; i < nw; ++i) a.cmap[i] = (unsigned)items[i].w | ((unsigned)items[i].fit << 12) | (1u << 24);
        a.ncl = nw;
    } else {
        a.ncl = 0;                                  // worker = first worker + cluster index (one fit)
        int wmin = items[0].w;
        for (const PlanItem& it : items) wmin = std::min(wmin, it.w);
        a.worker_base = wmin;
    }
    return nw;
}

// The samples of round r0 of fit c ready on c->st: drawn ahead on the
// sampling stream, or drawn now (and L read back first for the exploit
// policy, whose sizes depend on it).
bm_status round_samples(bm_fit_ctx* c, int r0) {
    bm_status s;
    if ((s = ensure_streams(c))) return s;
    const int parity = r0 & 1;
    if (c->pol.exploit > 0) {                   // sizes of this round depend on L so far
        Globals h;
        if ((s = read_globals(c, &h))) return s;
        c->L_sum0 = (long long)h.L_sum;
        c->L_len0 = (long long)h.accepts;
    }
    if (c->prefetched == r0) {
        CU(cudaStreamWaitEvent(c->st, c->ev_sdone, 0));           // drawn ahead on the sampling stream
    } else {
        if (c->prefetched >= 0) CU(cudaStreamWaitEvent(c->st, c->ev_sdone, 0));
        SampleArgs sa = make_sample_args(c, kSampleRound, c->jobs, parity);
        sa.rnd = r0;
        const size_t sp_s = span_begin(c, 2);
        CU(launch_sample(c->np, sa, (c->w_hi - c->w_lo) * (c->pol.passes + 1), c->st));
        span_end(c, sp_s);
        c->n_kernels++;
    }
    c->prefetched = -1;
    return BM_OK;
}

// After the worker launch of round r0 (already enqueued on c->st): draw the
// next round's samples into the other half on the sampling stream while the
// workers run; that half was last read by the previous round, which finished
// before ev_fork.
bm_status round_prefetch(bm_fit_ctx* c, int r0) {
    if (r0 + 1 < c->rounds_planned && c->pol.exploit == 0) {
        CU(cudaStreamWaitEvent(c->sst, c->ev_fork, 0));
        SampleArgs sa = make_sample_args(c, kSampleRound, c->jobs, (r0 + 1) & 1);
        sa.rnd = r0 + 1;
        const size_t sp_s = span_begin(c, 2, c->sst);
        CU(launch_sample(c->np, sa, (c->w_hi - c->w_lo) * (c->pol.passes + 1), c->sst));
        span_end(c, sp_s);
        CU(cudaEventRecord(c->ev_sdone, c->sst));
        c->n_kernels++;
        c->prefetched = r0 + 1;
    }
    return BM_OK;
}

// Round r0 of every worker of fit c: the round's samples, one launch of the
// worker kernel for all workers (plan_launch), the next round's samples.
bm_status run_round_launch(bm_fit_ctx* c, int r0, int r1) {
    bm_status s;
    if (r1 != r0 + 1) return fail(BM_EINTERNAL, "one round per launch");
    // (round_samples may read the globals back, which folds the finished
    // timing spans: no span of this round is open before it)
    if ((s = round_samples(c, r0))) return s;
    const size_t sp = span_begin(c, 0);
    std::vector<PlanItem> items;
    for (int w = c->w_lo; w < c->w_hi; ++w) items.push_back({0, w, size_of(c, w, r0)});
    WorkerArgs a = make_args(c, kModeRounds, r0 & 1);
    a.round_begin = r0;
    a.round_end = r1;
    a.deadline_ns = (c->bud.seconds > 0) ? c->t0_gpu + (unsigned long long)(c->bud.seconds * 1e9) : 0ull;
    const int clusters = plan_launch({c}, items, a);
    if (a.ncl > 0 && c->xbar) CU(cudaMemsetAsync(c->xbar, 0, (size_t)c->pol.workers * 2 * 4, c->st));   // barriers, aborts
    CU(cudaEventRecord(c->ev_fork, c->st));
    CU(launch_worker(c->np, a, clusters, c->st));
    c->n_kernels++;
    c->last_groups = (a.ncl > 0 && a.cs == kGroupCs) ? clusters : 0;
    if ((s = round_prefetch(c, r0))) return s;
    span_end(c, sp);
    return BM_OK;
}

bm_status run_fullpass(bm_fit_ctx* c, const double* sel, int* labels, int incumbent) {
    const int grid = sm_count();
    const size_t sp = span_begin(c, 1);
    CU(launch_fullpass(c->np, c->X, c->m, c->n, c->Cw, c->k, sel, c->pol.workers, labels, c->glob, c->gB,
                       c->gp2, incumbent, grid, c->st));
    c->n_kernels++;
    span_end(c, sp);
    return BM_OK;
}

}  // namespace

extern "C" {

const char* bm_last_error(void) { return g_err.c_str(); }

bm_status bm_set_fullpass_impl(int32_t impl) {
    if (impl < 0 || impl > 2) return fail(BM_EINVAL, "fullpass impl = %d must be 0, 1 or 2", impl);
    set_fullpass_impl(impl);
    return BM_OK;
}
int32_t bm_last_fullpass_impl(void) { return last_fullpass_impl(); }

bm_status bm_debug_fail_allocs(int32_t count) {
    if (count < 0) return fail(BM_EINVAL, "count = %d must be >= 0", count);
    g_fail_allocs.store(count);
    return BM_OK;
}

bm_status bm_debug_set_wait_limit(uint32_t polls, uint32_t sleep_ns) {
    if (sleep_ns > 1000000u) return fail(BM_EINVAL, "sleep_ns = %u above 1e6", sleep_ns);
    set_tcx_wait_limit(polls, sleep_ns);
    return BM_OK;
}
const char* bm_version(void) { return "bigmeans-gb300 0.1 (sm_103a)"; }

}  // extern "C"

namespace {
// Validation and sizing of a fit (no device work): the context with every
// planned field set and nothing allocated.
bm_status plan_fit(const float* X_dev, int64_t m, int32_t n, int32_t k, const bm_sample_policy* policy,
                   const bm_budget* budget, uint64_t seed, void* stream, bm_fit_ctx** out) {
    *out = nullptr;
    if (!policy || !budget) return fail(BM_EINVAL, "policy and budget are required");
    bm_status s;
    if ((s = check_shape(m, n, k))) return s;
    bm_sample_policy pol = *policy;
    bm_budget bud = *budget;
    if (pol.workers < 1 || pol.workers > 4096) return fail(BM_EINVAL, "workers = %d out of range", pol.workers);
    if (pol.passes < 1) return fail(BM_EINVAL, "passes = %d must be >= 1", pol.passes);
    if (pol.set_len < 0 || pol.set_len > 16) return fail(BM_EINVAL, "set_len = %d out of range", pol.set_len);
    if (pol.kind != 0 && pol.kind != 1) return fail(BM_EINVAL, "policy kind = %d must be 0 or 1", pol.kind);
    if (pol.exploit < 0 || pol.exploit > 100) return fail(BM_EINVAL, "exploit = %d out of [0, 100]", pol.exploit);
    long long s_lo, s_hi;
    if (pol.set_len > 0) {
        s_lo = s_hi = std::min<long long>(pol.set[0], m);
        for (int i = 0; i < pol.set_len; ++i) {
            pol.set[i] = std::min<long long>(pol.set[i], m);
            s_lo = std::min<long long>(s_lo, pol.set[i]);
            s_hi = std::max<long long>(s_hi, pol.set[i]);
        }
    } else {
        pol.s_max = std::min<long long>(pol.s_max, m);
        s_lo = pol.s_min;
        s_hi = pol.s_max;
        if (s_lo > s_hi) return fail(BM_EINVAL, "s_min = %lld > s_max = %lld", s_lo, s_hi);
    }
    if (s_lo < k) return fail(BM_EINVAL, "smallest sample size %lld is below k = %d", s_lo, k);
    if (bud.rounds < 0 || (bud.rounds == 0 && !(bud.seconds > 0)))
        return fail(BM_EINVAL, "need rounds > 0 or seconds > 0");
    if (bud.max_lloyd < 0) return fail(BM_EINVAL, "max_lloyd < 0");
    if (bud.kpp_candidates < 1 || bud.kpp_candidates > 3)
        return fail(BM_EINVAL, "kpp_candidates = %d out of range [1, 3]", bud.kpp_candidates);
    if (!(bud.tol >= 0) && bud.tol != -1.0 && !(bud.tol < 0))
        return fail(BM_EINVAL, "tol is NaN");

    bm_fit_ctx* c = new bm_fit_ctx();
    c->t0 = std::chrono::steady_clock::now();
    c->groups_ok = t_groups_ok;
    c->st = (cudaStream_t)stream;
    c->X = X_dev; c->m = m; c->n = n; c->k = k; c->np = padded_dim(n);
    c->pol = pol; c->bud = bud; c->seed = seed;
    c->s_lo = s_lo; c->s_hi = s_hi; c->s_cap = s_hi;
    c->w_lo = 0; c->w_hi = pol.workers;
    c->max_cs = worker_max_cluster(c->np, k);
    c->rows_per_cta = g_rows_per_cta.load();
    c->cs = cluster_size(s_hi, c->max_cs, c->rows_per_cta, rows_cap(c->np, k));
    if (c->cs == 0) {
        const long long most = (long long)c->max_cs * rows_cap(c->np, k);
        delete c;
        return fail(BM_EINVAL, "s_max = %lld above %lld", s_hi, most);
    }
    c->Tcap = draw_cap(m, s_hi);
    if (c->Tcap >= (1ll << 32) - 1) { delete c; return fail(BM_EINVAL, "sample size too close to m"); }
    c->H = next_pow2(2 * c->Tcap);
    if (c->H > (1ll << 31)) { delete c; return fail(BM_EINVAL, "sample sizes need a sampler table above 2^31"); }
    c->L_cap = (bud.rounds > 0 ? (long long)bud.rounds : 4096ll) * pol.workers * pol.passes;
    c->L_cap = std::min<long long>(c->L_cap, 1ll << 24);
    c->smem = worker_smem(c->np, k);
    c->rounds_planned = bud.rounds > 0 ? bud.rounds : 0x7fffffff;
    cert_constants(c->np, c->gB, c->gp2);
    *out = c;
    return BM_OK;
}
}  // namespace

extern "C" {

bm_status bm_trim_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& kv : g_pools) {
        const cudaError_t e = cudaMemPoolTrimTo(kv.second, 0);
        if (e != cudaSuccess) return fail(BM_ECUDA, "trim: %s", cudaGetErrorString(e));
    }
    return BM_OK;
}

bm_status bm_set_rows_per_cta(int32_t rows) {
    if (rows == 0) rows = kRowsPerCta;
    if (rows < 256 || rows > kMaxRowsPerCta) return fail(BM_EINVAL, "rows per CTA = %d out of [256, %lld]", rows,
                                                         (long long)kMaxRowsPerCta);
    g_rows_per_cta.store(rows);
    return BM_OK;
}
int32_t bm_get_rows_per_cta(void) { return g_rows_per_cta.load(); }

bm_status bm_set_big_clusters(int32_t on) {
    if (on != 0 && on != 1) return fail(BM_EINVAL, "big-cluster option = %d must be 0 or 1", on);
    g_big_tpb.store(on);
    return BM_OK;
}
int32_t bm_get_big_clusters(void) { return g_big_tpb.load(); }

bm_status bm_set_worker_groups(int32_t on) {
    if (on != 0 && on != 1) return fail(BM_EINVAL, "worker groups = %d must be 0 or 1", on);
    g_no_groups.store(on ? 0 : 1);
    return BM_OK;
}
int32_t bm_get_worker_groups(void) { return g_no_groups.load() ? 0 : 1; }

bm_status bm_set_sampler_impl(int32_t impl) {
    if (impl != 0 && impl != 1) return fail(BM_EINVAL, "sampler impl = %d must be 0 or 1", impl);
    g_sample_tables.store(impl);
    return BM_OK;
}
int32_t bm_get_sampler_impl(void) { return g_sample_tables.load(); }

bm_status bm_autotune_rows_per_cta(const float* X_dev, int64_t m, int32_t n, int32_t k,
                                   const bm_sample_policy* policy, const bm_budget* budget, uint64_t seed,
                                   void* stream, const int32_t* candidates, int32_t n_candidates,
                                   int32_t* best_out, double* ms_out) {
    if (!candidates || n_candidates < 1 || n_candidates > 16 || !best_out || !budget)
        return fail(BM_EINVAL, "autotune: bad candidate list or outputs");
    const int keep = g_rows_per_cta.load();
    bm_budget bud = *budget;
    bud.rounds = 2;
    bud.seconds = 0;
    double best_ms = 1e300;
    int best = keep;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n_candidates; ++i) {
        bm_status s = bm_set_rows_per_cta(candidates[i]);
        if (s) { g_rows_per_cta.store(keep); return s; }
        bm_fit_ctx* c = nullptr;
        if ((s = bm_fit_create(X_dev, m, n, k, policy, &bud, seed, stream, &c))) { g_rows_per_cta.store(keep); return s; }
        cudaEvent_t a = nullptr, b = nullptr;
        float ms = 0.f;
        if ((s = bm_fit_rounds(c, 1)) == BM_OK) {              // round 0 warms up
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, st);
            s = bm_fit_rounds(c, 1);
            cudaEventRecord(b, st);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&ms, a, b);
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
        bm_fit_destroy(c);
        if (s) { g_rows_per_cta.store(keep); return s; }
        if (ms_out) ms_out[i] = ms;
        if (ms < best_ms) { best_ms = ms; best = candidates[i]; }
    }
    g_rows_per_cta.store(best);
    *best_out = best;
    return BM_OK;
}

bm_status bm_fit_footprint(int64_t m, int32_t n, int32_t k, const bm_sample_policy* policy,
                           const bm_budget* budget, int64_t* bytes_out) {
    if (!bytes_out) return fail(BM_EINVAL, "bytes_out is NULL");
    bm_fit_ctx* c = nullptr;
    bm_status s = plan_fit(nullptr, m, n, k, policy, budget, 0, nullptr, &c);
    if (s) return s;
    *bytes_out = (int64_t)workspace_bytes(c, c->pol.workers);
    delete c;
    return BM_OK;
}

bm_status bm_fit_create(const float* X_dev, int64_t m, int32_t n, int32_t k, const bm_sample_policy* policy,
                        const bm_budget* budget, uint64_t seed, void* stream, bm_fit_ctx** out) {
    if (!out) return fail(BM_EINVAL, "out is NULL");
    *out = nullptr;
    bm_status s = check_ptr(X_dev, "X_dev");
    if (s) return s;
    bm_fit_ctx* c = nullptr;
    if ((s = plan_fit(X_dev, m, n, k, policy, budget, seed, stream, &c))) return s;
    const bm_sample_policy& pol = c->pol;
    if ((s = alloc_workspace(c, pol.workers))) { delete c; return s; }
    cudaError_t e;
    if ((e = launch_init_state(c->fhat, pol.workers, c->deg, (long long)pol.workers * k, c->glob, c->st)) ||
        (e = launch_prepass(X_dev, m * n, c->glob, 2 * sm_count(), c->st)) ||
        (e = launch_globaltimer(c->timer, c->st))) {
        bm_fit_destroy(c);
        return fail(BM_ECUDA, "launch failed: %s", cudaGetErrorString(e));
    }
    Globals h;
    if ((s = read_globals(c, &h))) { bm_fit_destroy(c); return s; }
    if ((s = status_from_flags(h))) { bm_fit_destroy(c); return s; }
    if ((e = cudaMemcpy(&c->t0_gpu, c->timer, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        bm_fit_destroy(c);
        return fail(BM_ECUDA, "%s", cudaGetErrorString(e));
    }
    *out = c;
    return BM_OK;
}

bm_status bm_fit_rounds(bm_fit_ctx* c, int32_t rounds) {
    if (!c) return fail(BM_EINVAL, "ctx is NULL");
    if (rounds < 0) return fail(BM_EINVAL, "rounds < 0");
    if (rounds == 0) return BM_OK;
    bm_status s;
    // one sampling launch plus one launch per worker for every round; with a
    // wall-clock budget the host checks the clock between rounds and the
    // kernels check it between passes
    for (int r = 0; r < rounds; ++r) {
        if (c->bud.seconds > 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - c->t0).count();
            if (el >= c->bud.seconds) break;
        }
        if ((s = run_round_launch(c, c->rounds_run, c->rounds_run + 1))) return s;
        c->rounds_run += 1;
        if (c->bud.eval_full_each_round)
            if ((s = run_fullpass(c, c->fhat, nullptr, 1))) return s;
        if (c->bud.seconds > 0) CU(cudaStreamSynchronize(c->st));
    }
    Globals h;
    if ((s = read_globals(c, &h))) return s;
    return status_from_flags(h);
}

bm_status bm_fit_rounds_batch(bm_fit_ctx* const* fits, int32_t nfits, int32_t rounds) {
    if (!fits || nfits < 1 || nfits > 16) return fail(BM_EINVAL, "nfits = %d out of range [1, 16]", nfits);
    if (rounds < 0) return fail(BM_EINVAL, "rounds < 0");
    int total = 0;
    for (int i = 0; i < nfits; ++i) {
        if (!fits[i]) return fail(BM_EINVAL, "fits[%d] is NULL", i);
        for (int j = 0; j < i; ++j)
            if (fits[j] == fits[i]) return fail(BM_EINVAL, "fits[%d] repeats fits[%d]", i, j);
        if (fits[i]->np != fits[0]->np)
            return fail(BM_EINVAL, "fits[%d] has another padded width (n = %d vs %d)", i, fits[i]->n, fits[0]->n);
        if (fits[i]->bud.seconds > 0) return fail(BM_EINVAL, "fits[%d] has a wall-clock budget", i);
        total += fits[i]->w_hi - fits[i]->w_lo;
    }
    if (nfits == 1) return bm_fit_rounds(fits[0], rounds);
    if (total > kMaxLaunchClusters) return fail(BM_EINVAL, "%d workers in all above %d", total, kMaxLaunchClusters);
    if (rounds == 0) return BM_OK;
    // Everything runs on the first fit's stream: the other fits' streams are
    // joined into it now and wait for it at the end.
    cudaStream_t st = fits[0]->st;
    std::vector<cudaStream_t> own(nfits);
    cudaEvent_t ev = nullptr;
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    struct EvGuard { cudaEvent_t e; ~EvGuard() { cudaEventDestroy(e); } } evg{ev};
    for (int i = 0; i < nfits; ++i) {
        own[i] = fits[i]->st;
        if (i > 0) {
            CU(cudaEventRecord(ev, own[i]));
            CU(cudaStreamWaitEvent(st, ev, 0));
        }
        fits[i]->st = st;
    }
    void* dargs = nullptr;
    bm_status s = BM_OK;
    if (lib_alloc(&dargs, sizeof(WorkerArgs) * nfits, st) != cudaSuccess) {
        cudaGetLastError();
        s = fail(BM_ENOMEM, "arguments of a batched launch");
    }
    std::vector<WorkerArgs> hargs(nfits);
    for (int r = 0; r < rounds && s == BM_OK; ++r) {
        std::vector<PlanItem> items;
        for (int i = 0; i < nfits && s == BM_OK; ++i) {
            bm_fit_ctx* c = fits[i];
            if ((s = round_samples(c, c->rounds_run))) break;
            for (int w = c->w_lo; w < c->w_hi; ++w) items.push_back({i, w, size_of(c, w, c->rounds_run)});
        }
        if (s) break;
        WorkerArgs plan;
        memset(&plan, 0, sizeof plan);
        std::vector<bm_fit_ctx*> fv(fits, fits + nfits);
        const int clusters = plan_launch(fv, items, plan);
        for (int i = 0; i < nfits; ++i) {
            bm_fit_ctx* c = fits[i];
            WorkerArgs& a = hargs[i];
            a = make_args(c, kModeRounds, c->rounds_run & 1);
            a.round_begin = c->rounds_run;
            a.round_end = c->rounds_run + 1;
            a.cs = plan.cs; a.rows_cta = plan.rows_cta; a.ncl = plan.ncl; a.coop = plan.coop;
            a.tpb = 256; a.k_smem = plan.k_smem;
            memcpy(a.cmap, plan.cmap, sizeof a.cmap);
            a.batch = (const WorkerArgs*)dargs;
            if (c->xbar && cudaMemsetAsync(c->xbar, 0, (size_t)c->pol.workers * 2 * 4, st) != cudaSuccess)
                s = fail(BM_ECUDA, "barrier reset");
        }
        if (s) break;
        // pageable source: the call returns once the arguments are staged,
        // and the copy runs after the previous round's launch on st
        if (cudaMemcpyAsync(dargs, hargs.data(), sizeof(WorkerArgs) * nfits, cudaMemcpyHostToDevice, st) !=
            cudaSuccess) { s = fail(BM_ECUDA, "arguments of a batched launch"); break; }
        const size_t sp = span_begin(fits[0], 0);
        for (int i = 0; i < nfits; ++i) cudaEventRecord(fits[i]->ev_fork, st);
        const cudaError_t e = launch_worker(fits[0]->np, hargs[0], clusters, st);
        span_end(fits[0], sp);
        if (e != cudaSuccess) { s = fail(BM_ECUDA, "batched worker launch: %s", cudaGetErrorString(e)); break; }
        fits[0]->n_kernels++;
        for (int i = 0; i < nfits && s == BM_OK; ++i) {
            bm_fit_ctx* c = fits[i];
            c->last_groups = clusters;
            if ((s = round_prefetch(c, c->rounds_run))) break;
            c->rounds_run += 1;
            if (c->bud.eval_full_each_round) s = run_fullpass(c, c->fhat, nullptr, 1);
        }
    }
    if (dargs) cudaFreeAsync(dargs, st);
    cudaEventRecord(ev, st);
    for (int i = 0; i < nfits; ++i) {
        fits[i]->st = own[i];
        if (i > 0) cudaStreamWaitEvent(own[i], ev, 0);
    }
    if (s) return s;
    for (int i = 0; i < nfits; ++i) {
        Globals h;
        if ((s = read_globals(fits[i], &h))) return s;
        if ((s = status_from_flags(h))) return s;
    }
    return BM_OK;
}

bm_status bm_fit_set_workers(bm_fit_ctx* c, int32_t w_begin, int32_t w_end) {
    if (!c) return fail(BM_EINVAL, "ctx is NULL");
    if (c->rounds_run > 0) return fail(BM_EINVAL, "the worker range is set before the first round");
    if (w_begin < 0 || w_end > c->pol.workers || w_begin >= w_end)
        return fail(BM_EINVAL, "worker range [%d, %d) not inside [0, %d)", w_begin, w_end, c->pol.workers);
    if (c->pol.exploit > 0) return fail(BM_EINVAL, "a shard of workers cannot use the exploit policy (L is global)");
    if (c->prefetched >= 0) {                  // drop a draw-ahead made for the old range
        CU(cudaStreamWaitEvent(c->st, c->ev_sdone, 0));
        c->prefetched = -1;
    }
    c->w_lo = w_begin;
    c->w_hi = w_end;
    return BM_OK;
}

bm_status bm_fit_recheck(bm_fit_ctx* c, int64_t s_opt, double* f_out_host) {
    if (!c || !f_out_host) return fail(BM_EINVAL, "ctx and f_out_host are required");
    const long long lo = c->pol.set_len > 0 ? c->s_lo : c->pol.s_min;
    if (s_opt < std::max<long long>(lo, c->k) || s_opt > c->s_hi)
        return fail(BM_EINVAL, "s_opt = %lld outside the size range [%lld, %lld]", (long long)s_opt, lo, c->s_hi);
    if (c->prefetched >= 0) {
        CU(cudaStreamWaitEvent(c->st, c->ev_sdone, 0));
        c->prefetched = -1;
    }
    const size_t sp = span_begin(c, 0);
    SampleArgs sa = make_sample_args(c, kSampleFinal, 1);
    sa.step_s = s_opt;
    CU(launch_sample(c->np, sa, 1, c->st));
    WorkerArgs a = make_args(c, kModeFinalEval);
    a.worker_base = c->w_lo;
    CU(launch_worker(c->np, a, c->w_hi - c->w_lo, c->st));
    c->n_kernels += 2;
    span_end(c, sp);
    CU(cudaMemcpyAsync(f_out_host, c->f_final + c->w_lo, (size_t)(c->w_hi - c->w_lo) * 8, cudaMemcpyDeviceToHost,
                       c->st));
    Globals h;
    bm_status s;
    if ((s = read_globals(c, &h))) return s;
    return status_from_flags(h);
}

bm_status bm_fit_worker_centroids(bm_fit_ctx* c, int32_t w, float* C_out_dev) {
    if (!c) return fail(BM_EINVAL, "ctx is NULL");
    if (w < c->w_lo || w >= c->w_hi) return fail(BM_EINVAL, "worker %d not in [%d, %d)", w, c->w_lo, c->w_hi);
    bm_status s = check_ptr(C_out_dev, "C_out_dev");
    if (s) return s;
    CU(launch_unpad(c->Cw + (size_t)w * c->k * c->np, c->k, c->n, c->np, C_out_dev, c->st));
    CU(cudaStreamSynchronize(c->st));
    return BM_OK;
}

static bm_status fit_finish(bm_fit_ctx* c, float* C_out_dev, int32_t* labels_out_dev, bm_report* rep,
                            bool full_pass);
bm_status bm_fit_finish(bm_fit_ctx* c, float* C_out_dev, int32_t* labels_out_dev, bm_report* rep) {
    return fit_finish(c, C_out_dev, labels_out_dev, rep, true);
}

// The common recheck and C_best; with full_pass, the exact full-data pass
// gives the labels and f(C_best, X) (else the caller takes them another way).
static bm_status fit_finish(bm_fit_ctx* c, float* C_out_dev, int32_t* labels_out_dev, bm_report* rep,
                            bool full_pass) {
    if (!c) return fail(BM_EINVAL, "ctx is NULL");
    if (c->w_lo != 0 || c->w_hi != c->pol.workers)
        return fail(BM_EINVAL, "a shard of workers finishes through bm_fit_recheck and the ranks' exchange");
    bm_status s = check_ptr(C_out_dev, "C_out_dev");
    if (s) return s;
    WorkerArgs a = make_args(c, kModeFinalEval);
    if (c->prefetched >= 0) {                  // a drawn-ahead round was not run
        CU(cudaStreamWaitEvent(c->st, c->ev_sdone, 0));
        c->prefetched = -1;
    }
    const size_t sp = span_begin(c, 0);
    SampleArgs sa = make_sample_args(c, kSampleFinal, 1);
    CU(launch_sample(c->np, sa, 1, c->st));
    CU(launch_worker(c->np, a, c->pol.workers, c->st));
    c->n_kernels += 2;
    span_end(c, sp);
    if (full_pass && (s = run_fullpass(c, c->f_final, labels_out_dev, 1))) return s;
    CU(launch_select_unpad(c->Cw, c->f_final, c->pol.workers, c->k, c->n, c->np, C_out_dev, c->st));
    Globals h;
    if ((s = read_globals(c, &h))) return s;
    if ((s = status_from_flags(h))) return s;
    if (rep) fill_report(c, h, rep);
    return BM_OK;
}

// ------------------------------------------------------ checkpoint/resume
// The state of a fit between rounds: the workers' incumbent centroids,
// degenerate flags and f_hat, the list L, the device counters and the round
// index.  Samples, seeds and sizes are functions of (seed, worker, round,
// pass), so a fit resumed from this state on the same X with the same
// arguments draws what the uninterrupted fit would draw.
}  // extern "C"

namespace {
struct StateHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int64_t m;
    int32_t n, k, np, W, P, w_lo, w_hi, rounds_run;
    uint64_t seed, fingerprint;
    int64_t n_L;                                  // entries of L exported
    uint64_t b_glob, b_Cw, b_deg, b_fhat, b_L;   // section sizes in bytes
    double t_worker, t_full, t_sample;
    int64_t n_worker, n_full, n_kernels;
};
constexpr char kStateMagic[8] = {'B', 'M', 'F', 'I', 'T', 'S', 'T', '1'};

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}
// The arguments that decide the computation (not the wall budget or T).
uint64_t state_fingerprint(const bm_fit_ctx* c, unsigned int maxbits) {
    uint64_t h = 1469598103934665603ull;
    const auto add = [&](const auto& v) { h = fnv1a(h, &v, sizeof v); };
    add(c->pol.s_min); add(c->s_hi); add(c->pol.set_len);
    for (int i = 0; i < c->pol.set_len && i < 16; ++i) add(c->pol.set[i]);
    add(c->pol.workers); add(c->pol.passes); add(c->pol.kind); add(c->pol.exploit);
    add(c->bud.max_lloyd); add(c->bud.tol); add(c->bud.kpp_candidates); add(c->bud.eval_full_each_round);
    add(maxbits);
    return h;
}
size_t state_sections(const bm_fit_ctx* c, int64_t n_L, uint64_t* b) {
    b[0] = sizeof(Globals);
    b[1] = (uint64_t)c->pol.workers * c->k * c->np * 4;
    b[2] = (uint64_t)c->pol.workers * c->k;
    b[3] = (uint64_t)c->pol.workers * 8;
    b[4] = (uint64_t)n_L * 8;
    return sizeof(StateHeader) + b[0] + b[1] + b[2] + b[3] + b[4];
}
// Both streams of the fit idle (the next round's samples may be drawn ahead).
bm_status fit_quiesce(bm_fit_ctx* c) {
    if (c->sst) CU(cudaStreamSynchronize(c->sst));
    CU(cudaStreamSynchronize(c->st));
    return BM_OK;
}
}  // namespace

extern "C" {

bm_status bm_fit_state_size(bm_fit_ctx* c, int64_t* bytes) {
    if (!c || !bytes) return fail(BM_EINVAL, "ctx and bytes are required");
    bm_status s = fit_quiesce(c);
    if (s) return s;
    Globals h;
    if ((s = read_globals(c, &h))) return s;
    uint64_t b[5];
    *bytes = (int64_t)state_sections(c, std::min<long long>((long long)h.accepts, c->L_cap), b);
    return BM_OK;
}

bm_status bm_fit_export(bm_fit_ctx* c, void* host_buf, int64_t bytes) {
    if (!c || !host_buf) return fail(BM_EINVAL, "ctx and host_buf are required");
    bm_status s = fit_quiesce(c);
    if (s) return s;
    Globals h;
    if ((s = read_globals(c, &h))) return s;
    if ((s = status_from_flags(h))) return s;
    const int64_t n_L = std::min<long long>((long long)h.accepts, c->L_cap);
    StateHeader hd;
    memset(&hd, 0, sizeof hd);
    uint64_t b[5];
    const size_t total = state_sections(c, n_L, b);
    hd.b_glob = b[0]; hd.b_Cw = b[1]; hd.b_deg = b[2]; hd.b_fhat = b[3]; hd.b_L = b[4];
    if (bytes < (int64_t)total) return fail(BM_EINVAL, "host_buf holds %lld bytes, the state %zu", (long long)bytes, total);
    memcpy(hd.magic, kStateMagic, 8);
    hd.version = 1;
    hd.header_bytes = sizeof hd;
    hd.m = c->m; hd.n = c->n; hd.k = c->k; hd.np = c->np; hd.W = c->pol.workers; hd.P = c->pol.passes;
    hd.w_lo = c->w_lo; hd.w_hi = c->w_hi; hd.rounds_run = c->rounds_run;
    hd.seed = c->seed;
    hd.fingerprint = state_fingerprint(c, h.maxbits);
    hd.n_L = n_L;
    hd.t_worker = c->t_worker; hd.t_full = c->t_full; hd.t_sample = c->t_sample;
    hd.n_worker = c->n_worker; hd.n_full = c->n_full; hd.n_kernels = c->n_kernels;
    char* out = static_cast<char*>(host_buf);
    memcpy(out, &hd, sizeof hd);
    size_t off = sizeof hd;
    memcpy(out + off, &h, sizeof h);
    off += hd.b_glob;
    const void* src[4] = {c->Cw, c->deg, c->fhat, c->L_buf};
    const uint64_t len[4] = {hd.b_Cw, hd.b_deg, hd.b_fhat, hd.b_L};
    for (int i = 0; i < 4; ++i) {
        if (len[i]) CU(cudaMemcpyAsync(out + off, src[i], len[i], cudaMemcpyDeviceToHost, c->st));
        off += len[i];
    }
    CU(cudaStreamSynchronize(c->st));
    return BM_OK;
}

bm_status bm_fit_import(bm_fit_ctx* c, const void* host_buf, int64_t bytes) {
    if (!c || !host_buf) return fail(BM_EINVAL, "ctx and host_buf are required");
    if (c->rounds_run != 0 || c->prefetched >= 0) return fail(BM_EINVAL, "import into a context before its first round");
    if (bytes < (int64_t)sizeof(StateHeader)) return fail(BM_EINVAL, "state of %lld bytes is truncated", (long long)bytes);
    StateHeader hd;
    memcpy(&hd, host_buf, sizeof hd);
    if (memcmp(hd.magic, kStateMagic, 8) != 0 || hd.version != 1 || hd.header_bytes != sizeof hd)
        return fail(BM_EINVAL, "not a fit state of this library version");
    bm_status s = fit_quiesce(c);
    if (s) return s;
    Globals h;
    if ((s = read_globals(c, &h))) return s;
    if (hd.m != c->m || hd.n != c->n || hd.k != c->k || hd.np != c->np || hd.W != c->pol.workers ||
        hd.P != c->pol.passes || hd.w_lo != c->w_lo || hd.w_hi != c->w_hi || hd.seed != c->seed)
        return fail(BM_EINVAL, "state of another fit (shape, workers, passes, shard or seed differ)");
    if (hd.fingerprint != state_fingerprint(c, h.maxbits))
        return fail(BM_EINVAL, "state of another fit (size policy, budget settings or X differ)");
    if (hd.rounds_run < 0 || hd.n_L < 0 || hd.n_L > c->L_cap)
        return fail(BM_EINVAL, "state's L (%lld entries) does not fit this context (%lld)", (long long)hd.n_L,
                    (long long)c->L_cap);
    uint64_t b[5];
    const size_t total = state_sections(c, hd.n_L, b);
    if (b[0] != hd.b_glob || b[1] != hd.b_Cw || b[2] != hd.b_deg || b[3] != hd.b_fhat || b[4] != hd.b_L)
        return fail(BM_EINVAL, "state sections do not match this context");
    if (bytes < (int64_t)total) return fail(BM_EINVAL, "state of %lld bytes is truncated (%zu)", (long long)bytes, total);
    const char* in = static_cast<const char*>(host_buf);
    size_t off = sizeof hd;
    Globals g;
    memcpy(&g, in + off, sizeof g);
    if (g.maxbits != h.maxbits) return fail(BM_EINVAL, "state of another X");
    off += hd.b_glob;
    CU(cudaMemcpyAsync(c->glob, &g, sizeof g, cudaMemcpyHostToDevice, c->st));
    void* dst[4] = {c->Cw, c->deg, c->fhat, c->L_buf};
    const uint64_t len[4] = {hd.b_Cw, hd.b_deg, hd.b_fhat, hd.b_L};
    for (int i = 0; i < 4; ++i) {
        if (len[i]) CU(cudaMemcpyAsync(dst[i], in + off, len[i], cudaMemcpyHostToDevice, c->st));
        off += len[i];
    }
    CU(cudaStreamSynchronize(c->st));
    c->rounds_run = hd.rounds_run;
    c->t_worker = hd.t_worker; c->t_full = hd.t_full; c->t_sample = hd.t_sample;
    c->n_worker = hd.n_worker; c->n_full = hd.n_full; c->n_kernels = hd.n_kernels;
    return BM_OK;
}

bm_status bm_fit_report(bm_fit_ctx* c, bm_report* rep) {
    if (!c || !rep) return fail(BM_EINVAL, "ctx and report are required");
    Globals h;
    bm_status s = read_globals(c, &h);
    if (s) return s;
    fill_report(c, h, rep);
    if (!c->bud.eval_full_each_round) { rep->f_full = 0.0; rep->f_incumbent = INFINITY; }
    return status_from_flags(h);
}

void bm_fit_destroy(bm_fit_ctx* c) {
    if (!c) return;
    if (c->prefetched >= 0 && c->ev_sdone) cudaStreamWaitEvent(c->st, c->ev_sdone, 0);
    // nothing of this fit may still run when its workspace is released (the
    // stream-ordered allocator may hand the memory to another stream at once)
    if (c->sst) cudaStreamSynchronize(c->sst);
    if (c->base) {
        cudaFreeAsync(c->base, c->st);
        cudaStreamSynchronize(c->st);
    }
    if (c->sst) cudaStreamSynchronize(c->sst);
    collect_spans(c);
    for (auto& sp : c->spans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    if (c->sst) cudaStreamDestroy(c->sst);
    if (c->ev_sdone) cudaEventDestroy(c->ev_sdone);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    delete c;
}

bm_status bigmeans_fit(const float* X_dev, int64_t m, int32_t n, int32_t k, const bm_sample_policy* policy,
                       const bm_budget* budget, uint64_t seed, void* stream, float* C_out_dev,
                       int32_t* labels_out_dev, bm_report* report_out) {
    bm_fit_ctx* c = nullptr;
    bm_status s = bm_fit_create(X_dev, m, n, k, policy, budget, seed, stream, &c);
    if (s) return s;
    const int T = budget->rounds > 0 ? budget->rounds : 0x3fffffff;
    if ((s = bm_fit_rounds(c, T))) { bm_fit_destroy(c); return s; }
    s = bm_fit_finish(c, C_out_dev, labels_out_dev, report_out);
    bm_fit_destroy(c);
    return s;
}

static bm_status assign_bf16(const void* Xb_dev, const float* norms_dev, const float* X_dev, int64_t m, int32_t n,
                             const float* C_dev, int32_t k, float tau, int certify, int32_t* labels_out_dev,
                             double* f_out_host, bm_report* rep, void* stream);

bm_status bigmeans_fit_dt(const void* X_dev, const float* X_master_dev, bm_dtype dt, int64_t m, int32_t n,
                          int32_t k, const bm_sample_policy* policy, const bm_budget* budget, uint64_t seed,
                          bm_mode mode, void* stream, float* C_out_dev, int32_t* labels_out_dev,
                          bm_report* report_out) {
    if (dt != BM_F32 && dt != BM_BF16) return fail(BM_EINVAL, "dt = %d is not BM_F32 or BM_BF16", (int)dt);
    if (mode != BM_MODE_EXACT && mode != BM_MODE_FAST) return fail(BM_EINVAL, "mode = %d is not a bm_mode", (int)mode);
    if (!X_dev) return fail(BM_EINVAL, "X_dev is NULL");
    if (dt == BM_F32 && X_master_dev && (const void*)X_master_dev != X_dev)
        return fail(BM_EINVAL, "BM_F32: X_master_dev must be NULL or X_dev");
    if (dt == BM_BF16 && !X_master_dev) return fail(BM_EINVAL, "BM_BF16 needs the FP32 master X_master_dev");
    const float* Xf = dt == BM_F32 ? static_cast<const float*>(X_dev) : X_master_dev;
    if (mode == BM_MODE_EXACT)
        return bigmeans_fit(Xf, m, n, k, policy, budget, seed, stream, C_out_dev, labels_out_dev, report_out);
    // fast: the fit on the FP32 rows, then labels and f(C_best, X) from the
    // precision pass (tau = 1e-3) on the BF16 rows
    bm_status s = check_shape(m, n, k);
    if (s) return s;
    if (n > 64 || k > 256) return fail(BM_EINVAL, "BM_MODE_FAST needs n <= 64 and k <= 256");
    if (dt == BM_BF16 && (((uintptr_t)X_dev) & 1023)) return fail(BM_EINVAL, "BF16 X_dev must be 1024-byte aligned");
    bm_fit_ctx* c = nullptr;
    if ((s = bm_fit_create(Xf, m, n, k, policy, budget, seed, stream, &c))) return s;
    const int T = budget->rounds > 0 ? budget->rounds : 0x3fffffff;
    if (!(s = bm_fit_rounds(c, T))) s = fit_finish(c, C_out_dev, nullptr, report_out, false);
    bm_fit_destroy(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const long long m_pad = (m + 127) / 128 * 128;
    const size_t xb_bytes = dt == BM_F32 ? (size_t)m_pad * 128 : 0;
    void* base = nullptr;
    CU(lib_alloc(&base, xb_bytes + (size_t)(m_pad + 1) * 4 + 1024, st));
    void* Xb = dt == BM_F32 ? (void*)(((uintptr_t)base + 1023) & ~(uintptr_t)1023) : const_cast<void*>(X_dev);
    float* norms = reinterpret_cast<float*>(((uintptr_t)base + 1023) & ~(uintptr_t)1023) + xb_bytes / 4;
    cudaError_t e = launch_pack_bf16(Xf, m, n, m_pad, dt == BM_F32 ? Xb : nullptr, norms, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(base, st);
        cudaStreamSynchronize(st);
        return fail(BM_ECUDA, "pack: %s", cudaGetErrorString(e));
    }
    double f = 0.0;
    bm_report rb;
    s = assign_bf16(Xb, norms, Xf, m, n, C_out_dev, k, 1e-3f, 0, labels_out_dev, &f, &rb, stream);
    cudaFreeAsync(base, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (s) return s;
    if (e2 != cudaSuccess) return fail(BM_ECUDA, "fast pass: %s", cudaGetErrorString(e2));
    if (report_out) {
        report_out->f_full = f;
        report_out->rescored_rows = rb.rescored_rows;
    }
    return BM_OK;
}

bm_status bigmeans_fit_host(const float* X_host, int64_t m, int32_t n, int32_t k,
                            const bm_sample_policy* policy, const bm_budget* budget, uint64_t seed,
                            void* stream, float* C_out_host, int32_t* labels_out_host, bm_report* rep) {
    if (!X_host || !C_out_host) return fail(BM_EINVAL, "X_host and C_out_host are required");
    bm_status s = check_shape(m, n, k);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    float* Xd = nullptr; float* Cd = nullptr; int32_t* Ld = nullptr;
    const size_t xb = (size_t)m * n * 4;
    CU(lib_alloc((void**)&Xd, xb, st));
    if (lib_alloc((void**)&Cd, (size_t)k * n * 4 + 16, st) != cudaSuccess ||
        (labels_out_host && lib_alloc((void**)&Ld, (size_t)m * 4, st) != cudaSuccess)) {
        cudaFreeAsync(Xd, st);
        if (Cd) cudaFreeAsync(Cd, st);
        cudaStreamSynchronize(st);
        return fail(BM_ENOMEM, "device buffers for the host-buffer fit");
    }
    cudaEvent_t hc[2] = {nullptr, nullptr};              // around the copy of X
    if (cudaEventCreate(&hc[0]) != cudaSuccess || cudaEventCreate(&hc[1]) != cudaSuccess) cudaGetLastError();
    if (hc[0]) cudaEventRecord(hc[0], st);
    cudaError_t e = cudaMemcpyAsync(Xd, X_host, xb, cudaMemcpyHostToDevice, st);
    if (hc[1]) cudaEventRecord(hc[1], st);
    float h2d_ms = 0.f;
    if (e == cudaSuccess) {
        s = bigmeans_fit(Xd, m, n, k, policy, budget, seed, stream, Cd, Ld, rep);
        if (s == BM_OK) {
            e = cudaMemcpyAsync(C_out_host, Cd, (size_t)k * n * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && labels_out_host)
                e = cudaMemcpyAsync(labels_out_host, Ld, (size_t)m * 4, cudaMemcpyDeviceToHost, st);
        }
    }
    cudaFreeAsync(Xd, st);
    cudaFreeAsync(Cd, st);
    if (Ld) cudaFreeAsync(Ld, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (hc[0] && hc[1] && cudaEventElapsedTime(&h2d_ms, hc[0], hc[1]) != cudaSuccess) cudaGetLastError();
    for (cudaEvent_t ev : hc)
        if (ev) cudaEventDestroy(ev);
    if (s) return s;
    if (e != cudaSuccess) return fail(BM_ECUDA, "copy: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(BM_ECUDA, "sync: %s", cudaGetErrorString(e2));
    if (rep) {
        rep->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        rep->t_h2d_s = h2d_ms * 1e-3;
    }
    return BM_OK;
}

// ------------------------------------------------------------- step calls
// A one-worker context with explicit sizes, used by the step entry points.
static bm_status step_ctx(bm_fit_ctx* c, const float* X, long long m, int n, int k, long long s_cap,
                          unsigned long long seed, void* stream) {
    c->st = (cudaStream_t)stream;
    c->X = X; c->m = m; c->n = n; c->k = k; c->np = padded_dim(n);
    c->pol = bm_sample_policy{};
    c->pol.workers = 1; c->pol.passes = 1; c->pol.s_min = s_cap; c->pol.s_max = s_cap;
    c->bud = bm_budget{};
    c->bud.rounds = 1; c->bud.max_lloyd = 300; c->bud.tol = 1e-4; c->bud.kpp_candidates = 3;
    c->seed = seed;
    c->s_lo = c->s_hi = c->s_cap = std::max<long long>(s_cap, 1);
    c->w_lo = 0; c->w_hi = 1;
    c->max_cs = worker_max_cluster(c->np, k);
    c->cs = cluster_size(c->s_cap, c->max_cs, 0, rows_cap(c->np, k));
    if (c->cs == 0)
        return fail(BM_EINVAL, "sample of %lld rows above %lld", c->s_cap,
                    (long long)c->max_cs * rows_cap(c->np, k));
    c->Tcap = m > 0 ? draw_cap(m, std::min<long long>(c->s_cap, m)) : 1024;
    c->H = next_pow2(2 * c->Tcap);
    c->L_cap = 1;
    c->smem = worker_smem(c->np, k);
    cert_constants(c->np, c->gB, c->gp2);
    return alloc_workspace(c, 1);
}

struct CtxGuard {
    bm_fit_ctx* c;
    ~CtxGuard() { bm_fit_destroy(c); }
};

bm_status bm_sample(uint64_t seed, int32_t purpose, int32_t worker, int32_t round, int32_t pass, int64_t m,
                    int64_t s, int64_t* idx_out_dev, void* stream) {
    if (m < 1 || m >= (1ll << 31)) return fail(BM_EINVAL, "m = %lld out of range", (long long)m);
    if (s < 0 || s > m) return fail(BM_EINVAL, "s = %lld out of range [0, m]", (long long)s);
    if (s > 0 && !idx_out_dev) return fail(BM_EINVAL, "idx_out_dev is NULL");
    if (worker < 0 || worker >= (1 << 16) || round < 0 || round >= (1 << 24) || pass < 0 || pass >= (1 << 16))
        return fail(BM_EINVAL, "stream coordinates out of range");
    bm_fit_ctx* c = new bm_fit_ctx();
    CtxGuard guard{c};
    bm_status st = step_ctx(c, nullptr, m, 1, 1, s, seed, stream);
    if (st) return st;
    SampleArgs a = make_sample_args(c, kSampleStep, 1);
    a.idx = reinterpret_cast<long long*>(idx_out_dev); a.idx_stride = 0;
    a.step_s = s; a.purpose = purpose; a.worker = worker; a.rnd = round; a.pss = pass;
    CU(launch_sample(c->np, a, 1, c->st));
    Globals h;
    if ((st = read_globals(c, &h))) return st;
    return status_from_flags(h);
}

bm_status bm_gather(const float* X_dev, int64_t m, int32_t n, const int64_t* idx_dev, int64_t s,
                    float* S_out_dev, void* stream) {
    bm_status st = check_shape(m, n, 1);
    if (st) return st;
    if (s < 0) return fail(BM_EINVAL, "s < 0");
    if (s == 0) return BM_OK;
    if (!X_dev || !idx_dev || !S_out_dev) return fail(BM_EINVAL, "NULL pointer");
    bm_fit_ctx* c = new bm_fit_ctx();
    CtxGuard guard{c};
    if ((st = step_ctx(c, X_dev, m, n, 1, s, 0, stream))) return st;
    SampleArgs a = make_sample_args(c, kSampleGather, 1);
    a.idx = const_cast<long long*>(reinterpret_cast<const long long*>(idx_dev));
    a.idx_stride = 0;
    a.step_s = s;
    CU(launch_sample(c->np, a, 1, c->st));
    CU(launch_unpad(c->S, s, n, c->np, S_out_dev, c->st));
    Globals h;
    if ((st = read_globals(c, &h))) return st;
    return status_from_flags(h);
}

static bm_status stage_sample_and_centroids(bm_fit_ctx* c, const float* S_dev, long long s, const float* C_dev,
                                            int k) {
    CU(launch_pad(S_dev, s, c->n, c->np, c->S, c->st));
    CU(launch_pad(C_dev, k, c->n, c->np, c->Cw, c->st));
    CU(launch_prepass(S_dev, s * c->n, c->glob, 2 * sm_count(), c->st));
    CU(launch_prepass(C_dev, (long long)k * c->n, c->glob, 1, c->st));
    return BM_OK;
}

bm_status bm_kmeanspp(const float* S_dev, int64_t s, int32_t n, float* C_inout_dev, int32_t k,
                      const uint8_t* degenerate_dev, int32_t trials, uint64_t seed, int32_t worker,
                      int32_t round, int32_t pass, void* stream) {
    bm_status st = check_shape(s, n, k);
    if (st) return st;
    if (!S_dev || !C_inout_dev || !degenerate_dev) return fail(BM_EINVAL, "NULL pointer");
    if (trials < 1 || trials > 3) return fail(BM_EINVAL, "trials = %d out of range [1, 3]", trials);
    bm_fit_ctx* c = new bm_fit_ctx();
    CtxGuard guard{c};
    if ((st = step_ctx(c, S_dev, s, n, k, s, seed, stream))) return st;
    if ((st = stage_sample_and_centroids(c, S_dev, s, C_inout_dev, k))) return st;
    CU(cudaMemcpyAsync(c->deg, degenerate_dev, k, cudaMemcpyDeviceToDevice, c->st));
    WorkerArgs a = make_args(c, kModeStepKpp);
    a.trials = trials; a.step_s = s; a.step_worker = worker; a.step_round = round; a.step_pass = pass;
    CU(launch_worker(c->np, a, 1, c->st));
    CU(launch_unpad(c->Cw, k, n, c->np, C_inout_dev, c->st));
    Globals h;
    if ((st = read_globals(c, &h))) return st;
    return status_from_flags(h);
}

bm_status bm_lloyd(const float* S_dev, int64_t s, int32_t n, float* C_inout_dev, int32_t k, int32_t max_iter,
                   double tol, double* f_out_host, int32_t* iters_out_host, uint8_t* empty_out_dev,
                   void* stream) {
    bm_status st = check_shape(s, n, k);
    if (st) return st;
    if (!S_dev || !C_inout_dev) return fail(BM_EINVAL, "NULL pointer");
    if (max_iter < 0) return fail(BM_EINVAL, "max_iter < 0");
    bm_fit_ctx* c = new bm_fit_ctx();
    CtxGuard guard{c};
    if ((st = step_ctx(c, S_dev, s, n, k, s, 0, stream))) return st;
    if ((st = stage_sample_and_centroids(c, S_dev, s, C_inout_dev, k))) return st;
    CU(cudaMemsetAsync(c->deg, 0, k, c->st));
    WorkerArgs a = make_args(c, kModeStepLloyd);
    a.max_lloyd = max_iter; a.tol = tol; a.step_s = s;
    a.rows_cta = (int)((s + c->cs - 1) / c->cs);
    a.step_f = c->f_final; a.step_iters = (int*)c->L_buf;
    a.step_empty = empty_out_dev ? empty_out_dev : c->deg;
    CU(launch_worker(c->np, a, 1, c->st));
    CU(launch_unpad(c->Cw, k, n, c->np, C_inout_dev, c->st));
    double f = 0;
    int it = 0;
    CU(cudaMemcpyAsync(&f, c->f_final, 8, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(&it, c->L_buf, 4, cudaMemcpyDeviceToHost, c->st));
    Globals h;
    if ((st = read_globals(c, &h))) return st;
    if ((st = status_from_flags(h))) return st;
    if (f_out_host) *f_out_host = f;
    if (iters_out_host) *iters_out_host = it;
    return BM_OK;
}

bm_status bm_assign(const float* X_dev, int64_t m, int32_t n, const float* C_dev, int32_t k,
                    int32_t* labels_out_dev, double* f_out_host, bm_report* rep, void* stream) {
    bm_status st = check_shape(m, n, k, false);
    if (st) return st;
    if ((st = check_ptr(X_dev, "X_dev"))) return st;
    if (!C_dev) return fail(BM_EINVAL, "C_dev is NULL");
    cudaStream_t sm = (cudaStream_t)stream;
    const int np = padded_dim(n);
    const size_t smem = fullpass_smem_bytes(np, k, n);
    if (smem > kSmemLimit && !(fullpass_impl_setting() != 1 && tcx_eligible(X_dev, m, n, np, k)))
        return fail(BM_EINVAL, "k too large for the full pass");
    void* base = nullptr;
    const size_t gb = (sizeof(Globals) + 255) & ~(size_t)255;
    CU(lib_alloc(&base, gb + (size_t)k * np * 4, sm));
    Globals* g = (Globals*)base;
    float* Cp = (float*)((char*)base + gb);
    float gB, gp2;
    cert_constants(np, gB, gp2);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (rep) {
        CU(cudaEventCreate(&ev[0]));
        CU(cudaEventCreate(&ev[1]));
    }
    cudaError_t e;
    if ((e = cudaMemsetAsync(g, 0, sizeof(Globals), sm)) ||
        (e = launch_pad(C_dev, k, n, np, Cp, sm)) ||
        (e = launch_prepass(X_dev, m * n, g, 2 * sm_count(), sm)) ||
        (e = launch_prepass(C_dev, (long long)k * n, g, 1, sm)) ||
        (ev[0] && (e = cudaEventRecord(ev[0], sm))) ||
        (e = launch_fullpass(np, X_dev, m, n, Cp, k, nullptr, 1, labels_out_dev, g, gB, gp2, 0, sm_count(), sm)) ||
        (ev[1] && (e = cudaEventRecord(ev[1], sm)))) {
        cudaFreeAsync(base, sm);
        cudaStreamSynchronize(sm);
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        return fail(BM_ECUDA, "full pass launch: %s", cudaGetErrorString(e));
    }
    Globals h;
    e = cudaMemcpyAsync(&h, g, sizeof(Globals), cudaMemcpyDeviceToHost, sm);
    cudaFreeAsync(base, sm);
    const cudaError_t e2 = cudaStreamSynchronize(sm);
    float ms = 0.f;
    if (ev[0]) {
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(BM_ECUDA, "full pass: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    if ((st = status_from_flags(h))) return st;
    if (f_out_host) *f_out_host = h.f_full;
    if (rep) {
        memset(rep, 0, sizeof *rep);
        rep->f_full = h.f_full;
        rep->f_incumbent = h.f_full;
        rep->rescored_rows = (int64_t)h.rescored;
        rep->inexact_terms = (int64_t)h.inexact;
        rep->t_fullpass_s = ms * 1e-3;
        rep->fullpass_launches = 1;
    }
    return BM_OK;
}

// --------------------------------------------------- precision form (BF16)
bm_status bm_pack_bf16(const float* X_dev, int64_t m, int32_t n, void* Xb_out_dev, float* norms_out_dev,
                       void* stream) {
    if (m < 1 || m >= (1ll << 31)) return fail(BM_EINVAL, "m = %lld out of range", (long long)m);
    if (n < 1 || n > 64) return fail(BM_EINVAL, "n = %d out of range [1, 64]", n);
    if (!X_dev || !Xb_out_dev || !norms_out_dev) return fail(BM_EINVAL, "NULL pointer");
    if (((uintptr_t)Xb_out_dev) & 1023) return fail(BM_EINVAL, "Xb_out_dev must be 1024-byte aligned");
    const long long m_pad = (m + 127) / 128 * 128;
    CU(launch_pack_bf16(X_dev, m, n, m_pad, Xb_out_dev, norms_out_dev, (cudaStream_t)stream));
    float mx = 0.f;
    CU(cudaMemcpyAsync(&mx, norms_out_dev + m_pad, sizeof mx, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    if (!(mx < INFINITY)) return fail(BM_EINVAL, "X contains non-finite values");
    if (mx >= 0x1p126f) return fail(BM_EINVAL, "max |x| must be below 2^126");
    return BM_OK;
}

static bm_status assign_bf16(const void* Xb_dev, const float* norms_dev, const float* X_dev, int64_t m, int32_t n,
                             const float* C_dev, int32_t k, float tau, int certify, int32_t* labels_out_dev,
                             double* f_out_host, bm_report* rep, void* stream) {
    if (m < 1 || m >= (1ll << 31)) return fail(BM_EINVAL, "m = %lld out of range", (long long)m);
    if (n < 1 || n > 64) return fail(BM_EINVAL, "n = %d out of range [1, 64]", n);
    if (k < 1 || k > 256) return fail(BM_EINVAL, "k = %d out of range [1, 256] for the tensor-core pass", k);
    if (!Xb_dev || !norms_dev || !X_dev || !C_dev) return fail(BM_EINVAL, "NULL pointer");
    if (((uintptr_t)Xb_dev) & 1023) return fail(BM_EINVAL, "Xb_dev must be 1024-byte aligned");
    if (!(tau >= 0.f)) return fail(BM_EINVAL, "tau must be >= 0");
    if (tc_smem_bytes(k) == 0) return fail(BM_EINVAL, "k too large");
    cudaStream_t sm = (cudaStream_t)stream;
    void* base = nullptr;
    const size_t gb = (sizeof(Globals) + 255) & ~(size_t)255;
    CU(lib_alloc(&base, gb + (size_t)m * 16, sm));     // Globals, queue of m 16-byte entries
    Globals* g = (Globals*)base;
    void* queue = (char*)base + gb;
    float gB, gp2;
    cert_constants(64, gB, gp2);                   // rows of the precision form are 64 wide
    cudaError_t e;
    if ((e = cudaMemsetAsync(g, 0, sizeof(Globals), sm)) ||
        (e = launch_prepass(C_dev, (long long)k * n, g, 1, sm)) ||
        (e = launch_tc_fullpass(Xb_dev, norms_dev, X_dev, m, n, C_dev, k, tau, certify, labels_out_dev, queue, g,
                                gp2, sm_count(), sm))) {
        cudaFreeAsync(base, sm);
        cudaStreamSynchronize(sm);
        return fail(BM_ECUDA, "tensor-core pass launch: %s", cudaGetErrorString(e));
    }
    Globals h;
    e = cudaMemcpyAsync(&h, g, sizeof(Globals), cudaMemcpyDeviceToHost, sm);
    cudaFreeAsync(base, sm);
    const cudaError_t e2 = cudaStreamSynchronize(sm);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(BM_ECUDA, "tensor-core pass: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    bm_status st;
    if ((st = status_from_flags(h))) return st;
    if (f_out_host) *f_out_host = h.f_full;
    if (rep) {
        memset(rep, 0, sizeof *rep);
        rep->f_full = h.f_full;
        rep->f_incumbent = h.f_full;
        rep->rescored_rows = (int64_t)h.rescored;
        rep->inexact_terms = (int64_t)h.inexact;
    }
    return BM_OK;
}

bm_status bm_assign_bf16(const void* Xb_dev, const float* norms_dev, const float* X_dev, int64_t m, int32_t n,
                         const float* C_dev, int32_t k, float tau, int32_t* labels_out_dev, double* f_out_host,
                         bm_report* rep, void* stream) {
    return assign_bf16(Xb_dev, norms_dev, X_dev, m, n, C_dev, k, tau, 0, labels_out_dev, f_out_host, rep, stream);
}

bm_status bm_assign_bf16_certified(const void* Xb_dev, const float* norms_dev, const float* X_dev, int64_t m,
                                   int32_t n, const float* C_dev, int32_t k, float tau, int32_t* labels_out_dev,
                                   double* f_out_host, bm_report* rep, void* stream) {
    return assign_bf16(Xb_dev, norms_dev, X_dev, m, n, C_dev, k, tau, 1, labels_out_dev, f_out_host, rep, stream);
}

}  // extern "C"
