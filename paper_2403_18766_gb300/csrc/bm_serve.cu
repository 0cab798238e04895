// Serving context: clustering jobs of different m, n, k submitted at any
// time, admitted by device-memory footprint, run concurrently.
//
// Each admitted job runs Algorithm 1 end to end (bigmeans_fit_host: copy of X
// to the device, the rounds, the recheck, the full-data pass, copy back) on
// its own CUDA streams from one of `max_active` host runner threads, so the
// kernels of all admitted jobs overlap on the GPU.  Admission is continuous:
// whenever a job finishes (memory and a runner free up), the scheduler admits
// the first queued jobs whose footprint fits the remaining budget (first fit
// in arrival order, so one large job does not hold back small ones; a job
// that was passed over four times blocks later arrivals until it fits).  X,
// the centroids and the per-worker statistics of a job stay resident on the
// device until its result is copied back.  Results do not depend on what else
// runs: every fit is deterministic given (X, arguments, seed).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"

namespace bm {
bm_status set_error(bm_status s, const char* msg);
void set_thread_groups(bool ok);
}
using bm::set_error;

namespace {

struct Job {
    bm_job_id id;
    bm_job spec;
    int64_t footprint;
    int passed_over = 0;
    int state = 0;                 // 0 queued, 1 running, 2 done
    bm_status status = BM_OK;
    std::string error;
    bm_report report{};
    double f_result = 0;           // f(C, X) of the job's full-data pass
    double t_submit = 0, t_admit = 0, t_done = 0;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

namespace {

// A BF16-stored job: the fit on the FP32 master (exact mode), then its
// labels and objective from the BF16 tensor-core pass over the packed copy.
bm_status run_bf16_job(const bm_job& s, cudaStream_t st, bm_report* rep, double* f_out) {
    const int64_t m = s.m, m_pad = (m + 127) / 128 * 128;
    float* Xd = nullptr; float* Cd = nullptr; int32_t* Ld = nullptr; float* norms = nullptr;
    unsigned char* raw = nullptr;
    bm_status r = BM_OK;
    auto alloc = [&](void** p, size_t bytes) {
        if (r == BM_OK && cudaMallocAsync(p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            r = set_error(BM_ENOMEM, "device buffers of a BF16-stored job");
        }
    };
    alloc((void**)&Xd, (size_t)m * s.n * 4);
    alloc((void**)&Cd, (size_t)s.k * s.n * 4 + 16);
    alloc((void**)&raw, (size_t)m_pad * 128 + 1024);
    alloc((void**)&norms, (size_t)(m_pad + 1) * 4);
    alloc((void**)&Ld, (size_t)m * 4);
    cudaEvent_t hc[2] = {nullptr, nullptr};              // around the copy of X
    if (cudaEventCreate(&hc[0]) != cudaSuccess || cudaEventCreate(&hc[1]) != cudaSuccess) cudaGetLastError();
    if (hc[0]) cudaEventRecord(hc[0], st);
    if (r == BM_OK && cudaMemcpyAsync(Xd, s.X_host, (size_t)m * s.n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        r = set_error(BM_ECUDA, "copy of X");
    if (hc[1]) cudaEventRecord(hc[1], st);
    if (r == BM_OK) r = bigmeans_fit(Xd, m, s.n, s.k, &s.policy, &s.budget, s.seed, st, Cd, nullptr, rep);
    void* Xb = raw ? (void*)(raw + ((1024 - ((uintptr_t)raw & 1023)) & 1023)) : nullptr;
    if (r == BM_OK) r = bm_pack_bf16(Xd, m, s.n, Xb, norms, st);
    bm_report rb{};
    if (r == BM_OK) r = bm_assign_bf16(Xb, norms, Xd, m, s.n, Cd, s.k, s.tau, Ld, f_out, &rb, st);
    if (r == BM_OK && cudaMemcpyAsync(s.C_out_host, Cd, (size_t)s.k * s.n * 4, cudaMemcpyDeviceToHost, st) !=
                          cudaSuccess)
        r = set_error(BM_ECUDA, "copy of C");
    if (r == BM_OK && s.labels_out_host &&
        cudaMemcpyAsync(s.labels_out_host, Ld, (size_t)m * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        r = set_error(BM_ECUDA, "copy of labels");
    for (void* p : {(void*)Xd, (void*)Cd, (void*)raw, (void*)norms, (void*)Ld})
        if (p) cudaFreeAsync(p, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && r == BM_OK) r = set_error(BM_ECUDA, "job stream");
    float h2d_ms = 0.f;
    if (hc[0] && hc[1] && cudaEventElapsedTime(&h2d_ms, hc[0], hc[1]) != cudaSuccess) cudaGetLastError();
    for (cudaEvent_t ev : hc)
        if (ev) cudaEventDestroy(ev);
    if (rep) {
        rep->rescored_rows += rb.rescored_rows;
        rep->t_h2d_s = h2d_ms * 1e-3;
    }
    return r;
}

}  // namespace

struct bm_ctx {
    int64_t budget = 0;
    int max_active = 1;
    int device = -1;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;          // runners: a job may be admissible
    std::condition_variable done_cv;     // waiters: a job finished
    std::deque<Job*> queue;
    std::map<bm_job_id, std::unique_ptr<Job>> jobs;
    std::vector<std::thread> runners;
    bm_job_id next_id = 1;
    int64_t in_use = 0, peak_in_use = 0;
    int active = 0, peak_active = 0;
    int64_t done_count = 0;
    int waiters = 0;                     // threads inside bm_wait
    bool stop = false;

    // First fit in arrival order; a job passed over 4 times blocks later
    // arrivals (no starvation).  Called with mu held.
    Job* admit() {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            Job* j = *it;
            if (j->footprint <= budget - in_use) {
                for (auto jt = queue.begin(); jt != it; ++jt) (*jt)->passed_over++;
                queue.erase(it);
                return j;
            }
            if (j->passed_over >= 4) return nullptr;
        }
        return nullptr;
    }

    void runner() {
        if (device >= 0) cudaSetDevice(device);
        // jobs run side by side: no worker groups (their cooperative
        // launches would wait for the other jobs' kernels)
        bm::set_thread_groups(false);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        for (;;) {
            Job* j = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || (j = admit()) != nullptr; });
                if (!j) break;                                // stopping
                in_use += j->footprint;
                peak_in_use = std::max(peak_in_use, in_use);
                active++;
                peak_active = std::max(peak_active, active);
                j->state = 1;
                j->t_admit = now_s(t0);
            }
            const bm_job& s = j->spec;
            bm_report rep{};
            double f_bf16 = 0.0;
            const bm_status st_fit = s.storage == 1
                                         ? run_bf16_job(s, st, &rep, &f_bf16)
                                         : bigmeans_fit_host(s.X_host, s.m, s.n, s.k, &s.policy, &s.budget, s.seed,
                                                             st, s.C_out_host, s.labels_out_host, &rep);
            const std::string err = st_fit ? std::string(bm_last_error()) : std::string();
            {
                std::lock_guard<std::mutex> lk(mu);
                in_use -= j->footprint;
                active--;
                j->status = st_fit;
                j->error = err;
                j->report = rep;
                j->f_result = (s.storage == 1) ? f_bf16 : rep.f_full;
                j->state = 2;
                j->t_done = now_s(t0);
                done_count++;
            }
            done_cv.notify_all();
            cv.notify_all();                                  // memory freed: admit more
        }
        if (st) cudaStreamDestroy(st);
    }
};

namespace {

void fill_result(const Job& j, bm_result* r) {
    memset(r, 0, sizeof *r);
    r->status = (j.state == 2) ? j.status : BM_EAGAIN;
    r->state = j.state;
    r->f_full = j.f_result;
    r->s_opt = j.report.s_opt;
    r->t_submit_s = j.t_submit;
    r->t_admit_s = j.t_admit;
    r->t_done_s = j.t_done;
    r->footprint_bytes = j.footprint;
    r->report = j.report;
}

}  // namespace

extern "C" {

bm_status bm_ctx_create(int64_t hbm_budget_bytes, int32_t max_active, bm_ctx** out) {
    if (!out) return set_error(BM_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0) return set_error(BM_EINVAL, "hbm_budget_bytes must be > 0");
    if (max_active < 1 || max_active > 64) return set_error(BM_EINVAL, "max_active out of range [1, 64]");
    bm_ctx* c = new bm_ctx();
    c->budget = hbm_budget_bytes;
    c->max_active = max_active;
    c->t0 = std::chrono::steady_clock::now();
    *out = c;
    return BM_OK;
}

bm_status bm_job_footprint(const bm_job* job, int64_t* bytes_out) {
    if (!job || !bytes_out) return set_error(BM_EINVAL, "job and bytes_out are required");
    if (job->storage != 0 && job->storage != 1) return set_error(BM_EINVAL, "storage must be 0 (FP32) or 1 (BF16)");
    if (job->storage == 1 && (job->n > 64 || !(job->tau >= 0.f)))
        return set_error(BM_EINVAL, "BF16 storage needs n <= 64 and tau >= 0");
    int64_t ws = 0;
    const bm_status s = bm_fit_footprint(job->m, job->n, job->k, &job->policy, &job->budget, &ws);
    if (s) return s;
    int64_t dev = job->m * job->n * 4 + (job->k * (int64_t)job->n * 4 + 16) +
                  (job->labels_out_host ? job->m * 4 : 0);
    if (job->storage == 1) {
        const int64_t m_pad = (job->m + 127) / 128 * 128;
        dev += m_pad * 128 + 1024 + (m_pad + 1) * 4 + job->m * 4;    // packed rows, norms, labels
        dev += 256 + job->m * 16;                                      // the precision pass's queue
    }
    *bytes_out = ws + dev + 6 * 256;                          // allocation rounding
    return BM_OK;
}



bm_status bm_submit(bm_ctx* c, const bm_job* job, bm_job_id* id_out) {
    if (!c || !job || !id_out) return set_error(BM_EINVAL, "ctx, job and id_out are required");
    if (!job->X_host || !job->C_out_host) return set_error(BM_EINVAL, "X_host and C_out_host are required");
    int64_t fp = 0;
    const bm_status s = bm_job_footprint(job, &fp);
    if (s) return s;
    if (fp > c->budget) return set_error(BM_ENOMEM, "job footprint above the context's whole budget");
    auto j = std::make_unique<Job>();
    j->spec = *job;
    j->footprint = fp;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->stop) return set_error(BM_EINVAL, "context is being destroyed");
        if (c->runners.empty()) {                             // start the runners on first use
            int dev = 0;
            const cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return set_error(BM_ECUDA, cudaGetErrorString(e));
            c->device = dev;
            for (int i = 0; i < c->max_active; ++i) c->runners.emplace_back([c] { c->runner(); });
        }
        j->id = c->next_id++;
        j->t_submit = now_s(c->t0);
        *id_out = j->id;
        c->queue.push_back(j.get());
        c->jobs[j->id] = std::move(j);
    }
    c->cv.notify_all();
    return BM_OK;
}

bm_status bm_poll(bm_ctx* c, bm_job_id id, bm_result* r) {
    if (!c || !r) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return BM_EINVAL;
    fill_result(*it->second, r);
    return (it->second->state == 2) ? BM_OK : BM_EAGAIN;
}

bm_status bm_wait(bm_ctx* c, bm_job_id id, double timeout_s, bm_result* r) {
    if (!c || !r) return BM_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return BM_EINVAL;
    Job* j = it->second.get();
    const auto pred = [&] { return j->state == 2; };
    c->waiters++;
    if (timeout_s < 0) c->done_cv.wait(lk, pred);
    else c->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
    fill_result(*j, r);
    const bm_status st = (j->state == 2) ? BM_OK : BM_EAGAIN;
    if (--c->waiters == 0) c->done_cv.notify_all();      // bm_ctx_destroy may be waiting for this
    return st;
}

bm_status bm_job_error(bm_ctx* c, bm_job_id id, char* buf, int64_t len) {
    if (!c || !buf || len < 1) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->jobs.find(id);
    if (it == c->jobs.end()) return BM_EINVAL;
    const std::string& e = it->second->error;
    const size_t n = std::min<size_t>(e.size(), (size_t)len - 1);
    memcpy(buf, e.data(), n);
    buf[n] = 0;
    return BM_OK;
}

bm_status bm_ctx_stats(bm_ctx* c, bm_ctx_info* s) {
    if (!c || !s) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    memset(s, 0, sizeof *s);
    s->budget_bytes = c->budget;
    s->in_use_bytes = c->in_use;
    s->peak_in_use_bytes = c->peak_in_use;
    s->active = c->active;
    s->peak_active = c->peak_active;
    s->queued = (int32_t)c->queue.size();
    s->done = c->done_count;
    s->now_s = now_s(c->t0);
    return BM_OK;
}

void bm_ctx_destroy(bm_ctx* c) {
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
        for (Job* j : c->queue) {                             // queued jobs are dropped:
            j->state = 2;                                     // reported as done, with an error
            j->status = BM_EINVAL;
            j->error = "dropped: the serving context was destroyed before the job was admitted";
            j->t_done = now_s(c->t0);
        }
        c->queue.clear();
    }
    c->cv.notify_all();
    c->done_cv.notify_all();
    for (auto& t : c->runners) t.join();                      // running jobs finish
    {
        // threads blocked in bm_wait return (every job is done now) before
        // the context goes away
        std::unique_lock<std::mutex> lk(c->mu);
        c->done_cv.notify_all();
        c->done_cv.wait(lk, [&] { return c->waiters == 0; });
    }
    delete c;
}

}  // extern "C"
