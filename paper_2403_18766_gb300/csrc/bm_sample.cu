// Sampling and gather (a1, a2) for all workers of a round in one launch.
//
// Algorithm 1 draws, for every worker and round, one sample to recompute
// f_hat_w and one sample per pass (Sec. 4.1: "a new uniformly random sample
// ... in each iteration").  None of them depends on clustering results, so
// they are all drawn up front, one CTA per (worker, sample) job, and gathered
// into contiguous padded rows that the worker kernel then reuses.
//
// A sample of size s is the first s distinct values among the bounded draws
// r_0, r_1, ... of its Philox stream, in order of first occurrence.  When a
// bitmap of the m values fits in shared memory, a job marks the values it has
// taken in that bitmap (sample_by_bitmap); otherwise it inserts its draws into
// an open-addressing table in global memory whose slots hold
// (generation << 32 | t): the generation of the job marks a slot as used, so
// the table never needs clearing, and the value of a slot is draws[t].  A
// draw t is kept when the slot of its value holds t itself (the least t).
#include <cstdint>

#include "bm_device.cuh"
#include "bm_sample.cuh"

namespace bm {

__device__ __forceinline__ unsigned int tab_hash(unsigned int r) { return r * 0x9E3779B1u; }

// Insert draw (r, t); the slot keeps the least t of value r.  Returns false
// only if the bounded retry or probe limits ran out (reported as an error).
__device__ bool tab_insert(unsigned long long* tab, unsigned int mask, unsigned int gen, unsigned int r,
                           unsigned int t, const unsigned int* draws) {
    unsigned int h = tab_hash(r) & mask;
    const unsigned long long mine = ((unsigned long long)gen << 32) | t;
    for (unsigned int probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = atomicAdd(&tab[h], 0ull);
        bool next = false;
        for (int spin = 0; spin < 1024 && !next; ++spin) {   // each retry sees a newer slot value
            if ((unsigned int)(cur >> 32) != gen) {          // free in this generation
                const unsigned long long prev = atomicCAS(&tab[h], cur, mine);
                if (prev == cur) return true;
                cur = prev;
                continue;
            }
            const unsigned int tt = (unsigned int)cur;
            if (draws[tt] != r) { next = true; break; }      // another value: next slot
            if (tt <= t) return true;                        // an earlier draw holds it
            const unsigned long long prev = atomicCAS(&tab[h], cur, mine);
            if (prev == cur) return true;
            cur = prev;
        }
        if (!next) return false;
        h = (h + 1u) & mask;
    }
    return false;
}

__device__ bool tab_is_first(const unsigned long long* tab, unsigned int mask, unsigned int gen,
                             unsigned int r, unsigned int t, const unsigned int* draws) {
    unsigned int h = tab_hash(r) & mask;
    for (unsigned int probe = 0; probe <= mask; ++probe) {
        const unsigned long long cur = tab[h];
        if ((unsigned int)(cur >> 32) != gen) return false;
        const unsigned int tt = (unsigned int)cur;
        if (draws[tt] == r) return tt == t;
        h = (h + 1u) & mask;
    }
    return false;
}

__device__ __forceinline__ long long pow2_at_least(long long v) {
    long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

// The same sample with a shared-memory bitmap of the m values (used when it
// fits): the draws are taken in chunks of kSampleDraws x kSampleThreads in
// counter order, kSampleDraws consecutive draws per thread.  A draw
// t of value r is the first occurrence of r when r's bit is clear at the
// start of t's chunk and t is the least draw of r inside the chunk (a small
// shared hash table keyed by r keeps that least t).  The chunk's first
// occurrences extend the sample in t order and then set their bits.  Returns
// the number of values found (s, or fewer when `cap` draws were not enough).
__device__ long long sample_by_bitmap(const SampleArgs& a, long long s, unsigned long long k1, long long cap,
                                      long long* idx, long long* red64) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* mini = reinterpret_cast<unsigned long long*>(smem_raw);   // kMiniSlots
    unsigned int* bits = reinterpret_cast<unsigned int*>(mini + kMiniSlots);      // bitmap_words
    const long long m = a.m;
    for (int i = threadIdx.x; i < a.bitmap_words; i += kSampleThreads) bits[i] = 0u;
    for (int i = threadIdx.x; i < kMiniSlots; i += kSampleThreads) mini[i] = ~0ull;
    __syncthreads();
    const unsigned long long thr = lemire_thr((unsigned long long)m);
    long long got = 0;
    constexpr int D = kSampleDraws;
    for (long long t0 = 0; t0 < cap && got < s; t0 += (long long)D * kSampleThreads) {     // block-uniform
        unsigned int r[D], h[D];
        bool cand[D];
        unsigned long long key[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {             // this thread's D consecutive draws
            const long long t = t0 + (long long)D * threadIdx.x + d;
            r[d] = 0; h[d] = 0; cand[d] = false;
            if (t < cap) {
                const P4 blk = philox4x64_10((unsigned long long)t, 0, 0, 0, a.seed, k1);
                r[d] = (unsigned int)uniform_below(blk, (unsigned long long)m, thr);
                cand[d] = ((bits[r[d] >> 5] >> (r[d] & 31)) & 1u) == 0u;
            }
            key[d] = ((unsigned long long)r[d] << 32) | (unsigned int)t;
            // at most D kSampleThreads keys in 2 D kSampleThreads slots: a
            // free slot always exists
            if (cand[d]) {
                h[d] = tab_hash(r[d]) & (kMiniSlots - 1);
                for (int p = 0; p < kMiniSlots; ++p) {
                    unsigned long long cur = mini[h[d]];
                    if (cur == ~0ull) {
                        cur = atomicCAS(&mini[h[d]], ~0ull, key[d]);
                        if (cur == ~0ull) break;
                    }
                    if ((unsigned int)(cur >> 32) == r[d]) { atomicMin(&mini[h[d]], key[d]); break; }
                    h[d] = (h[d] + 1u) & (kMiniSlots - 1);
                }
            }
        }
        __syncthreads();
        bool first[D];
        int cnt = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            first[d] = cand[d] && mini[h[d]] == key[d];
            cnt += first[d];
        }
        __syncthreads();
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (cand[d]) mini[h[d]] = ~0ull;             // empty again for the next chunk
            if (first[d]) atomicOr(&bits[r[d] >> 5], 1u << (r[d] & 31));
        }
        long long total;
        long long pos = got + block_exscan((long long)cnt, red64, &total);
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (first[d]) {
                if (pos < s) idx[pos] = (long long)r[d];
                ++pos;
            }
        got += total;
    }
    __syncthreads();
    return got < s ? got : s;
}

template <int NP>
__global__ void __launch_bounds__(kSampleThreads, 1) sample_kernel(const SampleArgs a) {
    __shared__ long long red64[kSampleThreads / 32 + 1];
    __shared__ int fail;
    const int job = blockIdx.x;
    int purpose = a.purpose, worker = a.worker, rnd = a.rnd, pss = a.pss;
    long long s = a.step_s;
    if (a.mode == kSampleRound) {
        const int slots = a.P + 1;
        worker = a.worker_base + job / slots;
        const int q = job % slots;
        rnd = a.rnd;
        purpose = (q < a.P) ? kPurposePass : kPurposeEval;
        pss = (q < a.P) ? q : 0;
        s = policy_size(a.sp, a.seed, stream_k1(kPurposeSize, worker, rnd, 0));
    } else if (a.mode == kSampleFinal) {
        long long s_lo = a.s_min, s_hi = a.s_max;
        if (a.set_len > 0) {
            s_lo = a.set[0]; s_hi = a.set[0];
            for (int i = 1; i < a.set_len; ++i) { s_lo = min(s_lo, a.set[i]); s_hi = max(s_hi, a.set[i]); }
        }
        const long long acc = (long long)a.glob->accepts, Ls = (long long)a.glob->L_sum;
        s = s_hi;
        if (acc > 0) s = min(max((2 * Ls + acc) / (2 * acc), s_lo), s_hi);
        if (a.step_s > 0) s = a.step_s;        // s_opt given by the host (a fit sharded over ranks)
        purpose = kPurposeFinal; worker = 0; rnd = 0; pss = 0;
        if (threadIdx.x == 0) a.glob->s_opt = (int)s;
    }
    long long* idx = a.idx + (long long)job * a.idx_stride;
    float* S = a.S + (long long)job * a.S_stride;
    if (a.mode != kSampleGather && a.bitmap_words > 0) {
        const unsigned long long k1 = stream_k1(purpose, worker, rnd, pss);
        const long long got = s > 0 ? sample_by_bitmap(a, s, k1, a.Tcap, idx, red64) : 0;
        if (got < s) {
            if (threadIdx.x == 0) atomicOr(&a.glob->err, kErrSample);
            s = 0;
        }
        __threadfence_block();
        __syncthreads();
    } else if (a.mode != kSampleGather) {
        const long long m = a.m;
        unsigned int* draws = a.draws + (long long)job * a.draws_stride;
        unsigned long long* tab = a.table + (long long)job * a.table_stride;
        // table size for this job: small samples need only about 2 s draws
        const long long H = (2 * s <= m) ? min(a.H, pow2_at_least(4 * s + 2048)) : a.H;
        const unsigned int mask = (unsigned int)(H - 1);
        const long long cap = min(a.Tcap, H / 2);
        const unsigned int gen = a.gen_base + (unsigned int)job;
        const unsigned long long k1 = stream_k1(purpose, worker, rnd, pss);
        const unsigned long long thr = lemire_thr((unsigned long long)m);
        long long T_done = 0, T = min(cap, s + (s * s) / m + 64);
        if (threadIdx.x == 0) fail = 1;
        __syncthreads();
        for (int batch = 0; batch < 64 && s > 0; ++batch) {
            for (long long t = T_done + threadIdx.x; t < T; t += kSampleThreads) {
                const P4 blk = philox4x64_10((unsigned long long)t, 0, 0, 0, a.seed, k1);
                draws[t] = (unsigned int)uniform_below(blk, (unsigned long long)m, thr);
            }
            __threadfence_block();
            __syncthreads();
            bool ok = true;
            for (long long t = T_done + threadIdx.x; t < T; t += kSampleThreads)
                ok &= tab_insert(tab, mask, gen, draws[t], (unsigned int)t, draws);
            if (!ok) atomicOr(&a.glob->err, kErrSample);
            __threadfence_block();
            __syncthreads();
            const long long ch = (T + kSampleThreads - 1) / kSampleThreads;
            const long long c0 = ch * threadIdx.x, c1 = min(T, c0 + ch);
            long long mine = 0;
            for (long long t = c0; t < c1; ++t) mine += tab_is_first(tab, mask, gen, draws[t], (unsigned int)t, draws);
            long long total;
            const long long excl = block_exscan(mine, red64, &total);
            if (total >= s) {
                long long pos = excl;
                for (long long t = c0; t < c1 && pos < s; ++t) {
                    const unsigned int r = draws[t];
                    if (tab_is_first(tab, mask, gen, r, (unsigned int)t, draws)) idx[pos++] = (long long)r;
                }
                if (threadIdx.x == 0) fail = 0;
                break;
            }
            if (T >= cap) break;
            T_done = T;
            T = min(cap, 2 * T);
        }
        __syncthreads();
        if (s > 0 && fail) {
            if (threadIdx.x == 0) atomicOr(&a.glob->err, kErrSample);
            s = 0;
        }
        __threadfence_block();
        __syncthreads();
    }
    if (a.mode == kSampleStep) {
        if (threadIdx.x == 0 && a.job_s) a.job_s[job] = (int)s;
        return;
    }
    // gather (padded rows, zeros in the padding); 16-byte loads when the rows
    // of X are 16-byte aligned.  A thread takes kGatherBatch items (16-byte
    // pieces of padded rows) at a time: their row indices, then their loads,
    // are all in flight together, so that a large sample does not pay two
    // dependent memory latencies per item.
    const int n = a.n;
    const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(a.X) & 15) == 0;
    constexpr int U = kGatherBatch;
    constexpr int RS = kSampleThreads / (NP / 4);          // rows a pass of the CTA covers
    static_assert(kSampleThreads % (NP / 4) == 0, "a thread keeps its piece q of every row");
    const int q = threadIdx.x % (NP / 4);                  // this thread's 16-byte piece of a row
    for (long long i0 = threadIdx.x / (NP / 4); i0 < s; i0 += (long long)U * RS) {
        long long row[U];
#pragma unroll
        for (int u = 0; u < U; ++u) row[u] = (i0 + u * RS < s) ? idx[i0 + u * RS] : 0;
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i0 + u * RS >= s) continue;
            if (row[u] >= 0 && row[u] < a.m) {
                const float* xr = a.X + row[u] * (long long)n;
                if (vec) {
                    if (4 * q < n) v[u] = __ldg(reinterpret_cast<const float4*>(xr) + q);
                } else {
                    v[u].x = (4 * q + 0 < n) ? xr[4 * q + 0] : 0.f;
                    v[u].y = (4 * q + 1 < n) ? xr[4 * q + 1] : 0.f;
                    v[u].z = (4 * q + 2 < n) ? xr[4 * q + 2] : 0.f;
                    v[u].w = (4 * q + 3 < n) ? xr[4 * q + 3] : 0.f;
                }
            } else if (q == 0) {
                atomicOr(&a.glob->err, kErrArgs);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * RS < s) reinterpret_cast<float4*>(S + (i0 + u * RS) * NP)[q] = v[u];
    }
    if (threadIdx.x == 0 && a.job_s) a.job_s[job] = (int)s;
}

template <int NP>
static cudaError_t launch_sample_t(const SampleArgs& a, int jobs, cudaStream_t st) {
    const size_t smem = sample_smem_bytes(a.bitmap_words);
    // every launch goes through allow_max_smem (which raises the limit once,
    // under a lock): a launch from one host thread must not race with the
    // attribute being set from another
    const cudaError_t e = allow_max_smem((const void*)sample_kernel<NP>);
    if (e != cudaSuccess) return e;
    sample_kernel<NP><<<jobs, kSampleThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sample(int np, const SampleArgs& a, int jobs, cudaStream_t st) {
    switch (np) {
        case 4: return launch_sample_t<4>(a, jobs, st);
        case 8: return launch_sample_t<8>(a, jobs, st);
        case 16: return launch_sample_t<16>(a, jobs, st);
        case 32: return launch_sample_t<32>(a, jobs, st);
        case 64: return launch_sample_t<64>(a, jobs, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bm
