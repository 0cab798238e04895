// Launch arguments of the sampling + gather kernel (a1, a2).
#pragma once
#include <cstdint>

#include "bm_device.cuh"

namespace bm {

enum SampleMode : int {
    kSampleRound = 0,   // every (worker, slot) job of one round: slots 0..P-1 passes, P = eval
    kSampleFinal = 1,   // the common sample of size s_opt (one job)
    kSampleStep = 2,    // one explicit stream, indices only
    kSampleGather = 3,  // one job, indices given in idx: gather only
};

// Sample-size policy of one round (Alg. 1 "s_w <- random size", and the
// exploration / exploitation variants of the paper's future work): the
// range, the optional set, and L as it stood at the start of the round.
struct SizePolicy {
    long long s_min, s_hi;      // range, s_hi clipped to m
    long long set[16];
    int set_len;
    int kind;                   // 0 uniform, 1 octave-uniform
    int exploit;                // percent
    long long L_sum, L_len;     // L before the round
};

// One bounded draw (c0, 0) of the size stream, same bits on host and device.
__host__ __device__ inline uint64_t size_draw(uint64_t seed, uint64_t k1, uint64_t c0, uint64_t bound) {
#ifdef __CUDA_ARCH__
    return draw_below(seed, k1, c0, 0, bound);
#else
    return host_draw_below(seed, k1, c0, 0, bound);
#endif
}

// s_w for the size stream k1 = (SIZE, w, round, 0): draw (1, 0) decides
// exploitation, draw (0, 0) the set entry / value / octave, draw (2, 0) the
// value inside the octave.
__host__ __device__ inline long long policy_size(const SizePolicy& p, uint64_t seed, uint64_t k1) {
    if (p.exploit > 0 && p.L_len > 0 && size_draw(seed, k1, 1, 100) < (uint64_t)p.exploit) {
        long long lo = p.s_min, hi = p.s_hi;
        if (p.set_len > 0) {
            lo = hi = p.set[0];
            for (int i = 1; i < p.set_len; ++i) {
                lo = p.set[i] < lo ? p.set[i] : lo;
                hi = p.set[i] > hi ? p.set[i] : hi;
            }
        }
        const long long v = (2 * p.L_sum + p.L_len) / (2 * p.L_len);     // mean, half up
        return v < lo ? lo : (v > hi ? hi : v);
    }
    if (p.set_len > 0) return p.set[size_draw(seed, k1, 0, (uint64_t)p.set_len)];
    if (p.kind == 1) {
        int t = 0;
        while ((p.s_min << t) < p.s_hi) ++t;
        const int octaves = t > 1 ? t : 1;
        const int i = (int)size_draw(seed, k1, 0, (uint64_t)octaves);
        const long long a = p.s_min << i;
        const long long b = (i == octaves - 1) ? p.s_hi : (p.s_min << (i + 1)) - 1;
        return a + (long long)size_draw(seed, k1, 2, (uint64_t)(b - a + 1));
    }
    return p.s_min + (long long)size_draw(seed, k1, 0, (uint64_t)(p.s_hi - p.s_min + 1));
}

struct SampleArgs {
    const float* X;
    long long m;
    int n;
    int mode;
    unsigned long long seed;
    int W, P, worker_base;
    long long s_min, s_max;
    long long set[16];
    int set_len;
    SizePolicy sp;                             // round mode: the size of each worker
    // explicit stream (kSampleStep)
    int purpose, worker, rnd, pss;
    long long step_s;
    // per-job buffers
    float* S; long long S_stride;              // s_cap * NP floats
    long long* idx; long long idx_stride;      // s_cap
    unsigned int* draws; long long draws_stride;
    long long Tcap;
    unsigned long long* table; long long H; long long table_stride;
    unsigned int gen_base;                     // generation of job 0 (tables are never cleared)
    int bitmap_words;                          // > 0: draw with a shared-memory bitmap of the m
                                               // values ((m + 31) / 32 words) instead of the tables
    int* job_s;                                // out: sample size of each job
    Globals* glob;
};

// Threads of a sampling CTA (one CTA per sample).
constexpr int kSampleThreads = 1024;
// Draws per thread in a chunk of the bitmap path, and the slots of its
// per-chunk hash table (2 per draw).
constexpr int kSampleDraws = 2;
constexpr int kMiniSlots = 2 * kSampleDraws * kSampleThreads;
// Items a thread of the gather has in flight at once.
constexpr int kGatherBatch = 8;
// Dynamic shared memory of a sampling launch.
inline size_t sample_smem_bytes(int bitmap_words) {
    return bitmap_words > 0 ? (size_t)kMiniSlots * 8 + (((size_t)bitmap_words * 4 + 15) & ~(size_t)15) : 0;
}
cudaError_t launch_sample(int np, const SampleArgs& a, int jobs, cudaStream_t st);

}  // namespace bm
