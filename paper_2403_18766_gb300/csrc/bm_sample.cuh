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
    int* job_s;                                // out: sample size of each job
    Globals* glob;
};

cudaError_t launch_sample(int np, const SampleArgs& a, int jobs, cudaStream_t st);

}  // namespace bm
