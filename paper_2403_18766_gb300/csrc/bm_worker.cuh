// Launch arguments of the fused worker kernel (host and device view).
#pragma once
#include <cstdint>

#include "bm_device.cuh"

namespace bm {

enum WorkerMode : int {
    kModeRounds = 0,      // Algorithm 1 rounds [round_begin, round_end)
    kModeFinalEval = 1,   // common recheck on the FINAL sample of size s_opt
    kModeStepKpp = 4,     // a3 on a given sample
    kModeStepLloyd = 5,   // a4-a6 on a given sample
};

// A worker whose sample is large may span several clusters of one launch (a
// group): the clusters exchange their partial sums through global memory and
// a barrier among the group's CTAs, which needs every CTA of the launch to be
// resident at once (a cooperative launch).
constexpr int kMaxGroup = 8;               // clusters per worker
constexpr int kMaxLaunchClusters = 160;    // entries of the cluster map

struct WorkerArgs {
    // data
    const float* X;
    long long m;
    int n, k;
    // policy / budget
    long long s_min, s_max;        // s_max already clipped to m
    long long set[16];
    int set_len;
    int W, P;
    int worker_base;                  // worker index of cluster 0 of this launch
    int max_lloyd, trials;
    double tol;
    unsigned long long seed;
    int round_begin, round_end;
    unsigned long long deadline_ns;   // %globaltimer deadline, 0 = none
    int mode;
    int cs;                           // CTAs per cluster
    int rows_cta;                     // most sample rows of one CTA in a Lloyd run of this launch
                                      // (sizes the label buckets in shared memory; 0: no Lloyd)
    // cluster map (ncl > 0): cluster c of the launch works for worker
    // cmap[c] & 0xfff of fit (cmap[c] >> 12) & 0xf, as cluster
    // (cmap[c] >> 16) & 0xff of a group of cmap[c] >> 24 clusters; ncl = 0:
    // cluster c is worker worker_base + c alone
    int ncl;
    int coop;                         // host: launch cooperatively (all CTAs resident at once)
    int k_smem;                       // host: k that sizes the launch's shared memory (0: k)
    unsigned cmap[kMaxLaunchClusters];
    // a launch for several fits (same padded width): the arguments of fit f
    // are batch[f] (device memory, each with this launch's cs, rows_cta,
    // ncl and cmap); null: a launch for this fit alone
    const WorkerArgs* batch;
    // group exchange in global memory (per worker; two parity halves)
    long long* xpart;                 // W x 2 x kMaxGroup x k x NP x 3 words
    int* xcnt;                        // W x 2 x kMaxGroup x k counts
    unsigned long long* xobj;         // W x 2 x kMaxGroup x 4 (objective partial, counters)
    unsigned* xbar;                   // W barrier counters (zero at launch)
    int* xabort;                      // W abort flags (zero at launch)
    float* xC;                        // W x k x NP centroids re-seeded by cluster 0
    int* xflag;                       // W x 2 deadline decisions
    int tpb;                          // threads per CTA: 256, or 512 (largest clusters)
    Globals* glob;
    // samples drawn by the sampling kernel: job (w, slot) = w * (P + 1) + slot
    float* S; long long S_stride;                 // s_cap * NP floats per job
    const int* job_s;                             // sample size of each job
    float* D2; long long D2_stride;               // s_cap per worker (K-means++ D^2)
    int* lab;                                     // s_cap per worker (labels, same stride)
    // worker state
    float* Cw;               // W * k * NP (canonical, read at launch start)
    float* Cw_cta;           // W * cs * k * NP (per-CTA working copies)
    unsigned char* deg;      // W * k
    double* fhat;            // W
    long long* L_buf; long long L_cap;
    double* f_final;         // W (common recheck)
    // step-mode I/O (worker 0 only)
    long long step_s;
    int step_purpose, step_worker, step_round, step_pass;
    double* step_f; int* step_iters; unsigned char* step_empty;
    // certificate constants (rounded up)
    float gB, gp2;
};

struct Xch {
    unsigned long long f_lo, f_hi;     // CTA partial of the exact objective
    unsigned long long inexact, rescored;
    long long wsum;                    // CTA sum of K-means++ weights
    long long pot[4];                  // CTA partial candidate potentials
    unsigned int maxbits;              // CTA max of D^2 bits
    int cand[4];                       // candidate row found by this CTA, -1 if none
    int stop;                          // rank-0 decision broadcast
    int flag;                          // rank-0 flag broadcast
    double fval;                       // rank-0 objective broadcast
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Objective partial of one CTA, pushed into rank 0's inbox (one slot per CTA).
struct ObjPart {
    unsigned long long f_lo, f_hi;     // 128-bit exact partial of the objective
    unsigned long long inexact, rescored;
};
// Rank 0's decision, pushed to every CTA of the cluster.
struct Decision {
    double f;
    int stop;
    int pad_;
};

// Exact coordinate sums: three int64 words per (cluster, dimension), value =
// w0 + w1 2^32 + w2 2^64 in units of 2^gx.  Each CTA holds the words of the
// clusters it owns (j % cs == rank, slot j / cs); every CTA adds its rows'
// contributions to the owner's words through distributed shared memory.
constexpr int kAccWords = 3;

template <int NP>
__host__ __device__ inline size_t worker_smem_bytes(int k) {
    size_t b = 0;
    b += align16((size_t)k * NP * 4);           // Ccur
    b += align16((size_t)k * NP * 4);           // Cnext (pushed by the owners)
    b += align16((size_t)k * 4);                // CC
    b += align16((size_t)k * NP * kAccWords * 8);  // OACC (owned slots; k of them when cs = 1)
    b += align16((size_t)k * 4);                // ocnt (owned counts)
    b += align16((size_t)k * 4);                // lcnt (this CTA's counts / bucket cursors)
    b += align16((size_t)(k + 1) * 4);          // lstart (bucket starts)
    b += align16((size_t)k) * 2;                // deg, emptyall
    b += align16(sizeof(Xch));
    b += align16(sizeof(ObjPart) * kMaxCluster);   // inbox (rank 0)
    b += align16(sizeof(Decision));
    b += align16(sizeof(unsigned __int128) * kMaxWarps);
    b += align16(8 * (kMaxWarps + 1));
    b += align16(4 * kMaxWarps);
    b += align16(sizeof(CertC));
    b += align16(8 * 16);
    return b;
}

// Shared memory of the label buckets of a Lloyd run: a 16-bit label and a
// 16-bit row offset per sample row of the CTA.
__host__ __device__ inline size_t bucket_smem_bytes(int rows_cta) { return align16((size_t)rows_cta * 4); }

cudaError_t launch_worker(int np, const WorkerArgs& a, int clusters, cudaStream_t st);
// Clusters of `cs` CTAs (256 threads, `smem` bytes each) that can be resident
// at once on the device (0 on error).
int worker_active_clusters(int np, int cs, size_t smem);
// Whether a cooperative launch keeps its cluster shape here (checked once per device).
bool cooperative_clusters_ok();
size_t worker_smem(int np, int k);
int worker_max_cluster(int np, int k);   // 16 if 16-CTA clusters fit, else 8

}  // namespace bm
