/*
 * bigmeans.h -- C ABI of libbigmeans, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of competitive-sample-size Big-means clustering
 * (R. Mussabayev, R. Mussabayev, "Superior Parallel Big Data Clustering
 * through Competitive Stochastic Sample Size Optimization in Big-means",
 * arXiv 2403.18766).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Data X is row-major m x n float32 (n fastest).  Centroids C are row-major
 *   k x n float32.  Labels are int32.  Sample indices are int64.
 * - Pointers named *_dev are CUDA device pointers owned by the caller; they
 *   must stay valid until the call returns.  Pointers named *_host are host
 *   pointers.  The library allocates its own workspace inside each call (or
 *   inside a bm_fit context) and frees it before returning (or on destroy).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   All device work is enqueued on it.  Every call returns only after its
 *   device work has completed, so outputs are ready on return.
 * - Errors are reported by status code only; nothing is thrown across the
 *   ABI.  bm_last_error() returns a thread-local message for the last
 *   non-OK status of the calling thread.
 * - Limits: 1 <= n <= 64, 1 <= k, k <= s_min, m < 2^31, s_max <= 524,272
 *   (16 CTAs of at most 32,767 sample rows per worker), and the centroid
 *   accumulators of one cluster must fit in shared memory
 *   (about k * round_up(n) * 32 bytes <= 220 KB; e.g. k <= 100 at n = 64).
 *   Non-finite values in X are rejected with BM_EINVAL.
 *
 * Numeric definition ("exact mode", the only mode so far)
 * -------------------------------------------------------
 * The paper fixes no precision, so per-point decisions are taken in FP32 with
 * one fixed operation order and every sum that feeds a decision is exact:
 *   d(x, c)   = FP32 direct form: t = x_d - c_d, acc = acc + t*t over
 *               ascending d, each operation rounded, no fused multiply-add;
 *   label(x)  = argmin_j d(x, c_j), lowest j on ties;
 *   f(C, P)   = the exact sum over x in P of d(x, c_label(x)), rounded once to
 *               double (Eq. 1 of the paper);
 *   centroid  = float( double(exact sum of members) / count ); an empty
 *               cluster keeps its centroid and is degenerate.
 * Exact sums are formed in integer fixed point; a value too small for the
 * fixed-point grid of its data set (below 2^-72 of the largest |x| for
 * coordinates, or below 2^-63 of the largest squared coordinate for distances)
 * is truncated and counted in bm_report.inexact_terms.
 */
#ifndef BIGMEANS_H
#define BIGMEANS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BM_OK = 0,
    BM_EINVAL = 1,     /* bad argument, unsupported size, non-finite X      */
    BM_ENOMEM = 2,     /* workspace allocation failed                       */
    BM_ECUDA = 3,      /* a CUDA runtime call failed (message has details)  */
    BM_ETIMEOUT = 4,   /* a bounded device wait ran out                     */
    BM_EINTERNAL = 5,  /* sampling ran out of draws or another device flag  */
    BM_EAGAIN = 6      /* serving: the job has not finished yet              */
} bm_status;

/* Purposes of the counter-based random streams (Philox4x64-10, Salmon et al.
 * SC'11).  key = {seed, purpose<<56 | worker<<40 | round<<16 | pass},
 * counter = {draw index, sub-stream, 0, 0}.  Bounded integers use Lemire's
 * multiply-and-reject rule on the four words of one block. */
typedef enum {
    BM_RNG_SIZE = 1,   /* s_w of a (worker, round)               Alg. 1      */
    BM_RNG_EVAL = 2,   /* sample that recomputes f_hat_w         Alg. 1      */
    BM_RNG_PASS = 3,   /* sample S_w of a pass                   Sec. 4.1    */
    BM_RNG_KPP = 4,    /* K-means++ draws of a pass              Sec. 4.1, 5 */
    BM_RNG_FINAL = 5   /* common sample of size s_opt            Alg. 1      */
} bm_rng_purpose;

/* Sample-size policy of Algorithm 1: each round every worker draws s_w
 * uniformly from [s_min, s_max] (set_len == 0) or uniformly from set[]
 * (set_len > 0, at most 16 entries).  s_max and the set entries are clipped
 * to m (Sec. 5: s_max = min(2 s, m)). */
typedef struct {
    int64_t s_min;
    int64_t s_max;
    int64_t set[16];
    int32_t set_len;
    int32_t workers;   /* W, competing workers (>= 1)                       */
    int32_t passes;    /* p, passes per round (Sec. 5: 10)                  */
    int32_t kind;      /* exploration of [s_min, s_max] (ignored with a set):
                          0 = uniform integer (the paper, Alg. 1);
                          1 = octave-uniform: octave i in [0, O) uniform,
                              then uniform inside [s_min 2^i, s_min 2^(i+1) - 1]
                              (the last octave ends at s_max), O = max(1,
                              least t with s_min 2^t >= s_max)              */
    int32_t exploit;   /* 0..100: percent chance that a worker's size for a
                          round is the rounded mean of L accumulated before
                          the round (exploiting the current best size, the
                          paper's future work, Sec. 7); 0 = the paper.
                          Nonzero values read L back to the host once per
                          round and draw no samples ahead                  */
} bm_sample_policy;

/* Stop conditions (Alg. 1 round count T and/or a wall-clock budget) and the
 * K-means settings of Sec. 5. */
typedef struct {
    int32_t rounds;                /* T; 0 = unlimited (seconds must be > 0)  */
    double seconds;                /* wall budget; 0 = none                   */
    int32_t max_lloyd;             /* Lloyd iterations cap (Sec. 5: 300)      */
    double tol;                    /* relative objective tolerance (1e-4)     */
    int32_t kpp_candidates;        /* K-means++ trials per centroid (3)       */
    int32_t eval_full_each_round;  /* 1: after each round evaluate f(C, X) of
                                      the worker with least f_hat_w and keep
                                      the least value seen (the incumbent)    */
} bm_budget;

/* Filled on return when the caller passes a non-NULL pointer. */
typedef struct {
    double f_full;          /* f(C_best, X), Eq. (1)                          */
    double f_incumbent;     /* least full f seen over rounds (or f_full)      */
    int64_t s_opt;          /* rounded mean of L                              */
    int32_t best_worker;    /* argmin of the common recheck                   */
    int32_t rounds_done;    /* rounds launched (with a time budget the workers
                               stop between passes at the deadline, so the last
                               round can be partial: see passes_done)         */
    int64_t passes_done;    /* passes over all workers                        */
    int64_t lloyd_iters;    /* centroid updates over all Lloyd runs           */
    int64_t assign_rows;    /* rows assigned inside Lloyd runs (sum s_w per
                               assignment); Lloyd pts*k = assign_rows * k     */
    int64_t accepts;        /* |L|                                            */
    int64_t L_sum;          /* sum of L                                       */
    int64_t rescored_rows;  /* rows whose FP32 expanded-form argmin was not
                               certified and were re-scored in direct form    */
    int64_t inexact_terms;  /* values truncated by the fixed-point grids      */
    double t_total_s;       /* wall time of the call                          */
    double t_worker_s;      /* device time of the worker-kernel launches
                               (CUDA events on the caller's stream)           */
    double t_fullpass_s;    /* device time of the full-data passes            */
    int64_t kernel_launches;    /* kernels of this library launched so far    */
    int64_t fullpass_launches;  /* full-pass launches                         */
    int64_t reseeded;       /* centroids (re)seeded by K-means++              */
    int64_t trace_cycles[16]; /* SM cycles on rank 0 of each worker cluster:
                                 [0] K-means++, [1] Lloyd assignment,
                                 [2] Lloyd exchange (barriers, reduction,
                                 update), [3] f_hat recompute, [4] sum of
                                 worker-kernel times, [5] longest worker
                                 kernel, [6] Lloyd assignments (count),
                                 [7] worker kernels (count), [8] assignment
                                 main loop, [9] its block reductions,
                                 [10] first cluster barrier, [11] owner
                                 update + objective, [12] second cluster
                                 barrier, [13] centroid pull + prep     */
    double t_sample_s;      /* device time of the sampling launches (part of
                               t_worker_s)                                    */
    double t_h2d_s;         /* host-buffer calls (bigmeans_fit_host, serving
                               jobs): device time of the copy of X to the
                               device (CUDA events); 0 elsewhere               */
} bm_report;

/* ---------------------------------------------------------------------------
 * bigmeans_fit -- Algorithm 1 end to end (Sec. 4.2, 4.3; settings Sec. 5).
 * X_dev: m x n float32 device, 16-byte aligned.  C_out_dev: k x n float32
 * device (written).  labels_out_dev: m int32 device, may be NULL.
 * Returns C_best, the labels Y of X and f(C_best, X) (in the report).
 * ------------------------------------------------------------------------- */
bm_status bigmeans_fit(const float* X_dev, int64_t m, int32_t n, int32_t k,
                       const bm_sample_policy* policy, const bm_budget* budget,
                       uint64_t seed, void* stream,
                       float* C_out_dev, int32_t* labels_out_dev,
                       bm_report* report_out);

/* Same as bigmeans_fit with host buffers: X_host is copied to the device,
 * C_out_host (k x n) and labels_out_host (m, may be NULL) are copied back,
 * all inside the call. */
bm_status bigmeans_fit_host(const float* X_host, int64_t m, int32_t n, int32_t k,
                            const bm_sample_policy* policy, const bm_budget* budget,
                            uint64_t seed, void* stream,
                            float* C_out_host, int32_t* labels_out_host,
                            bm_report* report_out);

/* ---------------------------------------------------------------------------
 * bigmeans_fit_dt -- bigmeans_fit with the storage type of X and the mode of
 * the full-data pass (the precision form of the full pass, NEXT-2, reached
 * through the fit entry point).
 *   dt = BM_F32:  X_dev is the m x n float32 matrix; X_master_dev is NULL or
 *                 X_dev.
 *   dt = BM_BF16: X_dev holds X packed by bm_pack_bf16 (m_pad x 128 bytes,
 *                 1024-byte aligned) and X_master_dev the m x n float32
 *                 master, the same matrix (required).
 *   mode = BM_MODE_EXACT: results of bigmeans_fit on the FP32 rows.
 *   mode = BM_MODE_FAST:  the same fit (samples, Lloyd and the recheck read
 *                 the FP32 rows: the exact-mode sums and certificates are
 *                 defined on them), then labels and f(C_best, X) from the
 *                 precision pass, bm_assign_bf16 with tau = 1e-3, on the BF16
 *                 rows (BM_F32: packed into a workspace of m_pad x 128 bytes
 *                 first); report->f_full is that f and report->rescored_rows
 *                 its re-scored rows.  n <= 64 and k <= 256 (checked before
 *                 the fit runs).
 * Other arguments, ownership and errors as for bigmeans_fit; BM_EINVAL for
 * an unknown dt or mode, a missing master, or a misaligned BF16 X_dev.
 * ------------------------------------------------------------------------- */
typedef enum { BM_F32 = 0, BM_BF16 = 1 } bm_dtype;
typedef enum { BM_MODE_EXACT = 0, BM_MODE_FAST = 1 } bm_mode;
bm_status bigmeans_fit_dt(const void* X_dev, const float* X_master_dev, bm_dtype dt,
                          int64_t m, int32_t n, int32_t k,
                          const bm_sample_policy* policy, const bm_budget* budget,
                          uint64_t seed, bm_mode mode, void* stream,
                          float* C_out_dev, int32_t* labels_out_dev,
                          bm_report* report_out);

/* ---------------------------------------------------------------------------
 * Staged fit: the same computation as bigmeans_fit, split so that rounds can
 * be run (and timed) one batch at a time.  bm_fit_create validates X,
 * allocates the workspace and initialises the workers (Alg. 1
 * initialisation); bm_fit_rounds runs the next `rounds` rounds;
 * bm_fit_finish does s_opt, the common recheck and the full assignment.
 * The context owns its workspace until bm_fit_destroy.
 * ------------------------------------------------------------------------- */
typedef struct bm_fit_ctx bm_fit_ctx;
bm_status bm_fit_create(const float* X_dev, int64_t m, int32_t n, int32_t k,
                        const bm_sample_policy* policy, const bm_budget* budget,
                        uint64_t seed, void* stream, bm_fit_ctx** out);
bm_status bm_fit_rounds(bm_fit_ctx* ctx, int32_t rounds);
/* bm_fit_rounds for several fits at once (Alg. 1 rounds of independent
 * Big-means problems, e.g. groups of competing workers with different k over
 * the same data): every round of every fit runs in ONE launch of the worker
 * kernel, each fit's workers planned together (see bm_set_worker_groups), so
 * workers of different fits share the GPU in one persistent grid.  Each fit's
 * results are identical to running it alone.  Requirements: 1 <= nfits <= 16
 * distinct fits on the current device whose n round up to the same padded
 * width (4, 8, 16, 32 or 64), no wall-clock budget, at most 160 workers in
 * all (else BM_EINVAL).  The work is enqueued on fits[0]'s stream; the other
 * fits' streams are ordered before it at the start and after it at the end.
 * Returns after the rounds have completed, with the first failing fit's
 * status. */
bm_status bm_fit_rounds_batch(bm_fit_ctx* const* fits, int32_t nfits, int32_t rounds);
bm_status bm_fit_finish(bm_fit_ctx* ctx, float* C_out_dev, int32_t* labels_out_dev,
                        bm_report* report_out);
/* ---------------------------------------------------------------------------
 * A fit sharded over ranks (one GPU each, X replicated: the paper's workers
 * all see the whole data set, Sec. 4.3).  Workers are independent until the
 * end of Alg. 1 except for the list L of improving sizes (Sec. 4.2) and the
 * final common recheck (Sec. 4.3), so rank r runs the workers [w_begin,
 * w_end) of a W-worker fit and the ranks exchange three small things on the
 * host (paper_2403_18766_gb300/shard.py):
 *   1. after the rounds, every rank's (sum of L, |L|) from bm_fit_report
 *      (L_sum, accepts), summed: s_opt = the mean of the global L, rounded
 *      half up and clipped to the size range (s_max if L is empty);
 *   2. bm_fit_recheck(ctx, s_opt, f): f_hat_w of the rank's workers on the
 *      common sample of size s_opt (the same draws on every rank), then the
 *      least (f_hat_w, w) over all ranks (lowest w on ties) picks w*;
 *   3. the owner of w* exports its centroids (bm_fit_worker_centroids), they
 *      are broadcast, and the full-data pass (bm_assign) gives labels and f.
 * The results equal the unsharded fit's bit for bit.
 * bm_fit_set_workers: before the first round; 0 <= w_begin < w_end <= W;
 *   not with the exploit policy (its sizes need L every round).  A shard's
 *   draws are the workers' own (keyed by their global index).
 * bm_fit_recheck: f_out_host receives w_end - w_begin doubles; s_opt must lie
 *   in the size range.  bm_fit_finish refuses a shard (BM_EINVAL).
 * bm_fit_worker_centroids: C_out_dev (k x n floats, device) receives worker
 *   w's current centroids; w must be one of the context's workers.
 * ------------------------------------------------------------------------- */
bm_status bm_fit_set_workers(bm_fit_ctx* ctx, int32_t w_begin, int32_t w_end);
bm_status bm_fit_recheck(bm_fit_ctx* ctx, int64_t s_opt, double* f_out_host);
bm_status bm_fit_worker_centroids(bm_fit_ctx* ctx, int32_t w, float* C_out_dev);
/* Counters and phase times so far (no final recheck); f_full and
 * f_incumbent hold the incumbent's full objective when
 * eval_full_each_round is set, else 0 and +inf. */
bm_status bm_fit_report(bm_fit_ctx* ctx, bm_report* report_out);
void bm_fit_destroy(bm_fit_ctx* ctx);

/* Checkpoint and resume of a staged fit (between rounds).
 * bm_fit_state_size: bytes of the state of ctx now (it grows with |L|).
 * bm_fit_export: waits for ctx's work, then writes its state to host_buf
 *   (bytes >= bm_fit_state_size): the workers' incumbent centroids,
 *   degenerate flags and f_hat, the list L of accepted sizes, the device
 *   counters of the report and the number of rounds run.  ctx is unchanged.
 * bm_fit_import: loads such a state into ctx, which must have been created
 *   by bm_fit_create on the same X with the same n, k, seed, size policy,
 *   max_lloyd, tol, kpp_candidates and eval_full_each_round (budget.rounds
 *   and budget.seconds may differ; L must fit the new budget), the same
 *   worker range, and must not have run a round yet.  Rounds run after the
 *   import continue the fit exactly: samples, seeds and sizes are functions
 *   of (seed, worker, round, pass), so in round-count mode the result equals
 *   the uninterrupted fit's bit for bit.  A wall-clock budget counts from the
 *   new context's creation.  BM_EINVAL for a truncated or foreign state or a
 *   context that differs (checked: shape, workers, passes, worker range,
 *   seed, a fingerprint of the policy and budget settings and of max |x|).
 *   host_buf is the caller's (plain host memory; the format is this
 *   library's, versioned, with no pointers in it). */
bm_status bm_fit_state_size(bm_fit_ctx* ctx, int64_t* bytes_out);
bm_status bm_fit_export(bm_fit_ctx* ctx, void* host_buf, int64_t bytes);
bm_status bm_fit_import(bm_fit_ctx* ctx, const void* host_buf, int64_t bytes);

/* ---------------------------------------------------------------------------
 * Step entry points (each one is a single step of the hot path; the fit runs
 * the same device code fused into one kernel per round).
 * ------------------------------------------------------------------------- */

/* a1 -- uniform sample without replacement (Sec. 4.1 "uniformly random
 * sample"): the first s distinct bounded draws r_0, r_1, ... in [0, m) of
 * stream (purpose, worker, round, pass), in order of first occurrence.
 * idx_out_dev: s int64 device.  Requires 0 <= s <= m. */
bm_status bm_sample(uint64_t seed, int32_t purpose, int32_t worker, int32_t round,
                    int32_t pass, int64_t m, int64_t s, int64_t* idx_out_dev,
                    void* stream);

/* a2 -- gather S[i, :] = X[idx[i], :] (Alg. 1, S_w).  S_out_dev: s x n. */
bm_status bm_gather(const float* X_dev, int64_t m, int32_t n, const int64_t* idx_dev,
                    int64_t s, float* S_out_dev, void* stream);

/* a3 -- greedy K-means++ re-seeding of the degenerate centroids (Sec. 4.1,
 * Sec. 5: `trials` candidates) on sample S (s x n), in increasing index
 * order; other centroids count as chosen.  The draws use stream
 * (BM_RNG_KPP, worker, round, pass).  C_inout_dev: k x n device;
 * degenerate_dev: k bytes device (nonzero = degenerate). */
bm_status bm_kmeanspp(const float* S_dev, int64_t s, int32_t n, float* C_inout_dev,
                      int32_t k, const uint8_t* degenerate_dev, int32_t trials,
                      uint64_t seed, int32_t worker, int32_t round, int32_t pass,
                      void* stream);

/* a4-a6 -- Lloyd K-means on S from C (Sec. 4.1; Sec. 5 stop rule): at most
 * max_iter centroid updates, stopping when f_prev - f_new <= tol * f_prev.
 * On return C_inout_dev holds the result, *f_out_host = f(C, S), *iters_out_host
 * the number of updates, empty_out_dev (k bytes, may be NULL) marks clusters
 * with no member in the final assignment. */
bm_status bm_lloyd(const float* S_dev, int64_t s, int32_t n, float* C_inout_dev,
                   int32_t k, int32_t max_iter, double tol, double* f_out_host,
                   int32_t* iters_out_host, uint8_t* empty_out_dev, void* stream);

/* a9 -- full-data pass (Alg. 1 last step; Eq. 1): labels of every row of X
 * and f(C, X).  labels_out_dev may be NULL.  *f_out_host receives f.  When
 * report_out is given it receives f, the re-scored row count and, in
 * t_fullpass_s, the device time of the pass kernel alone (CUDA events). */
bm_status bm_assign(const float* X_dev, int64_t m, int32_t n, const float* C_dev,
                    int32_t k, int32_t* labels_out_dev, double* f_out_host,
                    bm_report* report_out, void* stream);

/* ---------------------------------------------------------------------------
 * Precision form of the full-data pass (a9 with the distance contraction on
 * the tensor cores).
 *
 * bm_pack_bf16 -- pack X (m x n float32, n <= 64) into the layout the
 * tensor-core pass reads: m_pad = round_up(m, 128) rows of 64 bfloat16
 * (round to nearest, zero padded), 128 bytes per row, with the 16-byte
 * chunks of row r stored at chunk index (c XOR (r mod 8)); and
 * norms[r] = float(sum_d bf16(x_rd)^2), norms[m_pad] = max |x| (the
 * fixed-point grid of the objective).  Xb_out_dev: m_pad * 128 bytes,
 * 1024-byte aligned; norms_out_dev: m_pad + 1 floats.  Caller owns both;
 * they stay valid for any number of bm_assign_bf16 calls.  Non-finite X is
 * rejected with BM_EINVAL.
 *
 * bm_assign_bf16 -- labels of every row of X and the objective, with
 * g_j = ||c_j||^2 - 2 x.c_j formed from bfloat16 x and c with FP32
 * accumulation (tcgen05, kind::f16).  A row whose two least g differ by less
 * than tau * ||x||^2 is re-scored from the FP32 master X_dev with the exact
 * definition (FP32 direct form, lowest index on ties); otherwise its label is
 * the least g and its distance ||x||^2 + g (both in FP32).  f is the exact
 * sum of those distances rounded once to double; report->rescored_rows
 * counts re-scored rows.  A re-scored row is decided among its candidates,
 * the centroids whose g lies within the certificate bound of
 * bm_assign_bf16_certified of the least g (they contain the exact-mode
 * argmin), or over all k when it has more than 8.  1 <= k <= 256.  Labels
 * of rows that are not re-scored (the least g, lowest index on ties) can
 * differ from bm_assign where two centroids are within the BF16 error; the
 * difference in f is reported by the tests and the bench.  Workspace: 256 +
 * 16 m bytes, stream-ordered, freed before return.
 * ------------------------------------------------------------------------- */
bm_status bm_pack_bf16(const float* X_dev, int64_t m, int32_t n, void* Xb_out_dev,
                       float* norms_out_dev, void* stream);
bm_status bm_assign_bf16(const void* Xb_dev, const float* norms_dev, const float* X_dev,
                         int64_t m, int32_t n, const float* C_dev, int32_t k, float tau,
                         int32_t* labels_out_dev, double* f_out_host, bm_report* report_out,
                         void* stream);
/* bm_assign_bf16_certified -- bm_assign_bf16 with labels certified equal to
 * those of bm_assign: a row is also re-scored unless its two least g differ
 * by more than the bound of the BF16 form, 2 B + gp2 (g1 + B + ||x||^2) with
 * B = (2^-7 + 2^-13) (max ||c||^2 + 2 ||x|| max ||c||) (BF16 keeps 8
 * significant bits: rounding of x and c, FP32 accumulation, the final fma)
 * and gp2 the direct form's relative error at 64 dimensions; ||x||^2 is
 * bounded by norms[r] (1 + 2^-6).
 * That is, a row keeps the tensor-core label only where that label is
 * provably the exact-mode argmin.  Distances of rows that are not re-scored
 * are still ||x||^2 + g (f differs from bm_assign as for bm_assign_bf16).
 * Arguments, layout, ownership and errors as for bm_assign_bf16. */
bm_status bm_assign_bf16_certified(const void* Xb_dev, const float* norms_dev, const float* X_dev,
                                   int64_t m, int32_t n, const float* C_dev, int32_t k, float tau,
                                   int32_t* labels_out_dev, double* f_out_host, bm_report* report_out,
                                   void* stream);

/* ---------------------------------------------------------------------------
 * bm_assign_noalloc -- the full-data pass of bm_assign (labels of every row of
 * X and f(C, X), same numeric definition, same results) without allocating
 * any device memory.  The paper has no counterpart: this is a deployment
 * aid.  It is for callers that cannot allocate device memory when they need
 * the assignment, e.g. services that reserve all of their device memory in
 * their own pool at start-up, or loops with a fixed memory budget in which an
 * allocation could fail or wait for the device at an unpredictable moment.
 *   - Scratch: a fixed array of 65,792 bytes inside the library (a 256-byte
 *     accumulator record plus 16,384 floats of padded centroids).  Every GPU
 *     that loads the library holds it until the process exits.
 *   - Limit: k * round_up(n) <= 16,384, where round_up(n) is n rounded up to
 *     4, 8, 16, 32 or 64; larger sizes are rejected with BM_EINVAL (use
 *     bm_assign).  Other limits and arguments are those of bm_assign; the
 *     report is omitted.
 *   - The first call on each device looks up the scratch's device address
 *     (with that device current); make that first call before any stream
 *     capture begins.  Every call waits for its work to finish and reads
 *     f(C, X) back to the host before it returns.
 *   - Errors: the statuses of bm_assign for the same failures (the device
 *     flags are mapped by the same function), plus BM_EINVAL for the size
 *     limit above.
 *   - All calls share the one scratch array and each call clears its
 *     accumulators first, so calls that overlap on the GPU (different
 *     streams or threads without ordering) race: order them, e.g. issue them
 *     on one stream.  The call returns after its work has completed.
 * ------------------------------------------------------------------------- */
bm_status bm_assign_noalloc(const float* X_dev, int64_t m, int32_t n, const float* C_dev,
                            int32_t k, int32_t* labels_out_dev, double* f_out_host,
                            void* stream);

/* ---------------------------------------------------------------------------
 * bm_set_fullpass_impl / bm_last_fullpass_impl -- choice of implementation
 * for the full-data pass of Eq. (1) (bm_assign, bm_assign_noalloc and the
 * full passes inside a fit).  All implementations give identical labels and
 * f (the same FP32 direct-form definition, certified).
 *   impl 0 (default): by shape -- the tensor-core pass when n_pad * k > 512
 *          for n_pad <= 32 and n_pad * k > 1600 for n_pad = 64 (n_pad = n
 *          rounded up to 4, 8, 16, 32 or 64) and it applies, else the
 *          FP32-ALU pass;
 *   impl 1: always the FP32-ALU pass (register-tiled expanded form, certified,
 *          uncertain rows re-scored in FP32);
 *   impl 2: the tensor-core pass (tcgen05, split-TF32 products of the
 *          expanded form, certified, uncertain rows decided in the FP32
 *          direct form among the centroids the certificate leaves) where it
 *          applies -- n % 4 == 0, X 16-byte aligned, k <= 256 -- else the
 *          FP32-ALU pass.
 * Any other value is rejected with BM_EINVAL.  The setting is process-wide;
 * change it only while no call of this library is running.
 * bm_last_fullpass_impl returns which one the last full pass launched by the
 * calling thread used: 2 = tensor cores, 1 = FP32 ALU, 0 = none yet.
 * ------------------------------------------------------------------------- */
bm_status bm_set_fullpass_impl(int32_t impl);
int32_t bm_last_fullpass_impl(void);

/* ---------------------------------------------------------------------------
 * How the competing workers of a round (Sec. 4.2, Alg. 1) map onto the GPU.
 * Every round is one launch of the worker kernel for all workers of the fit.
 *   Worker groups (default): when every worker gets a cluster of 8 CTAs and
 *   the whole launch can be resident at once (a cooperative launch), the
 *   clusters the device can hold beyond one per worker go to the workers
 *   with the most sample rows per CTA, so a large sample spans up to 8
 *   clusters (64 CTAs) that add up their exact partial sums in global memory
 *   with a barrier among the group's CTAs; rows per CTA then stay about
 *   equal across workers.  Each such barrier is bounded (a few seconds):
 *   when one runs out the round returns BM_ETIMEOUT.
 *   Otherwise (bm_set_worker_groups(0), more workers than resident clusters,
 *   or bm_set_big_clusters(1)): one cluster per worker, all of the size the
 *   largest sample needs (the cluster tile below), in the same launch.
 * Results are identical either way (all reductions are exact).  Groups are
 * also off when a cooperative launch does not keep its cluster shape in the
 * process (checked once per device with a tiny probe launch): Nsight Compute
 * was seen to launch a cooperative cluster kernel without its clusters; the
 * worker kernel checks its launch shape and reports BM_EINVAL rather than
 * run so.
 * bm_set_worker_groups: 1 (default) allows groups, 0 disables them; other
 * values are BM_EINVAL.  Process-wide, read at each round's launch.
 * ------------------------------------------------------------------------- */
bm_status bm_set_worker_groups(int32_t on);
int32_t bm_get_worker_groups(void);

/* ---------------------------------------------------------------------------
 * Cluster tile of the worker kernel and its autotuner.
 * Without groups a worker runs as one thread-block cluster of up to 16 CTAs
 * with about `rows_per_cta` sample rows per CTA (default 1024).  The value
 * changes only speed: labels, centroids and objectives are identical for
 * every value (all reductions are exact).  The setting is process-wide and
 * read when a fit is created.
 * bm_set_rows_per_cta: 0 restores the default; otherwise 256 .. 32767.
 * bm_autotune_rows_per_cta: for each candidate, creates a 2-round fit of the
 * given arguments, runs round 0 as warm-up and times round 1 with CUDA
 * events on `stream`; sets the fastest candidate as the process value and
 * returns it in *best_out (per-candidate milliseconds in ms_out, n_candidates
 * entries, may be NULL).  1 <= n_candidates <= 16.
 * ------------------------------------------------------------------------- */
bm_status bm_set_rows_per_cta(int32_t rows);
int32_t bm_get_rows_per_cta(void);
/* on = 1: a worker whose cluster is at the size cap (16 CTAs) and still holds
 * more than rows_per_cta sample rows per CTA runs with 512-thread CTAs (one
 * per SM) instead of 256; on = 0 (default): always 256.  Speed only, as for
 * the tile.  Process-wide, read at each round's launch. */
bm_status bm_set_big_clusters(int32_t on);
int32_t bm_get_big_clusters(void);
/* How samples are drawn without replacement (Sec. 4.1: a uniform sample of
 * s distinct points, here the first s distinct values of the job's counter
 * stream of bounded draws, in order of first occurrence).  impl 0 (default):
 * a shared-memory bitmap of the m indices where it fits (m up to about
 * 1.37e6: the bitmap and the per-chunk hash table within 200 KB), else
 * per-job open-addressing tables in device memory; impl 1: always the
 * tables.
 * Both give identical samples.  Other values: BM_EINVAL.  Process-wide,
 * read when each sampling launch is prepared. */
bm_status bm_set_sampler_impl(int32_t impl);
int32_t bm_get_sampler_impl(void);
bm_status bm_autotune_rows_per_cta(const float* X_dev, int64_t m, int32_t n, int32_t k,
                                   const bm_sample_policy* policy, const bm_budget* budget, uint64_t seed,
                                   void* stream, const int32_t* candidates, int32_t n_candidates,
                                   int32_t* best_out, double* ms_out);

/* ---------------------------------------------------------------------------
 * bm_fit_footprint -- device bytes of the workspace a fit with these
 * arguments allocates (bigmeans_fit / bm_fit_create), without allocating.
 * Same argument checks as bm_fit_create.
 * ------------------------------------------------------------------------- */
bm_status bm_fit_footprint(int64_t m, int32_t n, int32_t k, const bm_sample_policy* policy,
                           const bm_budget* budget, int64_t* bytes_out);

/* ---------------------------------------------------------------------------
 * Serving (continuous batching of clustering jobs on one GPU).
 *
 * A context admits submitted jobs by device-memory footprint
 * (bm_job_footprint: the fit's workspace + X + C + labels) against
 * hbm_budget_bytes and runs up to max_active of them at once, each on its own
 * host runner thread and CUDA streams, so their kernels overlap on the GPU.
 * Whenever a job finishes, the queued jobs are scanned in arrival order and
 * every one that fits the freed memory is admitted (first fit; a job passed
 * over four times stops later arrivals from overtaking it).  A job runs
 * Algorithm 1 end to end as bigmeans_fit_host on the caller's host buffers:
 * X is copied to the device, stays resident with the centroids and the
 * per-worker statistics for the job's lifetime, and C (and labels, if
 * requested) are copied back before the job is reported done.  Results are
 * those of bigmeans_fit_host with the same arguments, whatever else runs.
 *
 * Ownership: the caller keeps X_host, C_out_host and labels_out_host alive
 * and untouched until the job is done (pinned memory makes the copies
 * asynchronous).  Times in bm_result are seconds since bm_ctx_create.
 * The runner threads start at the first bm_submit on the device current in
 * the submitting thread; bm_ctx_create itself makes no CUDA call.
 * A job with storage = 1 (BF16) keeps, beside its FP32 master, X packed in
 * BF16 on the device and takes its labels and f(C, X) from the tensor-core
 * precision pass (bm_assign_bf16 with its tau); bm_result.f_full is that
 * objective and report.f_full the exact-mode one of the same C.  Its
 * footprint includes the packed copy (128 + 4 bytes per row, n <= 64).
 * Errors: BM_EINVAL for bad arguments or shapes (checked at submit),
 * BM_ENOMEM at submit for a job larger than the whole budget; a job's own
 * failure is its bm_result.status (message via bm_job_error).
 * ------------------------------------------------------------------------- */
typedef struct bm_ctx bm_ctx;
typedef int64_t bm_job_id;
typedef struct {
    const float* X_host;         /* m x n row-major float32                    */
    int64_t m;
    int32_t n;
    int32_t k;
    bm_sample_policy policy;
    bm_budget budget;
    uint64_t seed;
    float* C_out_host;           /* k x n                                      */
    int32_t* labels_out_host;    /* m, or NULL                                 */
    int32_t storage;             /* 0: FP32; 1: X also held packed in BF16 for
                                    the full-data pass (bm_pack_bf16), whose
                                    labels and f come from bm_assign_bf16 with
                                    the re-score bound `tau`; the samples and the
                                    centroids still come from the FP32 master  */
    float tau;                   /* storage 1: re-score rule of bm_assign_bf16  */
} bm_job;
typedef struct {
    int32_t status;              /* the job's status; BM_EAGAIN until done      */
    int32_t state;               /* 0 queued, 1 running, 2 done                */
    double f_full;
    int64_t s_opt;
    double t_submit_s, t_admit_s, t_done_s;
    int64_t footprint_bytes;
    bm_report report;
} bm_result;
typedef struct {
    int64_t budget_bytes, in_use_bytes, peak_in_use_bytes;
    int32_t active, peak_active, queued, pad_;
    int64_t done;
    double now_s;
} bm_ctx_info;

bm_status bm_ctx_create(int64_t hbm_budget_bytes, int32_t max_active, bm_ctx** out);
bm_status bm_job_footprint(const bm_job* job, int64_t* bytes_out);
bm_status bm_submit(bm_ctx* ctx, const bm_job* job, bm_job_id* id_out);
/* BM_OK when the job is done (result filled), BM_EAGAIN while queued or
 * running (result holds the state and times so far). */
bm_status bm_poll(bm_ctx* ctx, bm_job_id id, bm_result* result_out);
/* Blocks until the job is done or timeout_s passes (timeout_s < 0: no limit). */
bm_status bm_wait(bm_ctx* ctx, bm_job_id id, double timeout_s, bm_result* result_out);
/* The error message of a failed job (empty if none), NUL-terminated. */
bm_status bm_job_error(bm_ctx* ctx, bm_job_id id, char* buf, int64_t len);
bm_status bm_ctx_stats(bm_ctx* ctx, bm_ctx_info* stats_out);
/* Drops queued jobs (each is reported done with status BM_EINVAL and the
 * message "dropped: ..."), waits for running ones, wakes every thread blocked
 * in bm_wait on this context and waits until they have returned, then frees
 * the context.  No other call on the context may start once bm_ctx_destroy
 * has been called (the context is freed when it returns). */
void bm_ctx_destroy(bm_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Device memory of the library.  Workspaces and the device copies of host
 * buffers come from a stream-ordered memory pool the library creates per
 * device; freed memory stays in that pool (it is not returned to the driver)
 * so that the next fit reuses it without mapping it again.
 * bm_trim_memory releases all currently unused pool memory of every device
 * the library has used.  (bm_assign_noalloc uses no pool memory.)
 * ------------------------------------------------------------------------- */
bm_status bm_trim_memory(void);

/* ---------------------------------------------------------------------------
 * Failure-injection hooks for tests (the paper has no counterpart: they check
 * the library's own failure handling without faulting a GPU).
 * bm_debug_fail_allocs: the next `count` device allocations of the library
 *   (workspaces and the device copies of host buffers) fail as if the device
 *   were out of memory, so the calls that make them return BM_ENOMEM and
 *   release what they had taken.  0 turns it off; count < 0 is BM_EINVAL.
 * bm_debug_set_wait_limit: limit of every bounded wait of the tensor-core
 *   exact full pass (bm_set_fullpass_impl, impl 2) launched afterwards:
 *   `polls` polls of an mbarrier, each suspending for at most `sleep_ns`
 *   (0: plain polls).  A wait that runs out sets the timeout flag; every role
 *   of the CTA stops, the copies and MMAs still in flight are waited for,
 *   tensor memory is freed, and the call returns BM_ETIMEOUT with the
 *   context still usable.  polls = 0 restores the default (2^18 polls of at
 *   most 20 us); sleep_ns above 1e6 is BM_EINVAL.
 * Both settings are process-wide; change them only while no call of this
 * library is running.
 * ------------------------------------------------------------------------- */
bm_status bm_debug_fail_allocs(int32_t count);
bm_status bm_debug_set_wait_limit(uint32_t polls, uint32_t sleep_ns);

/* Thread-local message for the last non-OK status of this thread. */
const char* bm_last_error(void);

/* Library version string. */
const char* bm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BIGMEANS_H */
