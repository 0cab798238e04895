// Precision form of the full-data pass (Alg. 1 last step, Eq. 1) on the
// fifth-generation tensor cores of sm_103a.
//
// X is packed once into BF16 rows of 64 elements (128 bytes, zero padded),
// with the 16-byte chunks of every row XOR-swizzled by (row mod 8): exactly
// the 128-byte-swizzle K-major layout the tensor core reads from shared
// memory, so a plain 1-D bulk copy (TMA) of 128 consecutive rows lands in
// shared memory ready to use.  The pack also stores fl(||x_bf16||^2).
//
// Per tile of 128 rows the MMA thread issues four tcgen05.mma (M = 128, N =
// k rounded up to 16, K = 16 each) of X_bf16 x C_bf16^T into one of G
// tensor-memory accumulators (FP32), so that the MMAs and copies of later
// tiles overlap the epilogue of earlier ones; four warps of an epilogue group
// read their 32 rows with tcgen05.ld, form g_j = ||c_j||^2 - 2 x.c_j, keep
// the two least, and
//  * if g2 - g1 >= tau * ||x||^2: label = j1, distance = ||x||^2 + g1;
//  * otherwise the row goes to a queue with its candidates (the centroids
//    whose g lies within the certificate threshold of the BF16 form of g1),
//    and a second kernel re-scores the queued rows from the FP32 master copy
//    with the exact definition (FP32 direct form, lowest index on ties) over
//    the candidates, which contain the exact-mode argmin.
// The objective is the exact sum of the per-row distances (integer fixed
// point), rounded once.
#include <algorithm>
#include <mutex>
#include <cstdint>

#include <cuda_bf16.h>

#include "bm_device.cuh"
#include "bm_tcgen05.cuh"

namespace bm {

constexpr int kTcRows = 128;           // rows per tile (MMA M)
constexpr int kTcK = 64;               // packed row width (BF16 elements)

// ------------------------------------------------------------------ pack
// Xb[r][chunk c ^ (r & 7)] holds elements 8c .. 8c+7 of row r (BF16, RN);
// rows m .. m_pad-1 and elements n .. 63 are zero.  norms[r] = fl(sum x_b^2).
// Xb may be NULL: the norms (and the max |x|) alone.
__global__ void pack_bf16_kernel(const float* __restrict__ X, long long m, int n, long long m_pad,
                                 __nv_bfloat16* __restrict__ Xb, float* __restrict__ norms) {
    const long long total = Xb ? m_pad * (kTcK / 8) : 0;       // 16-byte chunks (none: norms only)
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / (kTcK / 8);
        const int c = (int)(e % (kTcK / 8));
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int d = 8 * c + i;
            v[i] = __float2bfloat16_rn((r < m && d < n) ? X[r * n + d] : 0.f);
        }
        const int pc = c ^ (int)(r & 7);
        *reinterpret_cast<uint4*>(Xb + r * kTcK + 8 * pc) = *reinterpret_cast<const uint4*>(v);
    }
    unsigned int mx = 0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < m_pad;
         r += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int d = 0; d < n && r < m; ++d) {
            const float x = X[r * n + d];
            mx = max(mx, __float_as_uint(x) & 0x7fffffffu);
            const float b = __bfloat162float(__float2bfloat16_rn(x));
            acc = __fmaf_rn(b, b, acc);
        }
        norms[r] = acc;
    }
    // norms[m_pad] = max |x| (bits; non-finite values compare above all finite ones)
    if (mx) atomicMax(reinterpret_cast<unsigned int*>(norms + m_pad), mx);
}

// ------------------------------------------------------- shape and layout
using tc::s_addr;

constexpr int kTcTileBytes = kTcRows * 128;   // one tile of packed rows
constexpr int kTcMaxStages = 8;
constexpr int kTcCand = 8;                    // candidates carried by a queued row
__host__ __device__ constexpr int tc_threads(int groups) { return 32 * (4 * groups + 2); }

struct TcShape {
    int Npad;            // MMA N: k rounded up to 16
    int acc_stride;      // tensor-memory columns per accumulator
    int tmem_cols;       // columns allocated (a power of two >= 32)
    int stages;          // X tiles in flight
    int groups;          // epilogue warpgroups = accumulators (4 or 2)
    tc::WaitLimit wait;  // limit of every bounded wait
};

// Shared memory: [X stages: stages x 16 KB][B: Npad x 128 B][ccb: Npad floats]
// (stages and B 1024-byte aligned).
__host__ __device__ inline size_t tc_smem_bytes(const TcShape& s) {
    return 1024 + (size_t)s.stages * kTcTileBytes + (size_t)s.Npad * 128 + (size_t)s.Npad * 4;
}

// Four accumulators where tensor memory allows (k <= 128), else two; as many
// stages as fit in 200 KB, at most kTcMaxStages.
bool tc_shape(int k, TcShape& s) {
    if (k < 1 || k > 256) return false;
    s.Npad = (k + 15) & ~15;
    s.acc_stride = (s.Npad + 31) & ~31;
    s.groups = 4 * s.acc_stride <= 512 ? 4 : 2;
    s.tmem_cols = 32;
    while (s.tmem_cols < s.groups * s.acc_stride) s.tmem_cols <<= 1;
    for (s.stages = kTcMaxStages; s.stages >= 2; --s.stages)
        if (tc_smem_bytes(s) <= 200 * 1024) return true;
    return false;
}

// ------------------------------------------------------ the full pass
// Roles of a CTA (one per SM, persistent over tiles blockIdx.x + i * grid):
//   * warp 4 G: the producer; one bulk copy (TMA) of 128 packed rows per tile
//     into a ring of stages;
//   * warp 4 G + 1: the MMA issuer; four tcgen05.mma (K = 16 each) of a tile
//     into accumulator (i mod G) once that accumulator is free, then two
//     commits: one tells epilogue group (i mod G) that the accumulator is
//     ready, one frees the stage for the producer;
//   * warps 0 .. 4 G - 1: G epilogue warpgroups; group b takes the tiles
//     i = b (mod G), warp q of a group the tensor-memory lanes 32 q .. 32 q +
//     31 (= the tile's rows).  Per row: g_j = fl(||c_j||^2 - 2 acc_j), the two
//     least in four interleaved chains, the rule, and for a close call a
//     second read of the accumulator that lists its candidates; then the
//     accumulator is handed back to the MMA issuer.
// A close call (g2 - g1 < tau ||x||^2, or with `certify` a row whose BF16 gap
// does not pass the certificate) goes to the queue with its candidates: the
// centroids whose g is at most fl_ru(g1 + thr), thr the certificate
// threshold.  Any other centroid has a larger FP32 direct-form distance than
// the centroid of g1 (the certificate's argument with the BF16 error factor),
// so the exact-mode label is the least direct form among the candidates,
// lowest index on ties.  A row with more than kTcCand candidates (or none,
// which only a NaN threshold gives) is flagged for all k.  Queue entry (16
// bytes): row | flag << 31, the candidate count, and up to eight candidate
// bytes in two words.  A settled row's label is the first column whose g
// equals g1, found by the same second read (threshold g1).
template <int NG>
__global__ void __launch_bounds__(tc_threads(NG), 1)
tc_fullpass_kernel(const __nv_bfloat16* __restrict__ Xb, const float* __restrict__ xnorm, long long m, int n,
                   const float* __restrict__ C, int k, float tau, int certify, float gBF, float gp2,
                   int* __restrict__ labels, uint4* __restrict__ queue, Globals* g, TcShape sh) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (s_addr(smem_raw) & 1023)) & 1023);
    unsigned char* xs = base;                                             // stages
    unsigned char* bs = xs + (size_t)sh.stages * kTcTileBytes;            // B operand
    float* ccb = reinterpret_cast<float*>(bs + (size_t)sh.Npad * 128);    // Npad
    constexpr int kEpi = 4 * NG, kProducer = kEpi, kMma = kEpi + 1, kThreads = tc_threads(NG);
    __shared__ __align__(8) unsigned long long full[kTcMaxStages], empty[kTcMaxStages], accf[NG], tfree[NG];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    __shared__ unsigned __int128 red128[kThreads / 32];
    __shared__ unsigned long long red64[kThreads / 32];
    __shared__ unsigned int redu[kThreads / 32];
    __shared__ CertC cert;

    if (g->nonfinite) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &abort_flag;
    const int S = sh.stages;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        for (int b = 0; b < NG; ++b) { tc::mbar_init(&accf[b], 1); tc::mbar_init(&tfree[b], 4); }
        tc::mbar_init_fence();
    }
    if (warp == kMma) tc::tmem_alloc(&tmem_slot, (unsigned)sh.tmem_cols);
    // centroids: BF16 B operand (swizzled), ||c_bf16||^2, and the
    // certificate constants from the FP32 centroids (upper bounds)
    for (int e = tid; e < sh.Npad * (kTcK / 8); e += kThreads) {
        const int j = e / (kTcK / 8), c = e % (kTcK / 8);
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int d = 8 * c + i;
            v[i] = __float2bfloat16_rn((j < k && d < n) ? C[(size_t)j * n + d] : 0.f);
        }
        const int pc = c ^ (j & 7);
        *reinterpret_cast<uint4*>(bs + (size_t)j * 128 + 16 * pc) = *reinterpret_cast<const uint4*>(v);
    }
    unsigned int mx = 0;
    for (int j = tid; j < sh.Npad; j += kThreads) {
        float acc = 0.f, up = 0.f;
        for (int d = 0; d < n && j < k; ++d) {
            const float c = C[(size_t)j * n + d];
            const float b = __bfloat162float(__float2bfloat16_rn(c));
            acc = __fmaf_rn(b, b, acc);
            up = __fmaf_ru(c, c, up);
        }
        ccb[j] = (j < k) ? acc : __int_as_float(0x7f800000);   // padded columns never win
        mx = max(mx, __float_as_uint(up));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) redu[warp] = mx;
    tc::fence_proxy_async();                                   // B visible to the tensor core
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        unsigned int mm = 0;
        for (int i = 0; i < kThreads / 32; ++i) mm = max(mm, redu[i]);
        cert.cmax2 = __uint_as_float(mm);
        cert.cmax = __fsqrt_ru(cert.cmax2);
    }
    __syncthreads();
    const unsigned tmem = tmem_slot;
    const long long ntiles = (m + kTcRows - 1) / kTcRows;
    const long long grid = gridDim.x;

    unsigned __int128 facc = 0;
    unsigned int inex = 0;
    long long issued = 0;             // producer: copies issued; MMA thread: tiles committed
    if (warp == kProducer) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            long long it = 0;
            int s = 0;
            unsigned ph = 0;                                // (it / S) & 1
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                if (it >= S && !tc::wait(&empty[s], ph ^ 1u, abort, g, sh.wait)) break;
                tc::expect_tx(&full[s], (unsigned)kTcTileBytes);
                tc::bulk_g2s(xs + (size_t)s * kTcTileBytes, Xb + tile * kTcRows * kTcK, (unsigned)kTcTileBytes,
                             &full[s]);
                if (++s == S) { s = 0; ph ^= 1u; }
            }
            issued = it;
        }
    } else if (warp == kMma) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            const unsigned idesc = tc::idesc_bf16(kTcRows, sh.Npad);
            const unsigned b0 = s_addr(bs);
            long long it = 0;
            int s = 0;
            unsigned ph = 0;                                // (it / S) & 1
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                const int b = (int)(it % NG);
                const long long u = it / NG;
                if (!tc::wait(&full[s], ph, abort, g, sh.wait)) break;
                if (u >= 1 && !tc::wait(&tfree[b], (unsigned)((u - 1) & 1), abort, g, sh.wait)) break;
                tc::fence_after();
                const unsigned a0 = s_addr(xs + (size_t)s * kTcTileBytes);
                const unsigned d = tmem + (unsigned)(b * sh.acc_stride);
#pragma unroll
                for (int kk = 0; kk < kTcK / 16; ++kk)
                    tc::mma_bf16(d, tc::desc_sw128(a0 + 32 * kk), tc::desc_sw128(b0 + 32 * kk), idesc, kk > 0);
                tc::commit(&accf[b]);
                tc::commit(&empty[s]);
                if (++s == S) { s = 0; ph ^= 1u; }
            }
            issued = it;
            // the last stage release arrives after every MMA of this CTA has
            // completed: wait for it, so that no arrival is pending at exit
            if (!*abort && issued > 0)
                tc::wait(&empty[(issued - 1) % S], (unsigned)(((issued - 1) / S) & 1), abort, g, sh.wait);
        }
    } else {
        // --------------------------------------------------- epilogue groups
        const long long m_pad = (m + kTcRows - 1) / kTcRows * kTcRows;
        const Grids gr = grids_from_maxbits(max(g->maxbits, __float_as_uint(xnorm[m_pad])));
        const CertC cc = cert;
        const int b = warp >> 2, q4 = warp & 3;
        const unsigned trow = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)(b * sh.acc_stride);
        for (long long it = b;; it += NG) {
            const long long tile = blockIdx.x + it * grid;
            if (tile >= ntiles) break;
            const long long row = tile * kTcRows + q4 * 32 + lane;
            const float xx = row < m ? __ldg(xnorm + row) : 0.f;
            int ok = 1;
            if (lane == 0) ok = tc::wait(&accf[b], (unsigned)((it / NG) & 1), abort, g, sh.wait);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc::fence_after();
            // 1. the two least g (four chains); chunks of 16 columns,
            //    double-buffered
            float t1[4], t2[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { t1[c] = __int_as_float(0x7f800000); t2[c] = t1[c]; }
            {
                unsigned va[16], vb[16];
                tc::ld16(trow, va);
                for (int c0 = 0; c0 < k; c0 += 32) {
                    tc::wait_ld16(va);
                    if (c0 + 16 < k) tc::ld16(trow + (unsigned)(c0 + 16), vb);
                    if (c0 + 16 <= k) tc::min2_chunk<false>(t1, t2, va, ccb, c0, 16);
                    else tc::min2_chunk<true>(t1, t2, va, ccb, c0, k - c0);
                    if (c0 + 16 < k) {
                        tc::wait_ld16(vb);
                        if (c0 + 32 < k) tc::ld16(trow + (unsigned)(c0 + 32), va);
                        if (c0 + 32 <= k) tc::min2_chunk<false>(t1, t2, vb, ccb, c0 + 16, 16);
                        else tc::min2_chunk<true>(t1, t2, vb, ccb, c0 + 16, k - c0 - 16);
                    }
                }
            }
            float g1 = t1[0], g2 = t2[0];
#pragma unroll
            for (int c = 1; c < 4; ++c) {   // merge two sorted pairs
                g2 = tc::min3f(g2, t2[c], fmaxf(g1, t1[c]));
                g1 = fminf(g1, t1[c]);
            }
            // 2. the rule; for a close call the certificate threshold (the
            //    bound on ||x||^2 is the BF16 norm x (1 + 2^-6))
            bool close = row < m && !(g2 - g1 >= tau * xx);
            float lim = g1;                 // the columns kept by pass 2: g <= lim
            if (row < m && (close || certify)) {
                const float xn2 = __fmul_ru(xx, 1.0f + 0x1p-6f);
                const float thr = cert_threshold(g1, xn2, __fsqrt_ru(xn2), cc, gBF, gp2);
                close = close || !(__fsub_rd(g2, g1) > thr);
                if (close) lim = __fadd_ru(g1, thr);
            }
            // 3. a second read of the accumulator: the label of a settled row
            //    (the first column with g = g1, i.e. the lowest index on
            //    ties), the candidates of a close call (up to kTcCand of
            //    them, two words of bytes, the newest in the low byte)
            int j1 = 0, cnt = 0;
            unsigned lo = 0, hi = 0;
            {
                unsigned va[16], vb[16];
                tc::ld16(trow, va);
                for (int c0 = 0; c0 < k; c0 += 32) {
                    tc::wait_ld16(va);
                    if (c0 + 16 < k) tc::ld16(trow + (unsigned)(c0 + 16), vb);
                    unsigned mk = (c0 + 16 <= k) ? tc::le_mask16<false>(va, ccb, c0, lim, 16)
                                                 : tc::le_mask16<true>(va, ccb, c0, lim, k - c0);
                    if (c0 + 16 < k) {
                        tc::wait_ld16(vb);
                        if (c0 + 32 < k) tc::ld16(trow + (unsigned)(c0 + 32), va);
                        mk |= ((c0 + 32 <= k) ? tc::le_mask16<false>(vb, ccb, c0 + 16, lim, 16)
                                              : tc::le_mask16<true>(vb, ccb, c0 + 16, lim, k - c0 - 16)) << 16;
                    }
                    if (cnt == 0 && mk) j1 = c0 + __ffs(mk) - 1;      // a settled row's label
                    if (!close) cnt += mk != 0u;
                    unsigned mc = close ? mk : 0u;                    // a close call's candidates
                    while (mc) {
                        const int j = c0 + __ffs(mc) - 1;
                        mc &= mc - 1u;
                        if (cnt < kTcCand) {
                            hi = (hi << 8) | (lo >> 24);
                            lo = (lo << 8) | (unsigned)j;
                        }
                        ++cnt;
                    }
                }
            }
            const unsigned cq = __ballot_sync(0xffffffffu, close);
            // 4. the accumulator is free for the MMA of tile it + NG
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::arrive(&tfree[b]);
            if (cq) {
                unsigned qbase = 0;
                if (lane == __ffs(cq) - 1) qbase = atomicAdd(&g->queue_len, (unsigned)__popc(cq));
                qbase = __shfl_sync(0xffffffffu, qbase, __ffs(cq) - 1);
                if (close) {
                    const unsigned all = (cnt < 1 || cnt > kTcCand) ? 0x80000000u : 0u;
                    queue[qbase + __popc(cq & ((1u << lane) - 1u))] =
                        make_uint4((unsigned)row | all, (unsigned)cnt, lo, hi);
                }
            }
            if (row < m && !close) {
                acc_obj(facc, fmaxf(0.f, xx + g1), gr.gf, inex);
                if (labels) labels[row] = j1;
            }
        }
    }

    // teardown.  Without an abort every copy and every MMA was consumed by a
    // wait.  After an abort (a bounded wait ran out), once every role has
    // stopped (the flag is final after the barrier), the producer waits for
    // its copies still in flight and the MMA thread for its last commit, so
    // that nothing writes this CTA's shared or tensor memory after release.
    tc::fence_before();
    __syncthreads();
    if (*abort) {
        if (warp == kProducer && lane == 0)
            for (long long i = (issued > S ? issued - S : 0); i < issued; ++i)
                for (unsigned p = 0; p < (1u << 22) && !tc::try_wait(&full[i % S], (unsigned)((i / S) & 1)); ++p) {}
        if (warp == kMma && lane == 0 && issued > 0)
            for (unsigned p = 0;
                 p < (1u << 22) && !tc::try_wait(&empty[(issued - 1) % S], (unsigned)(((issued - 1) / S) & 1));
                 ++p) {}
        __syncthreads();
    }
    if (warp == kMma) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, (unsigned)sh.tmem_cols);
    }
    // objective of the rows settled here: CTA reduction, then global words
    // (the re-score kernel adds its rows and rounds the total once)
    const unsigned __int128 F = warp_sum_u128(facc);
    const unsigned long long I = warp_sum((unsigned long long)inex);
    if (lane == 0) { red128[warp] = F; red64[warp] = I; }
    __syncthreads();
    if (tid == 0) {
        unsigned __int128 T = 0;
        unsigned long long in = 0;
        for (int i = 0; i < kThreads / 32; ++i) { T += red128[i]; in += red64[i]; }
        for (int i = 0; i < 4; ++i) {
            const unsigned long long chunk = (unsigned long long)((T >> (32 * i)) & 0xffffffffu);
            if (chunk) atomicAdd(&g->obj_words[i], chunk);
        }
        if (in) atomicAdd(&g->inexact, in);
        if (*abort) atomicOr(&g->err, kErrTimeout);
    }
}

// Exact re-score of the queued close calls: the exact-mode label (argmin of
// the FP32 direct form, lowest index on ties) and distance of each queued
// row.  A row with candidates takes the least direct form among them; a
// flagged row is resolved by the whole warp over all k (lanes over
// centroids, warp argmin).  Thread per row with the row in registers; adds
// the rows' distances to the objective words and, in its last CTA, rounds the
// objective of both kernels once.
constexpr int kRsStride = kTcK + 4;      // centroid rows: odd number of 16-byte units apart
__global__ void __launch_bounds__(256)
rescore_kernel(const float* __restrict__ Xf, const float* __restrict__ xnorm, long long m, int n,
               const float* __restrict__ C, int k, const uint4* __restrict__ queue, int* __restrict__ labels,
               Globals* g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* Cg = reinterpret_cast<float*>(smem_raw);                  // k x kRsStride
    __shared__ unsigned __int128 red128[8];
    __shared__ unsigned long long red64[8];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (g->nonfinite) return;
    for (int e = tid; e < k * kTcK; e += 256) {
        const int j = e / kTcK, d = e % kTcK;
        Cg[(size_t)j * kRsStride + d] = d < n ? C[(size_t)j * n + d] : 0.f;
    }
    __syncthreads();
    const long long m_pad = (m + kTcRows - 1) / kTcRows * kTcRows;
    const Grids gr = grids_from_maxbits(max(g->maxbits, __float_as_uint(xnorm[m_pad])));
    const long long q = g->queue_len;
    const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(Xf) & 15) == 0;
    // row `row` of Xf as m2x = -2 x, zero past n
    auto load_m2x = [&](long long row, float2 (&m2x)[kTcK / 2]) {
        const float* xr = Xf + row * (long long)n;
        if (vec) {                                                   // 16-byte loads of the row
#pragma unroll
            for (int q4 = 0; q4 < kTcK / 4; ++q4) {
                const float4 v = (4 * q4 < n) ? __ldg(reinterpret_cast<const float4*>(xr) + q4)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                m2x[2 * q4 + 0] = __fmul2_rn(make_float2(-2.f, -2.f), make_float2(v.x, v.y));
                m2x[2 * q4 + 1] = __fmul2_rn(make_float2(-2.f, -2.f), make_float2(v.z, v.w));
            }
        } else {
#pragma unroll
            for (int d = 0; d < kTcK / 2; ++d)
                m2x[d] = make_float2(2 * d < n ? -2.f * xr[2 * d] : 0.f, 2 * d + 1 < n ? -2.f * xr[2 * d + 1] : 0.f);
        }
    };
    unsigned __int128 facc = 0;
    unsigned int inex = 0;
    // warp-uniform trips of 32 queued rows
    const long long stride = (long long)gridDim.x * 256;
    long long w0 = ((long long)blockIdx.x * 8 + warp) * 32;
    uint4 en_next = (w0 + lane < q) ? queue[w0 + lane] : make_uint4(0u, 0u, 0u, 0u);
    for (; w0 < q; w0 += stride) {
        const long long i = w0 + lane;
        const bool valid = i < q;
        const uint4 en = en_next;
        // the next trip's entry, and its row into L2 while this one is scored
        en_next = (i + stride < q) ? queue[i + stride] : make_uint4(0u, 0u, 0u, 0u);
        if (i + stride < q) {
            const char* nr = reinterpret_cast<const char*>(Xf + (long long)(en_next.x & 0x7fffffffu) * n);
            for (int o = 0; o < n * 4; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(nr + o));
        }
        const long long row = (long long)(en.x & 0x7fffffffu);
        const bool all = valid && (en.x >> 31);
        const int cnt = (valid && !all) ? (int)en.y : 0;
        float2 m2x[kTcK / 2];                                        // -2 x, dimension pairs
        load_m2x(row, m2x);
        float dv = __int_as_float(0x7f800000);
        int lab = 0x7fffffff;
        for (int c = 0; c < cnt; ++c) {                               // the candidates, any order
            const int j = (int)(((c < 4 ? en.z : en.w) >> (8 * (c & 3))) & 0xffu);
            const float d = d32_m2x<kTcK>(m2x, Cg + (size_t)j * kRsStride);
            if (d < dv || (d == dv && j < lab)) { dv = d; lab = j; }
        }
        // flagged rows, one at a time: lanes take centroids lane, lane + 32,
        // ... of the row, then a warp argmin with the lowest index on ties
        unsigned pend = __ballot_sync(0xffffffffu, all);
        while (pend) {
            const int src = __ffs(pend) - 1;
            pend &= pend - 1u;
            float2 r2x[kTcK / 2];
            load_m2x(__shfl_sync(0xffffffffu, row, src), r2x);
            float bd = __int_as_float(0x7f800000);
            int bj = 0x7fffffff;
            for (int j = lane; j < k; j += 32) {
                const float dj = d32_m2x<kTcK>(r2x, Cg + (size_t)j * kRsStride);
                if (dj < bd || bj == 0x7fffffff) { bd = dj; bj = j; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                if (od < bd || (od == bd && oj < bj)) { bd = od; bj = oj; }
            }
            if (lane == src) { dv = bd; lab = bj; }
        }
        if (valid) {
            acc_obj(facc, dv, gr.gf, inex);
            if (labels) labels[row] = lab;
        }
    }
    unsigned __int128 F = warp_sum_u128(facc);
    const unsigned long long I = warp_sum((unsigned long long)inex);
    if (lane == 0) { red128[warp] = F; red64[warp] = I; }
    __syncthreads();
    if (tid == 0) {
        unsigned __int128 T = 0;
        unsigned long long in = 0;
        for (int i = 0; i < 8; ++i) { T += red128[i]; in += red64[i]; }
        for (int i = 0; i < 4; ++i) {
            const unsigned long long chunk = (unsigned long long)((T >> (32 * i)) & 0xffffffffu);
            if (chunk) atomicAdd(&g->obj_words[i], chunk);
        }
        if (in) atomicAdd(&g->inexact, in);
        __threadfence();
        last = (atomicAdd(&g->done_ctas, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && tid == 0) {
        __threadfence();
        unsigned __int128 T = 0;
        for (int i = 0; i < 4; ++i) {
            T += (unsigned __int128)atomicAdd(&g->obj_words[i], 0ull) << (32 * i);
            g->obj_words[i] = 0;
        }
        g->f_full = u128_to_double(T, gr.gf);
        g->rescored += (unsigned long long)q;
        g->done_ctas = 0;
    }
}

// ------------------------------------------------------------ launchers
// Shared memory of the pass for k centroids (0 when k is out of range).
size_t tc_smem_bytes(int k) {
    TcShape s;
    return tc_shape(k, s) ? tc_smem_bytes(s) : 0;
}

cudaError_t launch_pack_bf16(const float* X, long long m, int n, long long m_pad, void* Xb, float* norms,
                             cudaStream_t st) {
    const long long total = std::max<long long>(m_pad * (kTcK / 8) * (Xb ? 1 : 0), m_pad);
    const int grid = (int)std::min<long long>(8192, (total + 255) / 256);
    cudaError_t e = cudaMemsetAsync(norms + m_pad, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    pack_bf16_kernel<<<grid, 256, 0, st>>>(X, m, n, m_pad, (__nv_bfloat16*)Xb, norms);
    return cudaGetLastError();
}

// BF16 error factor of the precision form's certificate.  BF16 keeps 8
// significant bits (unit roundoff 2^-8), so a product of rounded x and c is
// within (2^-7 + 2^-16) |x c| of x c, and ||c_bf16||^2 (FP32 sum of 64
// squares) within (2^-7 + 2^-15) ||c||^2 of ||c||^2; the FP32 accumulation of
// the four K = 16 instructions adds at most 2^-16 of sum |x c| and the final
// fma 2^-24 of |g|.  Altogether |g - (||c||^2 - 2 x.c)| <= (2^-7 + 2^-13)
// (max ||c||^2 + 2 ||x|| max ||c||).
constexpr float kGammaBF16 = 0x1.04p-7f;     // 2^-7 + 2^-13

tc::WaitLimit tcx_wait_limit();

template <int NG>
cudaError_t launch_tc_t(const void* Xb, const float* xnorm, long long m, int n, const float* C, int k, float tau,
                        int certify, float gp2, int* labels, uint4* queue, Globals* g, int sms, const TcShape& sh,
                        cudaStream_t st) {
    constexpr int threads = tc_threads(NG);
    const size_t smem = tc_smem_bytes(sh);
    cudaFuncAttributes fa;
    cudaError_t e = func_attributes((const void*)tc_fullpass_kernel<NG>, &fa);
    if (e != cudaSuccess) return e;
    const int warps_alloc = (threads / 32 + 3) & ~3;            // warps are given registers in fours
    if ((long long)fa.numRegs * 32 * warps_alloc > 65536 || smem + fa.sharedSizeBytes > 227 * 1024)
        return cudaErrorNotSupported;
    e = allow_max_smem((const void*)tc_fullpass_kernel<NG>);
    if (e != cudaSuccess) return e;
    // one CTA per SM (its registers and tensor memory), persistent over tiles
    const long long tiles = (m + kTcRows - 1) / kTcRows;
    const long long grid = std::max<long long>(1, std::min<long long>((long long)sms, tiles));
    tc_fullpass_kernel<NG><<<(unsigned)grid, threads, smem, st>>>((const __nv_bfloat16*)Xb, xnorm, m, n, C, k, tau,
                                                                   certify, kGammaBF16, gp2, labels, queue, g, sh);
    return cudaGetLastError();
}

// The precision pass and the re-score of its queue.  `queue` holds m
// entries of 16 bytes.
cudaError_t launch_tc_fullpass(const void* Xb, const float* xnorm, const float* Xf, long long m, int n,
                               const float* C, int k, float tau, int certify, int* labels, void* queue, Globals* g,
                               float gp2, int sms, cudaStream_t st) {
    TcShape sh;
    if (!tc_shape(k, sh)) return cudaErrorNotSupported;
    sh.wait = tcx_wait_limit();
    uint4* qe = static_cast<uint4*>(queue);
    cudaError_t e = sh.groups == 4 ? launch_tc_t<4>(Xb, xnorm, m, n, C, k, tau, certify, gp2, labels, qe, g, sms, sh, st)
                                   : launch_tc_t<2>(Xb, xnorm, m, n, C, k, tau, certify, gp2, labels, qe, g, sms, sh, st);
    if (e != cudaSuccess) return e;
    const size_t rs = (size_t)k * kRsStride * 4;
    e = allow_max_smem((const void*)rescore_kernel);
    if (e != cudaSuccess) return e;
    rescore_kernel<<<sms * 2, 256, rs, st>>>(Xf, xnorm, m, n, C, k, qe, labels, g);
    return cudaGetLastError();
}

}  // namespace bm
