// Device helpers shared by the Big-means kernels (sm_103a).
//
// * Philox4x64-10 (Salmon et al., SC'11) and Lemire's bounded draw: the
//   random stream contract of include/bigmeans.h.
// * Exact sums in integer fixed point.  Coordinates are converted to signed
//   128-bit integers in units of 2^gx and summed in three int64 words
//   (value = w0 + w1*2^32 + w2*2^64); squared distances into an unsigned
//   128-bit accumulator in units of 2^gf.  Integer addition is associative, so the result does not
//   depend on thread, block or cluster order; it is rounded to double once.
// * The FP32 direct-form squared distance that defines labels (Eq. 1).
#pragma once
#include <cstdint>
#include <mutex>
#include <map>
#include <set>
#include <tuple>
#include <cuda_runtime.h>
#include <cooperative_groups.h>

namespace bm {
namespace cg = cooperative_groups;

constexpr int kThreads = 256;          // threads per CTA of the worker, sampling and prepass kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxWarps = 16;            // largest CTA of any kernel here: 512 threads
constexpr int kMaxCluster = 16;        // CTAs per worker cluster (non-portable above 8)

// ------------------------------------------------------------------ globals
// Per-call device state written by the kernels and read back by the host.
struct Globals {
    unsigned int maxbits;              // max over |x| (and |c|) float bits
    unsigned int nonfinite;            // count of NaN / Inf inputs
    unsigned int err;                  // error flags (kErr*)
    unsigned int done_ctas;            // last-CTA-done counter (full pass)
    unsigned long long lloyd_iters, assign_rows, passes, rescored, inexact;
    unsigned long long accepts, L_sum, eval_rows, reseeded;
    // device phase trace (SM cycles on rank 0 of each worker cluster):
    // 0 K-means++, 1 Lloyd assignment, 2 Lloyd exchange (barriers, DSMEM
    // reduction, centroid update), 3 f_hat recompute, 4 sum of worker kernel
    // times, 5 longest worker kernel, 6 Lloyd assignments, 7 worker kernels,
    // 8 assignment main loop, 9 assignment block reductions, 10 first cluster
    // barrier, 11 owner update + objective, 12 second cluster barrier,
    // 13 centroid copy + prep, 14 first assignment of a Lloyd run (whole),
    // 15 its labelling loop (the rest is the bucketed sums)
    unsigned long long trace[16];
    unsigned long long obj_words[4];   // full-pass objective, 32-bit chunks
    double f_full;                     // last full-pass objective
    double f_incumbent;                // least full objective seen
    int best_worker;                   // worker whose centroids were assessed
    int s_opt;
    int rounds_done;
    unsigned int queue_len;            // rows queued for exact re-scoring (tensor-core pass)
};
constexpr unsigned kErrSample = 1u;    // sampler ran out of draws
constexpr unsigned kErrDigits = 2u;    // fixed-point range exceeded
constexpr unsigned kErrNonFinite = 4u; // non-finite input seen
constexpr unsigned kErrTimeout = 8u;   // a bounded wait gave up
constexpr unsigned kErrArgs = 16u;     // inconsistent arguments on device

// Exponent grids derived from the largest magnitude (see file comment).
struct Grids { int Ex, gx, gf; };
__host__ __device__ inline Grids grids_from_maxbits(unsigned int maxbits) {
    unsigned ef = maxbits >> 23;
    int Ex = (maxbits == 0) ? -127 : (ef == 0 ? -127 : (int)ef - 127);
    Grids g;
    g.Ex = Ex;
    g.gx = Ex - 95;                     // coordinates: exponent of max|x| - 95
    g.gf = 2 * Ex - 86;                 // squared distances
    return g;
}

// ------------------------------------------------------------ Philox4x64-10
struct P4 { uint64_t v[4]; };

__device__ __forceinline__ P4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                            uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    P4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Stream purposes (high byte of key[1]); see include/bigmeans.h.
constexpr int kPurposeSize = 1, kPurposeEval = 2, kPurposePass = 3, kPurposeKpp = 4,
              kPurposeFinal = 5;

__host__ __device__ inline uint64_t stream_k1(int purpose, int worker, int round, int pass) {
    return ((uint64_t)(purpose & 0xff) << 56) | ((uint64_t)(worker & 0xffff) << 40) |
           ((uint64_t)(round & 0xffffff) << 16) | (uint64_t)(pass & 0xffff);
}

// Lemire: accept word w when low64(w * bound) >= (2^64 - bound) mod bound.
// Host copy of the library's sample-size draw (same Philox4x64-10 and Lemire
// rule as the device code), used to size each worker's cluster.
// Raise a kernel's dynamic shared-memory limit to the most the device allows,
// once per kernel.  The limit is a process-wide attribute of the kernel, so
// setting it per launch to that launch's size would race between host
// threads launching the same kernel with different sizes (one thread's
// smaller value failing the other's launch); every launch still passes its
// own size.
inline cudaError_t allow_max_smem(const void* func) {
    static std::mutex mu;
    static std::set<const void*> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(func)) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert(func);
    return e;
}

// Resident CTAs per SM of `func` at (threads, dynamic shared memory),
// computed once per triple (the launchers call this on every launch).
inline cudaError_t blocks_per_sm(const void* func, int threads, size_t smem, int* out) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> memo;
    const auto key = std::make_tuple(func, threads, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto it = memo.find(key);
        if (it != memo.end()) { *out = it->second; return cudaSuccess; }
    }
    int v = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, func, threads, smem);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    memo[key] = v;
    *out = v;
    return cudaSuccess;
}
// Attributes of `func`, read once.
inline cudaError_t func_attributes(const void* func, cudaFuncAttributes* out) {
    static std::mutex mu;
    static std::map<const void*, cudaFuncAttributes> memo;
    std::lock_guard<std::mutex> lk(mu);
    const auto it = memo.find(func);
    if (it != memo.end()) { *out = it->second; return cudaSuccess; }
    const cudaError_t e = cudaFuncGetAttributes(out, func);
    if (e == cudaSuccess) memo[func] = *out;
    return e;
}

inline uint64_t host_draw_below(uint64_t seed, uint64_t k1, uint64_t c0, uint64_t c1, uint64_t bound) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = c0, x1 = c1, x2 = 0, x3 = 0, k0 = seed, kk1 = k1;
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; kk1 += W1; }
        const unsigned __int128 p0 = (unsigned __int128)M0 * x0, p1 = (unsigned __int128)M1 * x2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        const uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ kk1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    const uint64_t w[4] = {x0, x1, x2, x3};
    const uint64_t thr = (0ull - bound) % bound;
    for (int i = 0; i < 4; ++i) {
        const unsigned __int128 p = (unsigned __int128)w[i] * bound;
        if ((uint64_t)p >= thr) return (uint64_t)(p >> 64);
    }
    return (uint64_t)(((unsigned __int128)w[3] * bound) >> 64);
}

__device__ __forceinline__ uint64_t lemire_thr(uint64_t bound) { return (0ull - bound) % bound; }

__device__ __forceinline__ uint64_t uniform_below(const P4& b, uint64_t bound, uint64_t thr) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (b.v[i] * bound >= thr) return __umul64hi(b.v[i], bound);
    return __umul64hi(b.v[3], bound);
}

__device__ __forceinline__ uint64_t draw_below(uint64_t seed, uint64_t k1, uint64_t c0,
                                               uint64_t c1, uint64_t bound) {
    P4 b = philox4x64_10(c0, c1, 0, 0, seed, k1);
    return uniform_below(b, bound, lemire_thr(bound));
}

// ------------------------------------------------------- float decomposition
// |v| = mant * 2^e2 with mant < 2^24.
__device__ __forceinline__ void f32_parts(uint32_t bits, uint32_t& mant, int& e2) {
    const uint32_t ef = (bits >> 23) & 0xff, fr = bits & 0x7fffff;
    mant = ef ? (fr | 0x800000u) : fr;
    e2 = ef ? (int)ef - 150 : -149;
}

// Add a non-negative float to a 128-bit fixed-point accumulator (unit 2^gf).
__device__ __forceinline__ void acc_obj(unsigned __int128& acc, float d, int gf,
                                        unsigned int& inexact) {
    const uint32_t b = __float_as_uint(d) & 0x7fffffffu;
    if (b == 0) return;
    uint32_t mant; int e2;
    f32_parts(b, mant, e2);
    const int sh = e2 - gf;
    if (sh >= 0) {
        acc += ((unsigned __int128)mant) << sh;
    } else {
        const int r = -sh;
        if (r >= 24) { inexact++; return; }
        if (mant & ((1u << r) - 1u)) inexact++;
        acc += (unsigned __int128)(mant >> r);
    }
}

// A coordinate on the grid of the exact sums (unit 2^gx) as a signed 128-bit
// integer.  Bits below the grid are truncated (counted in `inexact`); returns
// false if |x| / 2^gx needs more than 96 bits (outside the grid's range; the
// grid is set from the largest |x|, so data values never are).  Sums of such
// integers are exact and independent of their order.
constexpr long long kMaxRowsPerCta = 32767;
__device__ __forceinline__ bool fixed_of(float x, int gx, unsigned int& inexact, __int128& v) {
    v = 0;
    const uint32_t bits = __float_as_uint(x);
    const uint32_t mag = bits & 0x7fffffffu;
    if (mag == 0) return true;
    uint32_t mant; int e2;
    f32_parts(mag, mant, e2);
    int sh = e2 - gx;
    if (sh < 0) {
        const int r = -sh;
        if (r >= 24) { inexact++; return true; }
        if (mant & ((1u << r) - 1u)) inexact++;
        mant >>= r;
        sh = 0;
        if (!mant) return true;
    }
    if (sh + (32 - __clz((int)mant)) > 96) return false;
    const unsigned __int128 u = (unsigned __int128)mant << sh;
    v = (bits >> 31) ? -(__int128)u : (__int128)u;
    return true;
}

// Correctly rounded double of a (signed) 128-bit integer times 2^g.
__device__ __forceinline__ double i128_to_double(__int128 v, int g) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    unsigned __int128 a = neg ? (unsigned __int128)(-(v + 1)) + 1u : (unsigned __int128)v;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    double r;
    int e = g;
    if (hi == 0) {
        r = __ull2double_rn(lo);
    } else {
        const int sh = 64 - __clzll((long long)hi);          // 1..64
        uint64_t top = (uint64_t)(a >> sh);
        const uint64_t rest = (sh == 64) ? lo : (lo & ((1ull << sh) - 1ull));
        top |= (rest != 0) ? 1ull : 0ull;                      // sticky bit
        r = __ull2double_rn(top);
        e += sh;
    }
    r = ldexp(r, e);
    return neg ? -r : r;
}

__device__ __forceinline__ double u128_to_double(unsigned __int128 a, int g) {
    if (a == 0) return 0.0;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    double r;
    int e = g;
    if (hi == 0) {
        r = __ull2double_rn(lo);
    } else {
        const int sh = 64 - __clzll((long long)hi);
        uint64_t top = (uint64_t)(a >> sh);
        const uint64_t rest = (sh == 64) ? lo : (lo & ((1ull << sh) - 1ull));
        top |= (rest != 0) ? 1ull : 0ull;
        r = __ull2double_rn(top);
        e += sh;
    }
    return ldexp(r, e);
}

// ------------------------------------------------------------ distances
// FP32 direct form: t = x_d - c_d; acc = acc + t*t, ascending d, each op
// rounded to nearest, never fused (the __f*_rn intrinsics are not contracted).
// Padded dimensions hold x = c = 0 and add exact zeros.
template <int NP>
__device__ __forceinline__ float d32(const float (&x)[NP], const float* __restrict__ c) {
    float acc = 0.f;
#pragma unroll
    for (int d4 = 0; d4 < NP / 4; ++d4) {
        const float4 cv = reinterpret_cast<const float4*>(c)[d4];
        float t;
        t = __fsub_rn(x[4 * d4 + 0], cv.x); acc = __fadd_rn(acc, __fmul_rn(t, t));
        t = __fsub_rn(x[4 * d4 + 1], cv.y); acc = __fadd_rn(acc, __fmul_rn(t, t));
        t = __fsub_rn(x[4 * d4 + 2], cv.z); acc = __fadd_rn(acc, __fmul_rn(t, t));
        t = __fsub_rn(x[4 * d4 + 3], cv.w); acc = __fadd_rn(acc, __fmul_rn(t, t));
    }
    return acc;
}

// The same d32(x, c) from the row held as m2x = -2 x (dimension pairs):
// fma(1/2, -2 x_d, c_d) = fl(c_d - x_d) = -fl(x_d - c_d) (one rounding of an
// exact value), so its square is the direct form's t*t; the squares are
// added in ascending d as above.
template <int NP>
__device__ __forceinline__ float d32_m2x(const float2 (&m2x)[NP / 2], const float* __restrict__ c) {
    const float2 half = make_float2(0.5f, 0.5f);
    float acc = 0.f;
#pragma unroll
    for (int d4 = 0; d4 < NP / 4; ++d4) {
        const float4 cv = reinterpret_cast<const float4*>(c)[d4];
        float2 t0 = __ffma2_rn(half, m2x[2 * d4 + 0], make_float2(cv.x, cv.y));
        float2 t1 = __ffma2_rn(half, m2x[2 * d4 + 1], make_float2(cv.z, cv.w));
        t0 = __fmul2_rn(t0, t0);
        t1 = __fmul2_rn(t1, t1);
        acc = __fadd_rn(acc, t0.x);
        acc = __fadd_rn(acc, t0.y);
        acc = __fadd_rn(acc, t1.x);
        acc = __fadd_rn(acc, t1.y);
    }
    return acc;
}
// An upper bound of ||x||^2 from m2x = -2 x: every operation rounds upward
// (so any order bounds the sum from above); the factor 1/4 is applied last.
template <int NP>
__device__ __forceinline__ float xnorm2_up_m2x(const float2 (&m2x)[NP / 2]) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < NP / 2; ++d) s = __ffma2_ru(m2x[d], m2x[d], s);
    return __fmul_ru(0.25f, __fadd_ru(s.x, s.y));
}

// Certificate constants of one centroid set (upper bounds, rounded upward):
//   cmax2 >= max_j ||c_j||^2, cmax >= sqrt(cmax2).
struct CertC { float cmax2, cmax; };

// Per-row certificate for the expanded-form argmin.  g1 <= g2 are the two
// least values of g_j = fl(||c_j||^2 + sum(-2 x_d) c_j,d) over centroids;
// xn2 >= ||x||^2, xn >= ||x||.  Each g_j is within B = gB (cmax2 + 2 ||x||
// cmax) of the exact ||c_j||^2 - 2 x.c_j (an NP + 1 term sum of rounded
// products), so the exact squared distance to the centroid of g1 is at most
// d1 = g1 + B + ||x||^2; the FP32 direct form of a distance D lies within
// gamma_{NP+2} D of D.  Hence a centroid whose g exceeds g1 by more than
// 2 B + gp2 d1 has a larger FP32 direct-form distance.
// gB >= gamma_{2NP+2}, gp2 >= 2 (1 + 2^-14) gamma_{NP+2}.  Returns true when
// the argmin of the FP32 direct-form distances is certainly the index of g1.
// Threshold of the certificate: any centroid j with fl_rd(g_j - g1) > thr has
// a larger FP32 direct-form distance than the centroid of g1.
__device__ __forceinline__ float cert_threshold(float g1, float xn2, float xn, const CertC& cc, float gB,
                                                float gp2) {
    const float B = __fmul_ru(gB, __fadd_ru(cc.cmax2, __fmul_ru(2.f, __fmul_ru(xn, cc.cmax))));
    const float d1 = fmaxf(0.f, __fadd_ru(__fadd_ru(g1, B), xn2));
    return __fadd_ru(__fmul_ru(2.f, B), __fmul_ru(gp2, d1));
}
__device__ __forceinline__ bool certified(float g1, float g2, float xn2, float xn,
                                          const CertC& cc, float gB, float gp2) {
    const float thr = cert_threshold(g1, xn2, xn, cc, gB, gp2);
    const float gap = __fsub_rd(g2, g1);
    return gap > thr;                     // false for NaN; +inf gap (k = 1) passes
}

// ------------------------------------------------------------ block reduce
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned __int128 warp_sum_u128(unsigned __int128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)v, o);
        const uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(v >> 64), o);
        v += ((unsigned __int128)hi << 64) | lo;
    }
    return v;
}

// Block reductions over all warps of the CTA (blockDim.x / 32 of them);
// `red` holds at least that many entries (one more for the scan).
// Sum over the CTA; result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__device__ __forceinline__ unsigned __int128 block_sum_u128(unsigned __int128 v, unsigned __int128* red) {
    v = warp_sum_u128(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    unsigned __int128 s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__device__ __forceinline__ unsigned int block_max_u32(unsigned int v, unsigned int* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    unsigned int s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = max(s, red[i]);
    return s;
}

// Exclusive scan over the CTA of one int64 per thread; returns the thread's
// exclusive prefix and writes the CTA total to *total (all threads).
__device__ __forceinline__ long long block_exscan(long long v, long long* red, long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) red[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        const int nw = (int)(blockDim.x >> 5);
        for (int i = 0; i < nw; ++i) { const long long t = red[i]; red[i] = run; run += t; }
        red[nw] = run;
    }
    __syncthreads();
    const long long excl = red[wid] + x - v;
    *total = red[blockDim.x >> 5];
    __syncthreads();
    return excl;
}

}  // namespace bm
