// Exact full-data pass (Alg. 1 last step, Eq. 1) with the distance
// contraction on the fifth-generation tensor cores.
//
// Results are those of the plain definition used everywhere in exact mode:
// label = argmin_j d32(x, c_j) with the lowest index on ties, where d32 is
// the FP32 direct form, and f = the exact sum of d32(x, c_label) rounded once.
// The tensor cores only propose the winner:
//
//   * X (FP32, row-major, n % 4 == 0) is read by 2-D TMA copies into 128-row
//     tiles in the 128-byte-swizzle K-major layout (32 floats per row and
//     column block; columns past n are zero-filled by the copy);
//   * split TF32: every x is split into hi = trunc_tf32(x) (exact in TF32)
//     and the residual r = x - hi (exact in FP32), written to two tiles of
//     the epilogue group that takes the tile (which frees the TMA stage at
//     once), every c likewise; one tile of 128
//     rows takes the MMAs r(x).hi(c) and hi(x).r(c) first, then
//     hi(x).hi(c), all accumulated in FP32 in tensor memory
//     (tcgen05.mma kind::tf32, M = 128, N = k rounded up to 16, K = 8 per
//     instruction).  x = hi + r exactly, so the epilogue rebuilds the FP32
//     row from the two tiles;
//   * the epilogue forms g_j = fl(||c_j||^2 - 2 acc_j), keeps the two least,
//     and accepts j1 when the certificate of the expanded form holds with
//     the split-TF32 error in its bound; the distance of the row is then
//     d32(x, c_j1).  Rows whose certificate fails are re-scored by the warp
//     over all centroids in d32 (lowest index on ties).
//
// Error of acc_j against x.c_j (exact reals): the tensor core reads the
// residuals with at most 10 mantissa bits (|r~ - r| <= 2^-10 |r|, whether it
// truncates or rounds), and |r| <= 2^-10 |x|, so the representation error is
// at most |r~(x) - r(x)| |c| + |x| |r~(c) - r(c)| + |r(x)| |r(c)|
// <= 3 * 2^-20 |x| |c| per term; products of TF32 values are exact in FP32.  The accumulation is taken to add at most (K + 1) 2^-23 of the
// magnitude accumulated so far per MMA instruction (products aligned and
// truncated once against the largest term, then added to the accumulator):
// at most ksteps * 9 * 2^-23 sum |x c| over the hi.hi instructions, and far
// less over the small correction terms issued first.  The host passes the
// certificate factor gB = 2 (ksteps * 9 * 2^-23) + 8 * 2^-20, which bounds
// |g_j - (||c_j||^2 - 2 x.c_j)| by gB (cmax^2 + 2 ||x|| cmax).  A gap below
// 2^-60 is never accepted (subnormal data).
//
// CTA roles: the warp after the epilogue warps issues the TMA copies, the
// next one the MMAs; the epilogue warps form G = 2 or 3 warpgroups,
// warpgroup b taking the tiles it == b (mod G) with tensor-memory
// accumulator b and its own hi(x) / r(x) tiles, so the MMA of one tile
// overlaps the epilogues of the others.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "bm_device.cuh"
#include "bm_tcgen05.cuh"

namespace bm {

constexpr int kTxRows = 128;                  // rows per tile (MMA M)
constexpr int kTxAtomBytes = kTxRows * 128;   // one 32-float column block of a tile
constexpr int kTxMaxStages = 6;
__host__ __device__ constexpr int tx_threads(int groups) { return 32 * (4 * groups + 2); }
constexpr int kTxPairs = 64;                  // candidate pairs per warp and tile

struct TxShape {
    int atoms;       // 32-float column blocks per row (1 or 2)
    int ksteps;      // K = 8 steps per operand pair
    int Npad;        // MMA N: k rounded up to 16
    int acc_stride;  // tensor-memory columns per accumulator
    int tmem_cols;   // columns allocated
    int stages;      // X tiles in flight
    int groups;      // epilogue warpgroups (= accumulators = r(x) buffers)
    int inplace;     // 1: hi(x) written over the stage, which is held until the
                     //    group's epilogue ends; 0: hi(x) in a group buffer
    tc::WaitLimit wait;  // limit of every bounded wait
};

// Shared memory (1024-byte aligned pieces):
//   [X stages: stages x atoms x 16 KB][hi(x) (unless in place), r(x): groups
//   x atoms x 16 KB each][hi(c), r(c): 2 x atoms x Npad x 128 B][CC: Npad floats]
__host__ __device__ inline size_t tx_smem_bytes(const TxShape& s) {
    return 1024 + (size_t)(s.stages + (2 - s.inplace) * s.groups) * s.atoms * kTxAtomBytes +
           (size_t)2 * s.atoms * s.Npad * 128 + (size_t)s.Npad * 4;
}

__device__ __forceinline__ float trunc_tf32(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }

// Byte offset of the 16-byte chunk holding elements 4 q .. 4 q + 3 of row r in
// a tile of 32-float column blocks (128-byte swizzle).
__device__ __forceinline__ unsigned tile_off(int r, int q) {
    return (unsigned)((q >> 3) * kTxAtomBytes + r * 128 + (((q & 7) ^ (r & 7)) << 4));
}

// d32 of row rr of a tile against centroid j, both rebuilt as hi + r from
// their two swizzled tiles (exact: the parts do not overlap).  The X tiles
// have 32-float column blocks of 16 KB, the centroid tiles of Npad x 128 B.
template <int NP>
__device__ __forceinline__ float d32_split(const unsigned char* xh, const unsigned char* xr, int rr,
                                           const unsigned char* ch, const unsigned char* cr, int j,
                                           unsigned cstride) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
        const unsigned xo = tile_off(rr, q);
        const unsigned co = (unsigned)(q >> 3) * cstride + (unsigned)j * 128 + (unsigned)(((q & 7) ^ (j & 7)) << 4);
        const float4 h = *reinterpret_cast<const float4*>(xh + xo);
        const float4 l = *reinterpret_cast<const float4*>(xr + xo);
        const float4 a = *reinterpret_cast<const float4*>(ch + co);
        const float4 b = *reinterpret_cast<const float4*>(cr + co);
        float t;
        t = __fsub_rn(__fadd_rn(h.x, l.x), __fadd_rn(a.x, b.x)); acc = __fadd_rn(acc, __fmul_rn(t, t));
        t = __fsub_rn(__fadd_rn(h.y, l.y), __fadd_rn(a.y, b.y)); acc = __fadd_rn(acc, __fmul_rn(t, t));
        t = __fsub_rn(__fadd_rn(h.z, l.z), __fadd_rn(a.z, b.z)); acc = __fadd_rn(acc, __fmul_rn(t, t));
        t = __fsub_rn(__fadd_rn(h.w, l.w), __fadd_rn(a.w, b.w)); acc = __fadd_rn(acc, __fmul_rn(t, t));
    }
    return acc;
}

template <int NP, int NG>
__global__ void __launch_bounds__(tx_threads(NG), 1)
tcx_fullpass_kernel(const __grid_constant__ CUtensorMap tmap, long long m, const float* __restrict__ Cw, int k,
                    const double* sel_f, int W, int* __restrict__ labels, Globals* g, float gB, float gp2,
                    int incumbent, TxShape sh) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (tc::s_addr(smem_raw) & 1023)) & 1023);
    const size_t tile_bytes = (size_t)sh.atoms * kTxAtomBytes;
    unsigned char* xs = base;                                      // X stages
    unsigned char* xh = xs + (size_t)sh.stages * tile_bytes;       // hi(x), one per group
    unsigned char* xl = xh + (sh.inplace ? 0 : NG) * tile_bytes;   // r(x), one per group
    unsigned char* bh = xl + NG * tile_bytes;                      // hi(c)
    unsigned char* bl = bh + (size_t)sh.atoms * sh.Npad * 128;     // r(c)
    float* CC = reinterpret_cast<float*>(bl + (size_t)sh.atoms * sh.Npad * 128);
    constexpr int kEpi = 4 * NG, kProducer = kEpi, kMma = kEpi + 1, kThreads = tx_threads(NG);
    __shared__ __align__(8) unsigned long long full[kTxMaxStages], empty[kTxMaxStages], conv[NG], accf[NG];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    __shared__ unsigned __int128 red128[kThreads / 32];
    __shared__ unsigned long long red64[kThreads / 32];
    __shared__ unsigned int redu[kThreads / 32];
    __shared__ CertC cert;
    __shared__ int wsel;
    __shared__ bool last;
    __shared__ unsigned pairs[kEpi][kTxPairs];                      // candidate (lane, j) per warp
    __shared__ unsigned long long pkeys[kEpi][32];                  // (d32 bits, j) minimum per row

    if (g->nonfinite) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &abort_flag;
    if (tid == 0) {
        int best = 0;
        if (sel_f)
            for (int w = 1; w < W; ++w)
                if (sel_f[w] < sel_f[best]) best = w;
        wsel = best;
        abort_flag = 0;
        for (int s = 0; s < sh.stages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 4); }
        for (int b = 0; b < NG; ++b) { tc::mbar_init(&conv[b], 4); tc::mbar_init(&accf[b], 1); }
        tc::mbar_init_fence();
    }
    if (warp == kMma) tc::tmem_alloc(&tmem_slot, (unsigned)sh.tmem_cols);
    __syncthreads();
    const float* C = Cw + (long long)wsel * k * NP;

    // B operands hi(c), r(c) (swizzled like the X tiles); CC and the
    // certificate constants from the FP32 centroids.
    for (int e = tid; e < sh.atoms * sh.Npad * 8; e += kThreads) {
        const int a = e / (sh.Npad * 8), rem = e % (sh.Npad * 8), j = rem >> 3, c = rem & 7;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
        const int d0 = a * 32 + c * 4;
        if (j < k && d0 < NP) {
            const float4 cv = *reinterpret_cast<const float4*>(C + (size_t)j * NP + d0);
            h = make_float4(trunc_tf32(cv.x), trunc_tf32(cv.y), trunc_tf32(cv.z), trunc_tf32(cv.w));
            l = make_float4(cv.x - h.x, cv.y - h.y, cv.z - h.z, cv.w - h.w);     // exact
        }
        const size_t off = (size_t)a * sh.Npad * 128 + (size_t)j * 128 + ((c ^ (j & 7)) << 4);
        *reinterpret_cast<float4*>(bh + off) = h;
        *reinterpret_cast<float4*>(bl + off) = l;
    }
    unsigned int mx = 0;
    for (int j = tid; j < sh.Npad; j += kThreads) {
        float acc = 0.f, up = 0.f;
        if (j < k) {
#pragma unroll
            for (int d = 0; d < NP; ++d) {
                const float c = C[(size_t)j * NP + d];
                acc = __fmaf_rn(c, c, acc);
                up = __fmaf_ru(c, c, up);
            }
        }
        CC[j] = (j < k) ? acc : __int_as_float(0x7f800000);   // padded columns never win
        mx = max(mx, __float_as_uint(up));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) redu[warp] = mx;
    tc::fence_proxy_async();                 // B operands visible to the tensor core
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
    const long long ntiles = (m + kTxRows - 1) / kTxRows;
    const long long grid = gridDim.x;
    const int S = sh.stages;

    unsigned __int128 facc = 0;
    unsigned int inex = 0, resc = 0;
    long long issued = 0;             // producer: copies issued; MMA warp: tiles committed
    if (warp == kProducer) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            long long it = 0;
            int s = 0;
            unsigned ph = 0;                                // (it / S) & 1, kept incrementally
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                if (it >= S && !tc::wait(&empty[s], ph ^ 1u, abort, g, sh.wait)) break;
                tc::expect_tx(&full[s], (unsigned)tile_bytes);
                for (int a = 0; a < sh.atoms; ++a)
                    tc::tma_load_2d(xs + (size_t)s * tile_bytes + (size_t)a * kTxAtomBytes, &tmap, 32 * a,
                                    (int)(tile * kTxRows), &full[s]);
                if (++s == S) { s = 0; ph ^= 1u; }
            }
            issued = it;
        }
    } else if (warp == kMma) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            const unsigned idesc = tc::idesc_tf32(kTxRows, sh.Npad);
            const unsigned bstride = (unsigned)(sh.Npad * 128);
            long long it = 0;
            int s = 0;                                      // it % S, kept incrementally
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                const int b = (int)(it % NG);
                if (!tc::wait(&conv[b], (unsigned)((it / NG) & 1), abort, g, sh.wait)) break;
                tc::fence_after();
                const unsigned ax = tc::s_addr(sh.inplace ? xs + (size_t)s * tile_bytes
                                                          : xh + (size_t)b * tile_bytes);
                if (++s == S) s = 0;
                const unsigned al = tc::s_addr(xl + (size_t)b * tile_bytes);
                const unsigned ah = tc::s_addr(bh), alo = tc::s_addr(bl);
                const unsigned d = tmem + (unsigned)(b * sh.acc_stride);
                for (int kk = 0; kk < sh.ksteps; ++kk) {         // correction terms first
                    const unsigned off = (unsigned)((kk & 3) * 32);
                    const unsigned ao = (unsigned)(kk >> 2) * kTxAtomBytes + off;
                    const unsigned bo = (unsigned)(kk >> 2) * bstride + off;
                    tc::mma_tf32(d, tc::desc_sw128(al + ao), tc::desc_sw128(ah + bo), idesc, kk > 0);
                    tc::mma_tf32(d, tc::desc_sw128(ax + ao), tc::desc_sw128(alo + bo), idesc, 1);
                }
                for (int kk = 0; kk < sh.ksteps; ++kk) {
                    const unsigned off = (unsigned)((kk & 3) * 32);
                    const unsigned ao = (unsigned)(kk >> 2) * kTxAtomBytes + off;
                    const unsigned bo = (unsigned)(kk >> 2) * bstride + off;
                    tc::mma_tf32(d, tc::desc_sw128(ax + ao), tc::desc_sw128(ah + bo), idesc, 1);
                }
                tc::commit(&accf[b]);
            }
            issued = it;
        }
    } else {
        // --------------------------------------------------- epilogue groups
        const Grids gr = grids_from_maxbits(g->maxbits);
        const CertC cc = cert;
        const int b = warp >> 2, q4 = warp & 3;
        const int r = q4 * 32 + lane;                        // row within the tile = TMEM lane
        unsigned char* xlb = xl + (size_t)b * tile_bytes;
        const unsigned cstride = (unsigned)(sh.Npad * 128);
        int s = b;                                          // it % S and (it / S) & 1, kept
        unsigned ph = 0;                                    // incrementally (S is a multiple of NG)
        for (long long it = b;; it += NG) {
            const long long tile = blockIdx.x + it * grid;
            if (tile >= ntiles) break;
            unsigned char* st = xs + (size_t)s * tile_bytes;
            unsigned char* xhb = sh.inplace ? st : xh + (size_t)b * tile_bytes;
            // 1. the row: hi(x) and r(x) into this group's buffers; the stage
            //    is free again as soon as every warp of the group has read it
            int ok = 1;
            if (lane == 0) ok = tc::wait(&full[s], ph, abort, g, sh.wait);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            float xn2 = 0.f;
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                const float4 v = *reinterpret_cast<const float4*>(st + tile_off(r, q));
                xn2 = __fmaf_ru(v.x, v.x, xn2);
                xn2 = __fmaf_ru(v.y, v.y, xn2);
                xn2 = __fmaf_ru(v.z, v.z, xn2);
                xn2 = __fmaf_ru(v.w, v.w, xn2);
                const float4 h = make_float4(trunc_tf32(v.x), trunc_tf32(v.y), trunc_tf32(v.z), trunc_tf32(v.w));
                *reinterpret_cast<float4*>(xhb + tile_off(r, q)) = h;
                *reinterpret_cast<float4*>(xlb + tile_off(r, q)) =
                    make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                if (!sh.inplace) tc::arrive(&empty[s]);
                tc::arrive(&conv[b]);
            }
            const float xn = __fsqrt_ru(xn2);
            // 2. the accumulator of this tile
            if (lane == 0) ok = tc::wait(&accf[b], (unsigned)((it / NG) & 1), abort, g, sh.wait);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc::fence_after();
            // four interleaved top-2 chains over the accumulator columns
            float t1[4], t2[4];
            int tj[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { t1[c] = __int_as_float(0x7f800000); t2[c] = t1[c]; tj[c] = 0; }
            const unsigned trow = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)(b * sh.acc_stride);
            for (int c0 = 0; c0 < sh.Npad; c0 += 16) {
                unsigned va[16];
                tc::ld16(trow + (unsigned)c0, va);
                tc::wait_ld();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 cq = *reinterpret_cast<const float4*>(CC + c0 + 4 * q);
                    const float cv[4] = {cq.x, cq.y, cq.z, cq.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float e = __fmaf_rn(-2.f, __uint_as_float(va[4 * q + i]), cv[i]);
                        t2[i] = fminf(t2[i], fmaxf(t1[i], e));
                        tj[i] = (e < t1[i]) ? (c0 + 4 * q + i) : tj[i];
                        t1[i] = fminf(t1[i], e);
                    }
                }
            }
            float g1 = t1[0], g2 = t2[0];
            int j1 = tj[0];
#pragma unroll
            for (int c = 1; c < 4; ++c) {   // merge: least value, lowest index among equal values
                const bool take = t1[c] < g1 || (t1[c] == g1 && tj[c] < j1);
                g2 = take ? fminf(g1, t2[c]) : fminf(g2, t1[c]);
                g1 = take ? t1[c] : g1;
                j1 = take ? tj[c] : j1;
            }
            // 3. certificate, distance (x = hi + r from the two tiles); an
            //    uncertain row is decided among its candidates: the centroids
            //    whose g lies within the certificate threshold of g1
            const long long row = tile * kTxRows + r;
            const float thr = fmaxf(cert_threshold(g1, xn2, xn, cc, gB, gp2), 0x1p-60f);
            const bool good = row >= m || __fsub_rd(g2, g1) > thr;
            int lab = j1;
            float dv = 0.f;
            if (good && row < m) dv = d32_split<NP>(xhb, xlb, r, bh, bl, j1, cstride);
            const unsigned unc = __ballot_sync(0xffffffffu, !good);
            if (unc) {
                if (lane == 0) resc += __popc(unc);
                unsigned* plist = pairs[warp];
                unsigned long long* keys = pkeys[warp];
                keys[lane] = ~0ull;
                int np = 0;                                  // warp-uniform pair count
                for (int c0 = 0; c0 < sh.Npad; c0 += 16) {  // second pass over the accumulator
                    unsigned va[16];
                    tc::ld16(trow + (unsigned)c0, va);
                    tc::wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float e = __fmaf_rn(-2.f, __uint_as_float(va[i]), CC[c0 + i]);
                        const bool cand = !good && !(__fsub_rd(e, g1) > thr);
                        const unsigned cm = __ballot_sync(0xffffffffu, cand);
                        if (cm) {
                            const int slot = np + __popc(cm & ((1u << lane) - 1u));
                            if (cand && slot < kTxPairs) plist[slot] = ((unsigned)lane << 16) | (unsigned)(c0 + i);
                            np += __popc(cm);
                        }
                    }
                }
                __syncwarp();
                if (np <= kTxPairs) {                        // candidate pairs, one lane each
                    for (int p = lane; p < np; p += 32) {
                        const int l = (int)(plist[p] >> 16), j = (int)(plist[p] & 0xffffu);
                        const float d = d32_split<NP>(xhb, xlb, q4 * 32 + l, bh, bl, j, cstride);
                        atomicMin(&keys[l], ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)j);
                    }
                    __syncwarp();
                    if (!good) {
                        const unsigned long long key = keys[lane];
                        lab = (int)(key & 0xffffffffu);
                        dv = __uint_as_float((unsigned)(key >> 32));
                    }
                } else {                                     // many candidates: all centroids
                    unsigned pend = unc;
                    while (pend) {
                        const int src = __ffs(pend) - 1;
                        pend &= pend - 1;
                        const int rs = q4 * 32 + src;
                        float bd = __int_as_float(0x7f800000);
                        int bj = 0x7fffffff;
                        for (int j = lane; j < k; j += 32) {
                            const float dj = d32_split<NP>(xhb, xlb, rs, bh, bl, j, cstride);
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
                }
            }
            tc::fence_before();             // accumulator b read; its next MMA waits on conv[b]
            if (sh.inplace) {
                __syncwarp();
                if (lane == 0) tc::arrive(&empty[s]);     // this warp's rows of the stage are read
            }
            if (row < m) {
                acc_obj(facc, dv, gr.gf, inex);
                if (labels) labels[row] = lab;
            }
            s += NG;
            if (s >= S) { s -= S; ph ^= 1u; }
        }
    }

    // teardown.  Without an abort every copy and every MMA was consumed by a
    // wait of the epilogue.  After an abort (a bounded wait ran out), once
    // every role has stopped (the barrier below; the flag is final then),
    // the producer waits for its copies still in flight (only the last S can
    // be: each earlier stage was released by the epilogue after its copy
    // landed) and the MMA thread for its last commit, which covers every MMA
    // it issued, so that nothing writes this CTA's shared or tensor memory
    // after it is released.
    tc::fence_before();
    __syncthreads();
    if (*abort) {
        if (warp == kProducer && lane == 0)
            for (long long i = (issued > S ? issued - S : 0); i < issued; ++i)
                for (unsigned p = 0; p < (1u << 22) && !tc::try_wait(&full[i % S], (unsigned)((i / S) & 1)); ++p) {}
        if (warp == kMma && lane == 0 && issued > 0)
            for (unsigned p = 0;
                 p < (1u << 22) && !tc::try_wait(&accf[(issued - 1) % NG], (unsigned)(((issued - 1) / NG) & 1));
                 ++p) {}
        __syncthreads();
    }
    if (warp == kMma) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, (unsigned)sh.tmem_cols);
    }
    // objective: CTA reduction, then the grid-wide total (last CTA rounds it)
    const unsigned __int128 F = warp_sum_u128(facc);
    const unsigned long long IR = warp_sum(((unsigned long long)inex << 32) | resc);
    if (lane == 0) { red128[warp] = F; red64[warp] = IR; }
    __syncthreads();
    if (tid == 0) {
        unsigned __int128 T = 0;
        unsigned long long ir = 0;
        for (int i = 0; i < kThreads / 32; ++i) { T += red128[i]; ir += red64[i]; }
        for (int i = 0; i < 4; ++i) {
            const unsigned long long chunk = (unsigned long long)((T >> (32 * i)) & 0xffffffffu);
            if (chunk) atomicAdd(&g->obj_words[i], chunk);
        }
        if (ir >> 32) atomicAdd(&g->inexact, ir >> 32);
        if (ir & 0xffffffffull) atomicAdd(&g->rescored, ir & 0xffffffffull);
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
        const double f = u128_to_double(T, grids_from_maxbits(g->maxbits).gf);
        g->f_full = f;
        if (incumbent && f < g->f_incumbent) g->f_incumbent = f;
        g->best_worker = wsel;
        g->done_ctas = 0;
    }
}

// ------------------------------------------------- lean pass for n <= 32
// The same result as tcx_fullpass_kernel, for rows of at most 32 floats (one
// 16 KB column block per tile), with the roles of the BF16 precision pass:
//   * a producer warp keeps S tiles in flight (2-D TMA, 128-byte swizzle);
//   * G epilogue warpgroups; group b takes the tiles i = b (mod G) and has NB
//     buffer pairs (hi(x), r(x)) and NB accumulators.  It reads tile u + NB -
//     1 into registers (x of its row), writes hi(x) = trunc_tf32(x) and r(x)
//     = x - hi(x) to a buffer pair (the stage is then free) and hands it to
//     the MMA warp before it reads the accumulator of tile u;
//   * the MMA warp issues r(x).hi(c), hi(x).r(c), hi(x).hi(c) into the
//     accumulator (the split-TF32 products and bound of tcx_fullpass_kernel).
// Epilogue per row: pass 1 keeps the two least g (pairs of columns merged
// with a three-input min), pass 2 the bit mask of the columns with g <= lim,
// lim = g1 for a certified row (the first such column is its label) and
// fl_ru(g1 + thr) otherwise (its candidates: any other centroid has a larger
// direct form).  The distance is d32 of x (registers) against the label, or
// the least over the candidates (lowest index on ties), c read from an FP32
// copy; more than 8 candidates (or none: a NaN bound) are resolved by the
// whole warp over all k, the rows read again from X.
constexpr int kTx2MaxStages = 8;
constexpr int kTx2Cand = 8;
constexpr int kTx2CStride = 36;              // FP32 centroid rows: 9 units of 16 bytes apart

struct Tx2Shape {
    int ksteps, Npad, acc_stride, tmem_cols, stages, groups, nbuf;
    tc::WaitLimit wait;
};

// [X stages: S x 16 KB][hi(x): G NB x 16 KB][r(x): G NB x 16 KB][hi(c), r(c):
// 2 x Npad x 128 B][Cf: k x kTx2CStride floats][CC: Npad floats]
__host__ __device__ inline size_t tx2_smem_bytes(const Tx2Shape& s, int k) {
    return 1024 + (size_t)(s.stages + 2 * s.groups * s.nbuf) * kTxAtomBytes + (size_t)2 * s.Npad * 128 +
           (size_t)k * kTx2CStride * 4 + (size_t)s.Npad * 4;
}

template <int NP, int NG, int NB>
__global__ void __launch_bounds__(tx_threads(NG), 1)
tcx2_fullpass_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ X, long long m, int n,
                     const float* __restrict__ Cw, int k, const double* sel_f, int W, int* __restrict__ labels,
                     Globals* g, float gB, float gp2, int incumbent, Tx2Shape sh) {
    static_assert(NP <= 32, "one column block per row");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (tc::s_addr(smem_raw) & 1023)) & 1023);
    const int S = sh.stages;
    unsigned char* xs = base;                                        // X stages
    unsigned char* xh = xs + (size_t)S * kTxAtomBytes;               // hi(x), NB per group
    unsigned char* xl = xh + (size_t)NG * NB * kTxAtomBytes;         // r(x), NB per group
    unsigned char* bh = xl + (size_t)NG * NB * kTxAtomBytes;         // hi(c)
    unsigned char* bl = bh + (size_t)sh.Npad * 128;                  // r(c)
    float* Cf = reinterpret_cast<float*>(bl + (size_t)sh.Npad * 128);
    float* CC = Cf + (size_t)k * kTx2CStride;
    constexpr int kEpi = 4 * NG, kProducer = kEpi, kMma = kEpi + 1, kThreads = tx_threads(NG);
    __shared__ __align__(8) unsigned long long full[kTx2MaxStages], empty[kTx2MaxStages], conv[NG * NB],
        accf[NG * NB];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    __shared__ unsigned __int128 red128[kThreads / 32];
    __shared__ unsigned long long red64[kThreads / 32];
    __shared__ unsigned int redu[kThreads / 32];
    __shared__ CertC cert;
    __shared__ int wsel;
    __shared__ bool last;

    if (g->nonfinite) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &abort_flag;
    if (tid == 0) {
        int best = 0;
        if (sel_f)
            for (int w = 1; w < W; ++w)
                if (sel_f[w] < sel_f[best]) best = w;
        wsel = best;
        abort_flag = 0;
        for (int s = 0; s < S; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 4); }
        for (int b = 0; b < NG * NB; ++b) { tc::mbar_init(&conv[b], 4); tc::mbar_init(&accf[b], 1); }
        tc::mbar_init_fence();
    }
    if (warp == kMma) tc::tmem_alloc(&tmem_slot, (unsigned)sh.tmem_cols);
    __syncthreads();
    const float* C = Cw + (long long)wsel * k * NP;
    // B operands hi(c), r(c) (swizzled like the X tiles), the FP32 copy, CC
    // and the certificate constants
    for (int e = tid; e < sh.Npad * 8; e += kThreads) {
        const int j = e >> 3, c = e & 7;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
        if (j < k && 4 * c < NP) {
            const float4 cv = *reinterpret_cast<const float4*>(C + (size_t)j * NP + 4 * c);
            h = make_float4(trunc_tf32(cv.x), trunc_tf32(cv.y), trunc_tf32(cv.z), trunc_tf32(cv.w));
            l = make_float4(cv.x - h.x, cv.y - h.y, cv.z - h.z, cv.w - h.w);     // exact
            *reinterpret_cast<float4*>(Cf + (size_t)j * kTx2CStride + 4 * c) = cv;
        }
        const size_t off = (size_t)j * 128 + ((c ^ (j & 7)) << 4);
        *reinterpret_cast<float4*>(bh + off) = h;
        *reinterpret_cast<float4*>(bl + off) = l;
    }
    unsigned int mx = 0;
    for (int j = tid; j < sh.Npad; j += kThreads) {
        float acc = 0.f, up = 0.f;
        if (j < k) {
#pragma unroll
            for (int d = 0; d < NP; ++d) {
                const float c = C[(size_t)j * NP + d];
                acc = __fmaf_rn(c, c, acc);
                up = __fmaf_ru(c, c, up);
            }
        }
        CC[j] = (j < k) ? acc : __int_as_float(0x7f800000);
        mx = max(mx, __float_as_uint(up));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) redu[warp] = mx;
    tc::fence_proxy_async();
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
    const long long ntiles = (m + kTxRows - 1) / kTxRows;
    const long long grid = gridDim.x;

    unsigned __int128 facc = 0;
    unsigned int inex = 0, resc = 0;
    long long issued = 0;
    if (warp == kProducer) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            long long it = 0;
            int s = 0;
            unsigned ph = 0;
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                if (it >= S && !tc::wait(&empty[s], ph ^ 1u, abort, g, sh.wait)) break;
                tc::expect_tx(&full[s], (unsigned)kTxAtomBytes);
                tc::tma_load_2d(xs + (size_t)s * kTxAtomBytes, &tmap, 0, (int)(tile * kTxRows), &full[s]);
                if (++s == S) { s = 0; ph ^= 1u; }
            }
            issued = it;
        }
    } else if (warp == kMma) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            const unsigned idesc = tc::idesc_tf32(kTxRows, sh.Npad);
            const unsigned ah = tc::s_addr(bh), alo = tc::s_addr(bl);
            long long it = 0;
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                const long long u = it / NG;                     // the group's tile index
                const int b = (int)(it % NG) * NB + (int)(u % NB);   // buffer and accumulator
                if (!tc::wait(&conv[b], (unsigned)((u / NB) & 1), abort, g, sh.wait)) break;
                tc::fence_after();
                const unsigned ax = tc::s_addr(xh + (size_t)b * kTxAtomBytes);
                const unsigned al = tc::s_addr(xl + (size_t)b * kTxAtomBytes);
                const unsigned d = tmem + (unsigned)(b * sh.acc_stride);
                for (int kk = 0; kk < sh.ksteps; ++kk) {          // the correction terms first
                    tc::mma_tf32(d, tc::desc_sw128(al + 32 * kk), tc::desc_sw128(ah + 32 * kk), idesc, kk > 0);
                    tc::mma_tf32(d, tc::desc_sw128(ax + 32 * kk), tc::desc_sw128(alo + 32 * kk), idesc, 1);
                }
                for (int kk = 0; kk < sh.ksteps; ++kk)
                    tc::mma_tf32(d, tc::desc_sw128(ax + 32 * kk), tc::desc_sw128(ah + 32 * kk), idesc, 1);
                tc::commit(&accf[b]);
            }
            issued = it;
        }
    } else {
        // --------------------------------------------------- epilogue groups
        const Grids gr = grids_from_maxbits(g->maxbits);
        const CertC cc = cert;
        const int b = warp >> 2, q4 = warp & 3;
        const int r = q4 * 32 + lane;                        // row within the tile = TMEM lane
        constexpr int Q = (NP < 8 ? 8 : NP) / 4;            // 16-byte chunks the MMAs read
        int s = b;                                          // the splits' stage: it % S, (it / S) & 1
        unsigned ph = 0;                                    // (S is a multiple of NG)
        float xr[NB][Q * 4];                                // x of this thread's row, per buffer
        float xn2s[NB];                                     // bound on ||x||^2, per buffer
        // read the group's next tile into buffer XB; false on abort
        auto split = [&](auto XB) -> bool {
            constexpr int x = decltype(XB)::value;
            int ok = 1;
            if (lane == 0) ok = tc::wait(&full[s], ph, abort, g, sh.wait);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) return false;
            const unsigned char* st = xs + (size_t)s * kTxAtomBytes;
            unsigned char* xhb = xh + (size_t)(b * NB + x) * kTxAtomBytes;
            unsigned char* xlb = xl + (size_t)(b * NB + x) * kTxAtomBytes;
            float xn2 = 0.f;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const float4 w = *reinterpret_cast<const float4*>(st + tile_off(r, q));
                xr[x][4 * q] = w.x;
                xr[x][4 * q + 1] = w.y;
                xr[x][4 * q + 2] = w.z;
                xr[x][4 * q + 3] = w.w;
                xn2 = __fmaf_ru(w.x, w.x, xn2);
                xn2 = __fmaf_ru(w.y, w.y, xn2);
                xn2 = __fmaf_ru(w.z, w.z, xn2);
                xn2 = __fmaf_ru(w.w, w.w, xn2);
                const float4 h = make_float4(trunc_tf32(w.x), trunc_tf32(w.y), trunc_tf32(w.z), trunc_tf32(w.w));
                *reinterpret_cast<float4*>(xhb + tile_off(r, q)) = h;
                *reinterpret_cast<float4*>(xlb + tile_off(r, q)) =
                    make_float4(w.x - h.x, w.y - h.y, w.z - h.z, w.w - h.w);      // exact
            }
            xn2s[x] = xn2;
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                tc::arrive(&empty[s]);
                tc::arrive(&conv[b * NB + x]);
            }
            s += NG;
            if (s >= S) { s -= S; ph ^= 1u; }
            return true;
        };
        // the epilogue of the group's tile u, held in buffer XB: returns false
        // when the group is done (no tile u) or on abort
        auto epilogue = [&](long long u, auto XB) -> bool {
            constexpr int x = decltype(XB)::value;
            const long long it = b + u * NG;
            const long long tile = blockIdx.x + it * grid;
            if (tile >= ntiles) return false;
            {   // the next tile's split, before this tile's epilogue
                const long long ia = it + (long long)(NB - 1) * NG;
                if (blockIdx.x + ia * grid < ntiles && !split(std::integral_constant<int, (x + NB - 1) % NB>{}))
                    return false;
            }
            const long long row = tile * kTxRows + r;
            const unsigned trow = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)((b * NB + x) * sh.acc_stride);
            const float xn2 = xn2s[x];
            // d32 of x against c_j (ascending d, squares rounded then added)
            auto d32x = [&](int j) {
                const float* cj = Cf + (size_t)j * kTx2CStride;
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < NP / 4; ++q) {
                    const float4 c = *reinterpret_cast<const float4*>(cj + 4 * q);
                    float t;
                    t = __fsub_rn(xr[x][4 * q], c.x); acc = __fadd_rn(acc, __fmul_rn(t, t));
                    t = __fsub_rn(xr[x][4 * q + 1], c.y); acc = __fadd_rn(acc, __fmul_rn(t, t));
                    t = __fsub_rn(xr[x][4 * q + 2], c.z); acc = __fadd_rn(acc, __fmul_rn(t, t));
                    t = __fsub_rn(xr[x][4 * q + 3], c.w); acc = __fadd_rn(acc, __fmul_rn(t, t));
                }
                return acc;
            };
            const float xn = __fsqrt_ru(xn2);
            int okw = 1;
            if (lane == 0) okw = tc::wait(&accf[b * NB + x], (unsigned)((u / NB) & 1), abort, g, sh.wait);
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) return false;
            tc::fence_after();
            // pass 1: the two least g (chunks of 16 columns)
            float t1[4], t2[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { t1[c] = __int_as_float(0x7f800000); t2[c] = t1[c]; }
            for (int c0 = 0; c0 < k; c0 += 16) {
                unsigned va[16];
                tc::ld16(trow + (unsigned)c0, va);
                tc::wait_ld16(va);
                if (c0 + 16 <= k) tc::min2_chunk<false>(t1, t2, va, CC, c0, 16);
                else tc::min2_chunk<true>(t1, t2, va, CC, c0, k - c0);
            }
            float g1 = t1[0], g2 = t2[0];
#pragma unroll
            for (int c = 1; c < 4; ++c) {
                g2 = tc::min3f(g2, t2[c], fmaxf(g1, t1[c]));
                g1 = fminf(g1, t1[c]);
            }
            const float thr = fmaxf(cert_threshold(g1, xn2, xn, cc, gB, gp2), 0x1p-60f);
            const bool good = row >= m || __fsub_rd(g2, g1) > thr;
            const float lim = good ? g1 : __fadd_ru(g1, thr);
            // pass 2: the label of a certified row, the candidates of another
            int j1 = 0, cnt = 0;
            unsigned lo = 0, hi = 0;
            for (int c0 = 0; c0 < k; c0 += 16) {
                unsigned va[16];
                tc::ld16(trow + (unsigned)c0, va);
                tc::wait_ld16(va);
                const unsigned mk = (c0 + 16 <= k) ? tc::le_mask16<false>(va, CC, c0, lim, 16)
                                                   : tc::le_mask16<true>(va, CC, c0, lim, k - c0);
                if (cnt == 0 && mk) j1 = c0 + __ffs(mk) - 1;
                if (good) cnt += mk != 0u;
                unsigned mc = good ? 0u : mk;
                while (mc) {
                    const int j = c0 + __ffs(mc) - 1;
                    mc &= mc - 1u;
                    if (cnt < kTx2Cand) {
                        hi = (hi << 8) | (lo >> 24);
                        lo = (lo << 8) | (unsigned)j;
                    }
                    ++cnt;
                }
            }
            tc::fence_before();             // accumulator read; its next MMA waits on conv
            // the distance: d32 to the label, or the least over the candidates
            int lab = j1;
            float dv = __int_as_float(0x7f800000);
            const bool many = !good && (cnt < 1 || cnt > kTx2Cand);
            const int nd = (row >= m || many) ? 0 : (good ? 1 : cnt);
            for (int c = 0; c < nd; ++c) {
                const int j = good ? j1 : (int)(((c < 4 ? lo : hi) >> (8 * (c & 3))) & 0xffu);
                const float d = d32x(j);
                if (d < dv || (d == dv && j < lab)) { dv = d; lab = j; }
            }
            if (!good && row < m) ++resc;
            unsigned pend = __ballot_sync(0xffffffffu, many && row < m);
            while (pend) {                                  // all k, lanes over centroids
                const int src = __ffs(pend) - 1;
                pend &= pend - 1u;
                const long long srow = __shfl_sync(0xffffffffu, row, src);
                const float* xg = X + srow * n;
                float bd = __int_as_float(0x7f800000);
                int bj = 0x7fffffff;
                for (int j = lane; j < k; j += 32) {
                    const float* cj = Cf + (size_t)j * kTx2CStride;
                    float acc = 0.f;
                    for (int d = 0; d < n; ++d) {
                        const float t = __fsub_rn(xg[d], cj[d]);
                        acc = __fadd_rn(acc, __fmul_rn(t, t));
                    }
                    if (acc < bd || bj == 0x7fffffff) { bd = acc; bj = j; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                    if (od < bd || (od == bd && oj < bj)) { bd = od; bj = oj; }
                }
                if (lane == src) { dv = bd; lab = bj; }
            }
            if (row < m) {
                acc_obj(facc, dv, gr.gf, inex);
                if (labels) labels[row] = lab;
            }
            return true;
        };
        bool ok = true;
        if (NB == 2 && blockIdx.x + (long long)b * grid < ntiles)   // run ahead by one tile
            ok = split(std::integral_constant<int, 0>{});
        for (long long u = 0; ok; u += NB) {
            if (!epilogue(u, std::integral_constant<int, 0>{})) break;
            if (NB == 2 && !epilogue(u + 1, std::integral_constant<int, (NB == 2 ? 1 : 0)>{})) break;
        }
    }

    // teardown (as in tcx_fullpass_kernel)
    tc::fence_before();
    __syncthreads();
    if (*abort) {
        if (warp == kProducer && lane == 0)
            for (long long i = (issued > S ? issued - S : 0); i < issued; ++i)
                for (unsigned p = 0; p < (1u << 22) && !tc::try_wait(&full[i % S], (unsigned)((i / S) & 1)); ++p) {}
        if (warp == kMma && lane == 0 && issued > 0) {
            const long long il = issued - 1, ul = il / NG;
            const int bl = (int)(il % NG) * NB + (int)(ul % NB);
            for (unsigned p = 0; p < (1u << 22) && !tc::try_wait(&accf[bl], (unsigned)((ul / NB) & 1)); ++p) {}
        }
        __syncthreads();
    }
    if (warp == kMma) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, (unsigned)sh.tmem_cols);
    }
    const unsigned __int128 F = warp_sum_u128(facc);
    const unsigned long long IR = warp_sum(((unsigned long long)inex << 32) | resc);
    if (lane == 0) { red128[warp] = F; red64[warp] = IR; }
    __syncthreads();
    if (tid == 0) {
        unsigned __int128 T = 0;
        unsigned long long ir = 0;
        for (int i = 0; i < kThreads / 32; ++i) { T += red128[i]; ir += red64[i]; }
        for (int i = 0; i < 4; ++i) {
            const unsigned long long chunk = (unsigned long long)((T >> (32 * i)) & 0xffffffffu);
            if (chunk) atomicAdd(&g->obj_words[i], chunk);
        }
        if (ir >> 32) atomicAdd(&g->inexact, ir >> 32);
        if (ir & 0xffffffffull) atomicAdd(&g->rescored, ir & 0xffffffffull);
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
        const double f = u128_to_double(T, grids_from_maxbits(g->maxbits).gf);
        g->f_full = f;
        if (incumbent && f < g->f_incumbent) g->f_incumbent = f;
        g->best_worker = wsel;
        g->done_ctas = 0;
    }
}

// ------------------------------------------------------------ host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Groups: three epilogue warpgroups where the shared memory and tensor
// memory allow, else two, else one.  The stage count is a multiple of the
// group count, so that tile it and tile it - stages (the previous user of
// its stage, whose barrier phase precedes it) belong to the same group:
// every full-barrier phase is then waited on by one group, in order, and a
// wait can never be two phases ahead (where parity would alias).
bool tx_shape(int np, int k, TxShape& s) {
    if (k < 1 || k > 256 || np > 64) return false;
    s.atoms = np > 32 ? 2 : 1;
    s.ksteps = std::max(1, np / 8);
    s.Npad = (k + 15) & ~15;
    s.acc_stride = (s.Npad + 31) & ~31;
    // 227 KB per CTA, less 8 KB for the kernel's static shared memory
    constexpr size_t kDyn = 219 * 1024;
    // layouts in order of preference: hi(x) in group buffers with 3 or 2
    // groups; hi(x) in place with 2 groups; hi(x) in group buffers, 1 group
    const int order[4][2] = {{3, 0}, {2, 0}, {2, 1}, {1, 0}};
    for (const auto& o : order) {
        s.groups = o[0];
        s.inplace = o[1];
        int cols = 32;
        while (cols < s.groups * s.acc_stride) cols <<= 1;
        if (cols > 512) continue;
        s.tmem_cols = cols;
        for (s.stages = (kTxMaxStages / s.groups) * s.groups; s.stages >= s.groups; s.stages -= s.groups)
            if (tx_smem_bytes(s) <= kDyn) return true;
    }
    return false;
}

template <int NP, int NG>
cudaError_t launch_t(const CUtensorMap& tm, long long m, const float* C, int k, const double* sel_f, int W,
                     int* labels, Globals* g, float gB, float gp2, int incumbent, int sms, const TxShape& sh,
                     cudaStream_t st) {
    constexpr int threads = tx_threads(NG);
    // at most 512 / tmem_cols CTAs per SM, so that no allocation has to wait
    const int tmem_per_sm = 512 / sh.tmem_cols;
    size_t smem = tx_smem_bytes(sh);
    smem = std::max(smem, (size_t)(228 * 1024) / (size_t)(tmem_per_sm + 1) + 1024);
    smem = std::min<size_t>(smem, 219 * 1024);
    cudaFuncAttributes fa;
    cudaError_t e = func_attributes((const void*)tcx_fullpass_kernel<NP, NG>, &fa);
    if (e != cudaSuccess) return e;
    const int warps_alloc = (threads / 32 + 3) & ~3;            // warps are given registers in fours
    if ((long long)fa.numRegs * 32 * warps_alloc > 65536 || smem + fa.sharedSizeBytes > 227 * 1024)
        return cudaErrorNotSupported;
    e = allow_max_smem((const void*)tcx_fullpass_kernel<NP, NG>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = blocks_per_sm((const void*)tcx_fullpass_kernel<NP, NG>, threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, tmem_per_sm));
    const long long tiles = (m + kTxRows - 1) / kTxRows;
    const long long grid = std::max<long long>(1, std::min<long long>((long long)sms * per_sm, tiles));
    tcx_fullpass_kernel<NP, NG><<<(unsigned)grid, threads, smem, st>>>(tm, m, C, k, sel_f, W, labels, g, gB, gp2,
                                                                       incumbent, sh);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_g(const CUtensorMap& tm, long long m, const float* C, int k, const double* sel_f, int W,
                     int* labels, Globals* g, float gB, float gp2, int incumbent, int sms, const TxShape& sh,
                     cudaStream_t st) {
    if (sh.groups == 3)
        return launch_t<NP, 3>(tm, m, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, sh, st);
    if (sh.groups == 2)
        return launch_t<NP, 2>(tm, m, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, sh, st);
    return launch_t<NP, 1>(tm, m, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, sh, st);
}

// Lean pass (n <= 32): four groups with one buffer pair each where tensor
// memory and shared memory allow, else two groups with two pairs, else two
// with one; the stage count a multiple of the group count.
bool tx2_shape(int np, int k, Tx2Shape& s) {
    if (np > 32 || k < 1 || k > 256) return false;
    s.ksteps = std::max(1, np / 8);
    s.Npad = (k + 15) & ~15;
    s.acc_stride = (s.Npad + 31) & ~31;
    constexpr size_t kDyn = 219 * 1024;
    const int order[3][2] = {{4, 1}, {2, 2}, {2, 1}};
    for (const auto& o : order) {
        s.groups = o[0];
        s.nbuf = o[1];
        int cols = 32;
        while (cols < s.groups * s.nbuf * s.acc_stride) cols <<= 1;
        if (cols > 512) continue;
        s.tmem_cols = cols;
        for (s.stages = (kTx2MaxStages / s.groups) * s.groups; s.stages >= s.groups; s.stages -= s.groups)
            if (tx2_smem_bytes(s, k) <= kDyn) return true;
    }
    return false;
}

template <int NP, int NG, int NB>
cudaError_t launch2_t(const CUtensorMap& tm, const float* X, long long m, int n, const float* C, int k,
                      const double* sel_f, int W,
                      int* labels, Globals* g, float gB, float gp2, int incumbent, int sms, const Tx2Shape& sh,
                      cudaStream_t st) {
    constexpr int threads = tx_threads(NG);
    const size_t smem = tx2_smem_bytes(sh, k);
    cudaFuncAttributes fa;
    cudaError_t e = func_attributes((const void*)tcx2_fullpass_kernel<NP, NG, NB>, &fa);
    if (e != cudaSuccess) return e;
    const int warps_alloc = (threads / 32 + 3) & ~3;
    if ((long long)fa.numRegs * 32 * warps_alloc > 65536 || smem + fa.sharedSizeBytes > 227 * 1024)
        return cudaErrorNotSupported;
    e = allow_max_smem((const void*)tcx2_fullpass_kernel<NP, NG, NB>);
    if (e != cudaSuccess) return e;
    // one CTA per SM (its registers), persistent over tiles
    const long long tiles = (m + kTxRows - 1) / kTxRows;
    const long long grid = std::max<long long>(1, std::min<long long>((long long)sms, tiles));
    tcx2_fullpass_kernel<NP, NG, NB><<<(unsigned)grid, threads, smem, st>>>(tm, X, m, n, C, k, sel_f, W, labels, g,
                                                                            gB, gp2, incumbent, sh);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch2_g(const CUtensorMap& tm, const float* X, long long m, int n, const float* C, int k,
                      const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2, int incumbent, int sms,
                      const Tx2Shape& sh, cudaStream_t st) {
    if (sh.groups == 4)
        return launch2_t<NP, 4, 1>(tm, X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, sh, st);
    if (sh.nbuf == 2)
        return launch2_t<NP, 2, 2>(tm, X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, sh, st);
    return launch2_t<NP, 2, 1>(tm, X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, sh, st);
}

}  // namespace

// Whether the tensor-core pass takes (X, n, k): n % 4 == 0 (TMA row
// stride), X 16-byte aligned, n <= 64, 1 <= k <= 256, m < 2^31.
bool tcx_eligible(const float* X, long long m, int n, int np, int k) {
    TxShape s;
    Tx2Shape s2;
    return n % 4 == 0 && (((uintptr_t)X) & 15) == 0 && m >= 1 && m < (1ll << 31) &&
           (np <= 32 ? tx2_shape(np, k, s2) : tx_shape(np, k, s)) && encode_fn() != nullptr;
}

// Certificate factor of the split-TF32 products (see the file comment).
float tcx_gamma(int np) {
    const int ksteps = std::max(1, np / 8);
    return 2.0f * (float)(ksteps * 9) * 0x1p-23f + 8.0f * 0x1p-20f;
}


// Limits of the bounded waits of the next launches (process-wide).
static std::atomic<unsigned> g_wait_polls{tc::kDefaultWait.polls}, g_wait_ns{tc::kDefaultWait.ns};
void set_tcx_wait_limit(unsigned polls, unsigned ns) {
    g_wait_polls.store(polls ? polls : tc::kDefaultWait.polls);
    g_wait_ns.store(polls ? ns : tc::kDefaultWait.ns);
}
// The limit the tensor-core passes (exact and precision form) launch with.
tc::WaitLimit tcx_wait_limit() { return {g_wait_polls.load(), g_wait_ns.load()}; }

// Launch the tensor-core exact pass; cudaErrorNotSupported when not eligible.
cudaError_t launch_tcx_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                                const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                                int incumbent, int sms, cudaStream_t st) {
    if (!tcx_eligible(X, m, n, np, k)) return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 4};
    const cuuint32_t box[2] = {32, kTxRows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorNotSupported;
    const float gBt = std::max(gB, tcx_gamma(np));
    Tx2Shape s2;
    if (np <= 32 && tx2_shape(np, k, s2)) {
        s2.wait = tcx_wait_limit();
        switch (np) {
            case 4: return launch2_g<4>(tm, X, m, n, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, s2, st);
            case 8: return launch2_g<8>(tm, X, m, n, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, s2, st);
            case 16: return launch2_g<16>(tm, X, m, n, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, s2, st);
            case 32: return launch2_g<32>(tm, X, m, n, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, s2, st);
        }
        return cudaErrorNotSupported;
    }
    TxShape sh;
    if (!tx_shape(np, k, sh)) return cudaErrorNotSupported;
    sh.wait = tcx_wait_limit();
    switch (np) {
        case 4: return launch_g<4>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 8: return launch_g<8>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 16: return launch_g<16>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 32: return launch_g<32>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 64: return launch_g<64>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
    }
    return cudaErrorNotSupported;
}

}  // namespace bm
