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
//     atom; columns past n are filled with zeros by the copy);
//   * one tcgen05.mma kind::tf32 chain per tile computes acc_j = x.c_j for
//     all centroids into a tensor-memory accumulator (two accumulators, so
//     the MMA of tile t+1 overlaps the epilogue of tile t);
//   * the epilogue forms g_j = fl(||c_j||^2 - 2 acc_j), keeps the two least,
//     and accepts j1 when the certificate of the expanded form holds with
//     the TF32 error added to its bound (below); the distance of the row is
//     then d32(x, c_j1).  Rows whose certificate fails are re-scored by the
//     warp over all centroids in d32.
//
// Error bound behind the certificate: the tensor core reads x with at most
// 10 mantissa bits (|x~ - x| <= 2^-10 |x|), C is rounded to TF32 here
// (|c~ - c| <= 2^-11 |c|), products of TF32 values are exact in FP32, and
// the FP32 accumulation of at most 64 products adds far less than
// 2^-12 sum |x c|.  So |acc_j - x.c_j| <= 1.75 * 2^-10 ||x|| ||c_j|| and
// |g_j - (||c_j||^2 - 2 x.c_j)| <= 2^-9 (cmax^2 + 2 ||x|| cmax), which is the
// form certified() takes with its gamma factor set to 2^-9.  A gap below
// 2^-60 is never accepted (subnormal data).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "bm_device.cuh"
#include "bm_tcgen05.cuh"

namespace bm {

constexpr int kTxRows = 128;              // rows per tile (MMA M)
constexpr int kTxAtomBytes = kTxRows * 128;   // one 32-float-wide column block of a tile
constexpr int kTxEpiWarps = 4;            // epilogue warps (TMEM lane quarters)
constexpr int kTxThreads = 32 * (kTxEpiWarps + 2);   // + producer warp + MMA warp

struct TxShape {
    int atoms;       // 32-float column blocks per row (1 or 2)
    int ksteps;      // MMA instructions per tile (K = 8 each)
    int Npad;        // MMA N: k rounded up to 16
    int acc_stride;  // tensor-memory columns per accumulator
    int tmem_cols;   // columns allocated
    int stages;      // X tiles in flight
};

// Shared memory: [X stages: stages x atoms x 16 KB][B: atoms x Npad x 128 B]
// [CC: Npad floats]; X stages and B 1024-byte aligned.
__host__ __device__ inline size_t tx_smem_bytes(const TxShape& s) {
    return 1024 + (size_t)s.stages * s.atoms * kTxAtomBytes + (size_t)s.atoms * s.Npad * 128 + (size_t)s.Npad * 4;
}

template <int NP>
__global__ void __launch_bounds__(kTxThreads, 2)
tcx_fullpass_kernel(const __grid_constant__ CUtensorMap tmap, long long m, const float* __restrict__ Cw, int k,
                    const double* sel_f, int W, int* __restrict__ labels, Globals* g, float gB, float gp2,
                    int incumbent, TxShape sh) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (tc::s_addr(smem_raw) & 1023)) & 1023);
    unsigned char* xs = base;
    unsigned char* bs = xs + (size_t)sh.stages * sh.atoms * kTxAtomBytes;
    float* CC = reinterpret_cast<float*>(bs + (size_t)sh.atoms * sh.Npad * 128);
    constexpr int kMaxStages = 4;
    __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages], accf[2], acce[2];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    __shared__ unsigned __int128 red128[kTxThreads / 32];
    __shared__ unsigned long long red64[kTxThreads / 32];
    __shared__ unsigned int redu[kTxThreads / 32];
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
        for (int s = 0; s < sh.stages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], kTxEpiWarps); }
        for (int b = 0; b < 2; ++b) { tc::mbar_init(&accf[b], 1); tc::mbar_init(&acce[b], kTxEpiWarps); }
        tc::mbar_init_fence();
    }
    if (warp == kTxEpiWarps + 1) tc::tmem_alloc(&tmem_slot, (unsigned)sh.tmem_cols);
    __syncthreads();
    const float* C = Cw + (long long)wsel * k * NP;

    // B operand: TF32-rounded centroids, swizzled like the X tiles; CC and
    // the certificate constants from the FP32 centroids.
    for (int e = tid; e < sh.atoms * sh.Npad * 8; e += kTxThreads) {
        const int a = e / (sh.Npad * 8), rem = e % (sh.Npad * 8), j = rem >> 3, c = rem & 7;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        const int d0 = a * 32 + c * 4;
        if (j < k && d0 < NP) {
            const float4 cv = *reinterpret_cast<const float4*>(C + (size_t)j * NP + d0);
            v = make_float4(tc::to_tf32(cv.x), tc::to_tf32(cv.y), tc::to_tf32(cv.z), tc::to_tf32(cv.w));
        }
        *reinterpret_cast<float4*>(bs + (size_t)a * sh.Npad * 128 + (size_t)j * 128 + ((c ^ (j & 7)) << 4)) = v;
    }
    unsigned int mx = 0;
    for (int j = tid; j < sh.Npad; j += kTxThreads) {
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
    tc::fence_proxy_async();                 // B visible to the tensor core
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        unsigned int mm = 0;
        for (int i = 0; i < kTxThreads / 32; ++i) mm = max(mm, redu[i]);
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
    if (warp == kTxEpiWarps) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            long long it = 0;
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                const int s = (int)(it % S);
                if (it >= S && !tc::wait(&empty[s], (unsigned)((it / S - 1) & 1), abort, g)) break;
                tc::expect_tx(&full[s], (unsigned)(sh.atoms * kTxAtomBytes));
                for (int a = 0; a < sh.atoms; ++a)
                    tc::tma_load_2d(xs + (size_t)(s * sh.atoms + a) * kTxAtomBytes, &tmap, 32 * a,
                                    (int)(tile * kTxRows), &full[s]);
            }
            if (*abort)       // drain the copies still in flight before the CTA exits
                for (long long i = (it > S ? it - S : 0); i < it; ++i)
                    for (unsigned p = 0; p < (1u << 22) && !tc::try_wait(&full[i % S], (unsigned)((i / S) & 1)); ++p) {}
        }
    } else if (warp == kTxEpiWarps + 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            const unsigned idesc = tc::idesc_tf32(kTxRows, sh.Npad);
            long long it = 0;
            for (;; ++it) {
                const long long tile = blockIdx.x + it * grid;
                if (tile >= ntiles) break;
                const int s = (int)(it % S), b = (int)(it & 1);
                if (!tc::wait(&full[s], (unsigned)((it / S) & 1), abort, g)) break;
                if (it >= 2 && !tc::wait(&acce[b], (unsigned)((it / 2 - 1) & 1), abort, g)) break;
                tc::fence_after();
                const unsigned a0 = tc::s_addr(xs + (size_t)s * sh.atoms * kTxAtomBytes), b0 = tc::s_addr(bs);
                for (int kk = 0; kk < sh.ksteps; ++kk) {
                    const unsigned off = (unsigned)((kk & 3) * 32);
                    const unsigned aa = a0 + (unsigned)(kk >> 2) * kTxAtomBytes + off;
                    const unsigned ba = b0 + (unsigned)(kk >> 2) * (unsigned)(sh.Npad * 128) + off;
                    tc::mma_tf32(tmem + (unsigned)(b * sh.acc_stride), tc::desc_sw128(aa), tc::desc_sw128(ba), idesc,
                                 kk > 0);
                }
                tc::commit(&accf[b]);
            }
            if (*abort && it > 0)     // the last commit covers every MMA issued
                for (unsigned p = 0;
                     p < (1u << 22) && !tc::try_wait(&accf[(it - 1) & 1], (unsigned)(((it - 1) / 2) & 1)); ++p) {}
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const Grids gr = grids_from_maxbits(g->maxbits);
        const CertC cc = cert;
        const int r = warp * 32 + lane;                     // row within the tile = TMEM lane
        for (long long it = 0;; ++it) {
            const long long tile = blockIdx.x + it * grid;
            if (tile >= ntiles) break;
            const int s = (int)(it % S), b = (int)(it & 1);
            int ok = 1;
            if (lane == 0) ok = tc::wait(&accf[b], (unsigned)((it / 2) & 1), abort, g);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc::fence_after();
            // two interleaved top-2 chains over the accumulator columns
            float ga1 = __int_as_float(0x7f800000), ga2 = ga1, gb1 = ga1, gb2 = ga1;
            int ja = 0, jb = 0;
            const unsigned trow = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(b * sh.acc_stride);
            for (int c0 = 0; c0 < sh.Npad; c0 += 32) {
                unsigned va[16], vb[16];
                tc::ld16(trow + (unsigned)c0, va);
                const bool two = c0 + 16 < sh.Npad;
                if (two) tc::ld16(trow + (unsigned)(c0 + 16), vb);
                tc::wait_ld();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 cq = *reinterpret_cast<const float4*>(CC + c0 + 4 * q);
                    const float cv[4] = {cq.x, cq.y, cq.z, cq.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float e = __fmaf_rn(-2.f, __uint_as_float(va[4 * q + i]), cv[i]);
                        ga2 = fminf(ga2, fmaxf(ga1, e));
                        ja = (e < ga1) ? (c0 + 4 * q + i) : ja;
                        ga1 = fminf(ga1, e);
                    }
                }
                if (two) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 cq = *reinterpret_cast<const float4*>(CC + c0 + 16 + 4 * q);
                        const float cv[4] = {cq.x, cq.y, cq.z, cq.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float e = __fmaf_rn(-2.f, __uint_as_float(vb[4 * q + i]), cv[i]);
                            gb2 = fminf(gb2, fmaxf(gb1, e));
                            jb = (e < gb1) ? (c0 + 16 + 4 * q + i) : jb;
                            gb1 = fminf(gb1, e);
                        }
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::arrive(&acce[b]);          // accumulator b free for the MMA of tile it+2
            float g1, g2;
            int j1;
            if (ga1 <= gb1) { g1 = ga1; j1 = ja; g2 = fminf(ga2, gb1); }
            else { g1 = gb1; j1 = jb; g2 = fminf(gb2, ga1); }

            // this row of X, from the swizzled stage
            const unsigned char* st = xs + (size_t)s * sh.atoms * kTxAtomBytes;
            float x[NP];
#pragma unroll
            for (int d4 = 0; d4 < NP / 4; ++d4) {
                const float4 v = *reinterpret_cast<const float4*>(st + (size_t)(d4 >> 3) * kTxAtomBytes + r * 128 +
                                                                  (((d4 & 7) ^ (r & 7)) << 4));
                x[4 * d4 + 0] = v.x; x[4 * d4 + 1] = v.y; x[4 * d4 + 2] = v.z; x[4 * d4 + 3] = v.w;
            }
            const long long row = tile * kTxRows + r;
            float xn2 = 0.f;
#pragma unroll
            for (int d = 0; d < NP; ++d) xn2 = __fmaf_ru(x[d], x[d], xn2);
            const float xn = __fsqrt_ru(xn2);
            const bool good = certified(g1, g2, xn2, xn, cc, gB, gp2) && __fsub_rd(g2, g1) > 0x1p-60f;
            int lab = j1;
            float dv = 0.f;
            if (good) dv = d32<NP>(x, C + (size_t)j1 * NP);
            unsigned pend = __ballot_sync(0xffffffffu, row < m && !good);
            if (lane == 0) resc += __popc(pend);
            while (pend) {                                  // warp-cooperative exact re-score
                const int src = __ffs(pend) - 1;
                pend &= pend - 1;
                const int rs = warp * 32 + src;
                float xsr[NP];
#pragma unroll
                for (int d4 = 0; d4 < NP / 4; ++d4) {
                    const float4 v = *reinterpret_cast<const float4*>(
                        st + (size_t)(d4 >> 3) * kTxAtomBytes + rs * 128 + (((d4 & 7) ^ (rs & 7)) << 4));
                    xsr[4 * d4 + 0] = v.x; xsr[4 * d4 + 1] = v.y; xsr[4 * d4 + 2] = v.z; xsr[4 * d4 + 3] = v.w;
                }
                float bd = __int_as_float(0x7f800000);
                int bj = 0x7fffffff;
                for (int j = lane; j < k; j += 32) {
                    const float dj = d32<NP>(xsr, C + (size_t)j * NP);
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
            __syncwarp();
            if (lane == 0) tc::arrive(&empty[s]);          // stage s free for the copy of tile it+S
            if (row < m) {
                acc_obj(facc, dv, gr.gf, inex);
                if (labels) labels[row] = lab;
            }
        }
    }

    // teardown: every MMA has completed (consumed, or drained on abort)
    tc::fence_before();
    __syncthreads();
    if (warp == kTxEpiWarps + 1) {
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
        for (int i = 0; i < kTxThreads / 32; ++i) { T += red128[i]; ir += red64[i]; }
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

bool tx_shape(int np, int k, TxShape& s) {
    if (k < 1 || k > 256 || np > 64) return false;
    s.atoms = np > 32 ? 2 : 1;
    s.ksteps = std::max(1, np / 8);
    s.Npad = (k + 15) & ~15;
    s.acc_stride = (s.Npad + 31) & ~31;
    int cols = 32;
    while (cols < 2 * s.acc_stride) cols <<= 1;
    if (cols > 512) return false;
    s.tmem_cols = cols;
    // stages: as many as fit (2..4) while two CTAs still share an SM
    const size_t fixed = 1024 + (size_t)s.atoms * s.Npad * 128 + (size_t)s.Npad * 4;
    const size_t per = (size_t)s.atoms * kTxAtomBytes;
    const size_t budget = 113 * 1024;
    int st = budget > fixed ? (int)((budget - fixed) / per) : 0;
    s.stages = std::min(4, std::max(2, st));
    return tx_smem_bytes(s) <= 227 * 1024;
}

template <int NP>
cudaError_t launch_t(const CUtensorMap& tm, long long m, const float* C, int k, const double* sel_f, int W,
                     int* labels, Globals* g, float gB, float gp2, int incumbent, int sms, const TxShape& sh,
                     cudaStream_t st) {
    // at most 512 / tmem_cols CTAs per SM, so that no allocation has to wait
    const int tmem_per_sm = 512 / sh.tmem_cols;
    size_t smem = tx_smem_bytes(sh);
    smem = std::max(smem, (size_t)(228 * 1024) / (size_t)(tmem_per_sm + 1) + 1024);
    smem = std::min<size_t>(smem, 227 * 1024);
    cudaError_t e = cudaFuncSetAttribute(tcx_fullpass_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tcx_fullpass_kernel<NP>, kTxThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, tmem_per_sm));
    const long long tiles = (m + kTxRows - 1) / kTxRows;
    const long long grid = std::max<long long>(1, std::min<long long>((long long)sms * per_sm, tiles));
    tcx_fullpass_kernel<NP><<<(unsigned)grid, kTxThreads, smem, st>>>(tm, m, C, k, sel_f, W, labels, g, gB, gp2,
                                                                      incumbent, sh);
    return cudaGetLastError();
}

}  // namespace

// Whether the tensor-core pass takes (X, n, k): n % 4 == 0 (TMA row
// stride), X 16-byte aligned, n <= 64, 1 <= k <= 256, m < 2^31.
bool tcx_eligible(const float* X, long long m, int n, int np, int k) {
    TxShape s;
    return n % 4 == 0 && (((uintptr_t)X) & 15) == 0 && m >= 1 && m < (1ll << 31) && tx_shape(np, k, s) &&
           encode_fn() != nullptr;
}

// Launch the tensor-core exact pass; cudaErrorNotSupported when not eligible.
cudaError_t launch_tcx_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                                const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                                int incumbent, int sms, cudaStream_t st) {
    TxShape sh;
    if (!tcx_eligible(X, m, n, np, k) || !tx_shape(np, k, sh)) return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 4};
    const cuuint32_t box[2] = {32, kTxRows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorNotSupported;
    const float gBt = std::max(gB, 0x1p-9f);
    switch (np) {
        case 4: return launch_t<4>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 8: return launch_t<8>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 16: return launch_t<16>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 32: return launch_t<32>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
        case 64: return launch_t<64>(tm, m, C, k, sel_f, W, labels, g, gBt, gp2, incumbent, sms, sh, st);
    }
    return cudaErrorNotSupported;
}

}  // namespace bm
