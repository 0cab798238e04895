// Full-data pass of Algorithm 1 (its last step, Y <- nearest centroid of every
// x in X) and the objective f(C, X) of Eq. (1); plus the input prepass.
//
// The pass streams X once: a persistent grid of CTAs walks row tiles, each
// thread assigns RT rows against the centroids held in shared memory with the
// certified FP32 expanded form, re-scores uncertain rows in the FP32 direct
// form, stores labels and accumulates the exact objective in 128-bit fixed
// point.  CTA partials go to global memory as 32-bit chunks added into four
// 64-bit words; the last CTA to finish rounds the total once to double.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "bm_device.cuh"
#include "bm_worker.cuh"

namespace bm {

// Max |v| bit pattern and count of non-finite values over `count` floats.
__global__ void __launch_bounds__(kThreads) prepass_kernel(const float* __restrict__ v, long long count,
                                                           Globals* g) {
    __shared__ unsigned int red[kWarps];
    __shared__ unsigned long long redl[kWarps];
    unsigned int mx = 0;
    unsigned long long bad = 0;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count; i += stride) {
        const unsigned int b = __float_as_uint(v[i]) & 0x7fffffffu;
        if (b >= 0x7f800000u) bad++;
        else mx = max(mx, b);
    }
    const unsigned int m = block_max_u32(mx, red);
    const unsigned long long nb = block_sum<unsigned long long>(bad, redl);
    if (threadIdx.x == 0) {
        atomicMax(&g->maxbits, m);
        if (nb) atomicAdd(&g->nonfinite, (unsigned int)min(nb, 0xffffffffull));
    }
}

// ------------------------------------------------------------ TMA helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared, completing on `bar` (addresses and size
// multiples of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` polls and reports it.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, Globals* g) {
    for (unsigned i = 0; i < (1u << 24); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(&g->err, kErrTimeout);
    return false;
}

constexpr int kFpThreads = 256;      // rows per tile = threads per CTA (one row each)
template <int NP>
__host__ __device__ constexpr int fp_stages() { return NP >= 64 ? 2 : 3; }   // tiles in flight

// mode: selection of the centroid set.
//   sel_f == nullptr: use C directly (k x NP, padded).
//   otherwise: C = Cw + w* k NP with w* = argmin sel_f[0..W) (lowest index).
// incumbent: when set, f_incumbent = min(f_incumbent, f) and best_worker = w*.
//
// X is consumed in tiles of kFpThreads rows: a persistent CTA walks tiles
// t0, t0 + grid, ...; thread 0 keeps kFpStages tiles in flight with 1-D bulk
// copies (TMA) completing on per-stage mbarriers; every thread assigns one
// row of the current tile from shared memory.  The ragged last tile is read
// with plain loads.
template <int NP>
__global__ void __launch_bounds__(kFpThreads)
fullpass_kernel(const float* __restrict__ X, long long m, int n, const float* __restrict__ Cw,
                int k, const double* sel_f, int W, int* __restrict__ labels, Globals* g,
                float gB, float gp2, int incumbent) {
    constexpr int kW = kFpThreads / 32;
    constexpr int kFpStages = fp_stages<NP>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const size_t tile_bytes = (size_t)kFpThreads * n * 4;
    float* stage_buf = reinterpret_cast<float*>(smem_raw);                       // kFpStages tiles
    float* Cs = reinterpret_cast<float*>(smem_raw + kFpStages * tile_bytes);     // k * NP
    float* CC = Cs + (size_t)k * NP;                                             // k
    // per-warp row buffer with an odd stride (n + 1 words): conflict-free
    // both for the copy out of the stage and for one row per lane
    float* wbuf = CC + ((k + 3) & ~3) + (size_t)(threadIdx.x >> 5) * 32 * (n + 1);
    __shared__ __align__(8) unsigned long long bar[kFpStages];
    __shared__ unsigned __int128 red128[kW];
    __shared__ unsigned long long red64[kW];
    __shared__ unsigned int redu[kW];
    __shared__ CertC cert;
    __shared__ int wsel;
    __shared__ bool last;

    if (g->nonfinite) return;
    const int tid = threadIdx.x;
    if (tid == 0) {
        int best = 0;
        if (sel_f)
            for (int w = 1; w < W; ++w)
                if (sel_f[w] < sel_f[best]) best = w;
        wsel = best;
        for (int st = 0; st < kFpStages; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const long long ntiles = (m + kFpThreads - 1) / kFpThreads;
    const long long full_tiles = m / kFpThreads;              // tiles copied with TMA
    const long long grid = gridDim.x;
    auto issue = [&](long long tile, int st) {
        if (tile < full_tiles) {
            mbar_expect_tx(&bar[st], (unsigned)tile_bytes);
            bulk_g2s(stage_buf + (size_t)st * kFpThreads * n, X + tile * kFpThreads * (long long)n,
                     (unsigned)tile_bytes, &bar[st]);
        }
    };
    if (tid == 0)
        for (int st = 0; st < kFpStages; ++st) issue(blockIdx.x + st * grid, st);

    const float* C = Cw + (sel_f ? (long long)wsel * k * NP : 0ll);
    for (int e = tid; e < k * NP; e += kFpThreads) Cs[e] = C[e];
    __syncthreads();
    unsigned int mx = 0;
    for (int j = tid; j < k; j += kFpThreads) {
        float acc = 0.f, up = 0.f;
#pragma unroll
        for (int d = 0; d < NP; ++d) {
            const float c = Cs[(size_t)j * NP + d];
            acc = __fmaf_rn(c, c, acc);
            up = __fmaf_ru(c, c, up);
        }
        CC[j] = acc;
        mx = max(mx, __float_as_uint(up));
    }
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) redu[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            unsigned int mm = 0;
            for (int i = 0; i < kW; ++i) mm = max(mm, redu[i]);
            cert.cmax2 = __uint_as_float(mm);
            cert.cmax = __fsqrt_ru(cert.cmax2);
        }
        __syncthreads();
    }
    const CertC cc = cert;
    const Grids gr = grids_from_maxbits(g->maxbits);

    unsigned __int128 facc = 0;
    unsigned int inex = 0, resc = 0;
    for (long long it = 0;; ++it) {
        const long long tile = blockIdx.x + it * grid;
        if (tile >= ntiles) break;
        const int st = (int)(it % kFpStages);
        const unsigned parity = (unsigned)((it / kFpStages) & 1);
        const long long row = tile * kFpThreads + tid;
        float m2x[NP];
        if (tile < full_tiles) {
            mbar_wait(&bar[st], parity, g);
            const int lane = tid & 31;
            const float* src = stage_buf + (size_t)st * kFpThreads * n + (size_t)(tid & ~31) * n;
            __syncwarp();
            for (int r = 0; r < 32; ++r)
                for (int d = lane; d < n; d += 32) wbuf[r * (n + 1) + d] = src[r * n + d];
            __syncwarp();
            const float* xr = wbuf + lane * (n + 1);
#pragma unroll
            for (int d = 0; d < NP; ++d) m2x[d] = (d < n) ? -2.f * xr[d] : 0.f;
        } else {
            const float* xr = X + row * (long long)n;
#pragma unroll
            for (int d = 0; d < NP; ++d) m2x[d] = (row < m && d < n) ? -2.f * __ldg(xr + d) : 0.f;
        }
        // the stage is free once every thread has its row in registers
        __syncthreads();
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tile + kFpStages * grid, st);
        }
        float g1 = __int_as_float(0x7f800000), g2 = g1;
        int j1 = 0;
        for (int j = 0; j < k; ++j) {
            const float* cj = Cs + (size_t)j * NP;
            float e = CC[j];
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                const float4 cv = reinterpret_cast<const float4*>(cj)[q];
                e = __fmaf_rn(m2x[4 * q + 0], cv.x, e);
                e = __fmaf_rn(m2x[4 * q + 1], cv.y, e);
                e = __fmaf_rn(m2x[4 * q + 2], cv.z, e);
                e = __fmaf_rn(m2x[4 * q + 3], cv.w, e);
            }
            g2 = fminf(g2, fmaxf(g1, e));
            j1 = (e < g1) ? j : j1;
            g1 = fminf(g1, e);
        }
        if (row < m) {
            float x[NP];
            float xn2 = 0.f;
#pragma unroll
            for (int d = 0; d < NP; ++d) {
                x[d] = -0.5f * m2x[d];
                xn2 = __fmaf_ru(x[d], x[d], xn2);
            }
            const float xn = __fsqrt_ru(xn2);
            int lab;
            float dv;
            if (certified(g1, g2, xn2, xn, cc, gB, gp2)) {
                lab = j1;
                dv = d32<NP>(x, Cs + (size_t)lab * NP);
            } else {
                resc++;
                lab = 0;
                dv = d32<NP>(x, Cs);
                for (int j = 1; j < k; ++j) {
                    const float dj = d32<NP>(x, Cs + (size_t)j * NP);
                    if (dj < dv) { dv = dj; lab = j; }
                }
            }
            acc_obj(facc, dv, gr.gf, inex);
            if (labels) labels[row] = lab;
        }
    }
    // CTA reduction (one pass) and the grid-wide total
    unsigned __int128 F = warp_sum_u128(facc);
    const unsigned long long IR = warp_sum(((unsigned long long)inex << 32) | resc);
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) { red128[wid] = F; red64[wid] = IR; }
    __syncthreads();
    if (tid == 0) {
        unsigned __int128 T = 0;
        unsigned long long ir = 0;
        for (int i = 0; i < kW; ++i) { T += red128[i]; ir += red64[i]; }
        for (int i = 0; i < 4; ++i) {
            const unsigned long long chunk = (unsigned long long)((T >> (32 * i)) & 0xffffffffu);
            if (chunk) atomicAdd(&g->obj_words[i], chunk);
        }
        if (ir >> 32) atomicAdd(&g->inexact, ir >> 32);
        if (ir & 0xffffffffull) atomicAdd(&g->rescored, ir & 0xffffffffull);
        __threadfence();
        const unsigned int prev = atomicAdd(&g->done_ctas, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last && tid == 0) {
        __threadfence();
        unsigned __int128 T = 0;
        for (int i = 0; i < 4; ++i) {
            const unsigned long long wv = atomicAdd(&g->obj_words[i], 0ull);
            T += (unsigned __int128)wv << (32 * i);
            g->obj_words[i] = 0;
        }
        const double f = u128_to_double(T, gr.gf);
        g->f_full = f;
        if (incumbent) {
            if (f < g->f_incumbent) g->f_incumbent = f;
        }
        g->best_worker = wsel;
        g->done_ctas = 0;
    }
}

// ----------------------------------------------------------- small kernels
// Copy rows of width n into rows of width NP (zero padding), or back.
__global__ void pad_rows_kernel(const float* __restrict__ src, long long rows, int n, int np,
                                float* __restrict__ dst) {
    const long long total = rows * np;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / np;
        const int d = (int)(e % np);
        dst[e] = d < n ? src[i * n + d] : 0.f;
    }
}
__global__ void unpad_rows_kernel(const float* __restrict__ src, long long rows, int n, int np,
                                  float* __restrict__ dst) {
    const long long total = rows * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / n;
        const int d = (int)(e % n);
        dst[e] = src[i * np + d];
    }
}
// Select the centroids of argmin sel_f (lowest index) and unpad them.
__global__ void select_unpad_kernel(const float* __restrict__ Cw, const double* sel_f, int W, int k,
                                    int n, int np, float* __restrict__ dst) {
    __shared__ int wsel;
    if (threadIdx.x == 0) {
        int best = 0;
        for (int w = 1; w < W; ++w)
            if (sel_f[w] < sel_f[best]) best = w;
        wsel = best;
    }
    __syncthreads();
    const float* C = Cw + (long long)wsel * k * np;
    for (int e = threadIdx.x; e < k * n; e += blockDim.x) dst[e] = C[(e / n) * np + (e % n)];
}
__global__ void init_state_kernel(double* fhat, int W, unsigned char* deg, long long kdeg, Globals* g) {
    for (int w = threadIdx.x; w < W; w += blockDim.x) fhat[w] = __longlong_as_double(0x7ff0000000000000ll);
    for (long long e = threadIdx.x; e < kdeg; e += blockDim.x) deg[e] = 1;
    if (threadIdx.x == 0) g->f_incumbent = __longlong_as_double(0x7ff0000000000000ll);
}
__global__ void globaltimer_kernel(unsigned long long* out) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    *out = now;
}

// ------------------------------------------------------------ host launchers
size_t fullpass_smem_bytes(int np, int k, int n) {
    const int stages = np >= 64 ? 2 : 3;
    return (size_t)stages * kFpThreads * n * 4 + (size_t)k * np * 4 + (size_t)((k + 3) & ~3) * 4 +
           (size_t)(kFpThreads / 32) * 32 * (n + 1) * 4;
}

template <int NP>
static cudaError_t launch_fullpass_t(const float* X, long long m, int n, const float* C, int k,
                                     const double* sel_f, int W, int* labels, Globals* g, float gB,
                                     float gp2, int incumbent, int sms, cudaStream_t st) {
    const size_t smem = fullpass_smem_bytes(NP, k, n);
    cudaError_t e = allow_max_smem((const void*)fullpass_kernel<NP>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fullpass_kernel<NP>, kFpThreads, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (m + kFpThreads - 1) / kFpThreads;
    const long long grid = std::max<long long>(1, std::min<long long>((long long)sms * std::max(per_sm, 1), tiles));
    fullpass_kernel<NP><<<(unsigned)grid, kFpThreads, smem, st>>>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2,
                                                                   incumbent);
    return cudaGetLastError();
}

cudaError_t launch_tcx_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                                const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                                int incumbent, int sms, cudaStream_t st);

// Which implementation full passes use: 0 = the tensor-core pass where it
// applies, else the FP32-ALU pass; 1 = always the FP32-ALU pass.  Both give
// identical labels and objective (same definition, certified).
static std::atomic<int> g_fullpass_impl{0};
static thread_local int g_last_impl = 0;
void set_fullpass_impl(int impl) { g_fullpass_impl.store(impl); }
int last_fullpass_impl() { return g_last_impl; }
int fullpass_impl_setting() { return g_fullpass_impl.load(); }

cudaError_t launch_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                            const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                            int incumbent, int sms, cudaStream_t st) {
    if (g_fullpass_impl.load() == 0) {
        const cudaError_t e = launch_tcx_fullpass(np, X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, st);
        if (e != cudaErrorNotSupported) {
            g_last_impl = 2;
            return e;
        }
    }
    g_last_impl = 1;
    switch (np) {
        case 4: return launch_fullpass_t<4>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, st);
        case 8: return launch_fullpass_t<8>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, st);
        case 16: return launch_fullpass_t<16>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, st);
        case 32: return launch_fullpass_t<32>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, st);
        case 64: return launch_fullpass_t<64>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, sms, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_prepass(const float* v, long long count, Globals* g, int grid, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    prepass_kernel<<<grid, kThreads, 0, st>>>(v, count, g);
    return cudaGetLastError();
}
cudaError_t launch_pad(const float* src, long long rows, int n, int np, float* dst, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const long long total = rows * np;
    const int grid = (int)min(4096ll, (total + 255) / 256);
    pad_rows_kernel<<<grid, 256, 0, st>>>(src, rows, n, np, dst);
    return cudaGetLastError();
}
cudaError_t launch_unpad(const float* src, long long rows, int n, int np, float* dst, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const long long total = rows * n;
    const int grid = (int)min(4096ll, (total + 255) / 256);
    unpad_rows_kernel<<<grid, 256, 0, st>>>(src, rows, n, np, dst);
    return cudaGetLastError();
}
cudaError_t launch_select_unpad(const float* Cw, const double* sel_f, int W, int k, int n, int np,
                                float* dst, cudaStream_t st) {
    select_unpad_kernel<<<1, 256, 0, st>>>(Cw, sel_f, W, k, n, np, dst);
    return cudaGetLastError();
}
cudaError_t launch_init_state(double* fhat, int W, unsigned char* deg, long long kdeg, Globals* g,
                              cudaStream_t st) {
    init_state_kernel<<<1, 256, 0, st>>>(fhat, W, deg, kdeg, g);
    return cudaGetLastError();
}
cudaError_t launch_globaltimer(unsigned long long* out, cudaStream_t st) {
    globaltimer_kernel<<<1, 1, 0, st>>>(out);
    return cudaGetLastError();
}

}  // namespace bm
