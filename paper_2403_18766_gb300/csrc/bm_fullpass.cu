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

constexpr int kFpThreads = 256;
// Rows per thread: enough independent FMA chains per centroid to hide the
// FMA latency, few enough registers for two CTAs per SM.
template <int NP>
struct FpRows { static constexpr int v = NP <= 4 ? 8 : NP == 8 ? 6 : NP == 16 ? 4 : NP == 32 ? 2 : 1; };

// mode: selection of the centroid set.
//   sel_f == nullptr: use C directly (k x NP, padded).
//   otherwise: C = Cw + w* k NP with w* = argmin sel_f[0..W) (lowest index).
// incumbent: when set, f_incumbent = min(f_incumbent, f) and best_worker = w*.
//
// A persistent grid of warps walks X in warp tiles of 32 RT rows (row
// base + 32 r + lane for lane's r-th row, so every 16-byte load of the warp
// covers 32 consecutive rows); each warp asks L2 for its next tile while it
// computes the current one.  Per row: g_j = fl(||c_j||^2) + sum_d (-2 x_d) c_j,d
// as two interleaved partial sums (even and odd d, packed FP32 FMA) added
// at the end -- NP + 1 terms in some order, inside the certificate's
// gamma_{2NP+2} bound -- then the certificate of the least two, and d32 of
// the winner (or of every centroid for an uncertain row).
template <int NP>
__global__ void __launch_bounds__(kFpThreads, 2)
fullpass_kernel(const float* __restrict__ X, long long m, int n, const float* __restrict__ Cw,
                int k, const double* sel_f, int W, int* __restrict__ labels, Globals* g,
                float gB, float gp2, int incumbent) {
    constexpr int RT = FpRows<NP>::v;
    constexpr int kW = kFpThreads / 32;
    // Cs: rows NP floats apart (every lane reads the same centroid);
    // Cg: a copy with rows an odd number of 16-byte units apart, read at
    // per-lane labels (8 lanes of different clusters per 128-bit phase fall
    // in 8 different 4-bank groups).
    constexpr int kCs = ((NP / 4) & 1) ? NP : NP + 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Cs = reinterpret_cast<float*>(smem_raw);          // k * NP
    float* Cg = Cs + (size_t)k * NP;                          // k * kCs
    float* CC = Cg + (size_t)k * kCs;                         // k
    __shared__ unsigned __int128 red128[kW];
    __shared__ unsigned long long red64[kW];
    __shared__ unsigned int redu[kW];
    __shared__ CertC cert;
    __shared__ int wsel;
    __shared__ bool last;

    if (g->nonfinite) return;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        int best = 0;
        if (sel_f)
            for (int w = 1; w < W; ++w)
                if (sel_f[w] < sel_f[best]) best = w;
        wsel = best;
    }
    __syncthreads();
    const float* C = Cw + (sel_f ? (long long)wsel * k * NP : 0ll);
    for (int e = tid; e < k * NP; e += kFpThreads) {
        const float v = C[e];
        Cs[e] = v;
        Cg[(size_t)(e / NP) * kCs + e % NP] = v;
    }
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
        if (lane == 0) redu[tid >> 5] = mx;
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
    const bool vec = (n % 4) == 0 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

    unsigned __int128 facc = 0;
    unsigned int inex = 0, resc = 0;
    const long long tile_rows = 32ll * RT;
    const long long step = (long long)gridDim.x * kW * tile_rows;
    const long long xbytes = m * (long long)n * 4;
    for (long long base = ((long long)blockIdx.x * kW + (tid >> 5)) * tile_rows; base < m; base += step) {
        float2 m2x[RT][NP / 2];                               // -2 x, dimension pairs
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const long long row = base + 32 * r + lane;
            if (row < m) {
                const float* p = X + row * (long long)n;
                if (vec) {
#pragma unroll
                    for (int q = 0; q < NP / 4; ++q) {
                        const float4 v = (4 * q < n) ? __ldg(reinterpret_cast<const float4*>(p) + q)
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                        m2x[r][2 * q + 0] = __fmul2_rn(make_float2(-2.f, -2.f), make_float2(v.x, v.y));
                        m2x[r][2 * q + 1] = __fmul2_rn(make_float2(-2.f, -2.f), make_float2(v.z, v.w));
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < NP / 2; ++d)
                        m2x[r][d] = make_float2((2 * d < n) ? -2.f * __ldg(p + 2 * d) : 0.f,
                                                (2 * d + 1 < n) ? -2.f * __ldg(p + 2 * d + 1) : 0.f);
                }
            } else {
#pragma unroll
                for (int d = 0; d < NP / 2; ++d) m2x[r][d] = make_float2(0.f, 0.f);
            }
        }
        {   // next warp tile of this warp: L2 prefetch, one 128-byte line per lane
            const long long nb = (base + step) * (long long)n * 4;
            const long long bytes = tile_rows * (long long)n * 4;
            for (long long o = (long long)lane * 128; o < bytes; o += 32 * 128)
                if (nb + o < xbytes)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(X) + nb + o));
        }
        float g1[RT], g2[RT];
        int j1[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) { g1[r] = __int_as_float(0x7f800000); g2[r] = g1[r]; j1[r] = 0; }
        for (int j = 0; j < k; ++j) {
            const float* cj = Cs + (size_t)j * NP;
            const float ccj = CC[j];
            float2 e2[RT];
#pragma unroll
            for (int r = 0; r < RT; ++r) e2[r] = make_float2(ccj, 0.f);
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                const float4 cv = reinterpret_cast<const float4*>(cj)[q];
                const float2 c01 = make_float2(cv.x, cv.y), c23 = make_float2(cv.z, cv.w);
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    e2[r] = __ffma2_rn(m2x[r][2 * q + 0], c01, e2[r]);
                    e2[r] = __ffma2_rn(m2x[r][2 * q + 1], c23, e2[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float e = __fadd_rn(e2[r].x, e2[r].y);
                g2[r] = fminf(g2[r], fmaxf(g1[r], e));
                j1[r] = (e < g1[r]) ? j : j1[r];
                g1[r] = fminf(g1[r], e);
            }
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const long long row = base + 32 * r + lane;
            const bool valid = row < m;
            const float xn2 = xnorm2_up_m2x<NP>(m2x[r]);
            const float xn = __fsqrt_ru(xn2);
            const bool good = certified(g1[r], g2[r], xn2, xn, cc, gB, gp2);
            int lab = j1[r];
            float dv = good ? d32_m2x<NP>(m2x[r], Cg + (size_t)lab * kCs) : 0.f;
            // uncertain rows, one at a time by the whole warp (no divergence
            // into a per-lane scan of all k): lanes take centroids lane,
            // lane + 32, ... of the row (read again by every lane; its lane's
            // registers are free by now), then a warp argmin, lowest index on
            // ties
            unsigned pend = __ballot_sync(0xffffffffu, valid && !good);
            if (lane == 0) resc += __popc(pend);
            while (pend) {
                const int src = __ffs(pend) - 1;
                pend &= pend - 1u;
                const float* p = X + (base + 32 * r + src) * (long long)n;
#pragma unroll
                for (int d = 0; d < NP / 2; ++d)
                    m2x[r][d] = make_float2((2 * d < n) ? -2.f * __ldg(p + 2 * d) : 0.f,
                                            (2 * d + 1 < n) ? -2.f * __ldg(p + 2 * d + 1) : 0.f);
                float bd = __int_as_float(0x7f800000);
                int bj = 0x7fffffff;
                for (int j = lane; j < k; j += 32) {
                    const float dj = d32_m2x<NP>(m2x[r], Cs + (size_t)j * NP);
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
    }
    // CTA reduction (one pass) and the grid-wide total
    unsigned __int128 F = warp_sum_u128(facc);
    const unsigned long long IR = warp_sum(((unsigned long long)inex << 32) | resc);
    const int wid = tid >> 5;
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
    (void)n;
    const int cs = ((np / 4) & 1) ? np : np + 4;
    return (size_t)k * np * 4 + (size_t)k * cs * 4 + (size_t)k * 4;
}

template <int NP>
static cudaError_t launch_fullpass_t(const float* X, long long m, int n, const float* C, int k,
                                     const double* sel_f, int W, int* labels, Globals* g, float gB,
                                     float gp2, int incumbent, int sms, cudaStream_t st) {
    const size_t smem = fullpass_smem_bytes(NP, k, n);
    cudaError_t e = allow_max_smem((const void*)fullpass_kernel<NP>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = blocks_per_sm((const void*)fullpass_kernel<NP>, kFpThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const long long warp_tiles = (m + 32ll * FpRows<NP>::v - 1) / (32ll * FpRows<NP>::v);
    const long long ctas = (warp_tiles + kFpThreads / 32 - 1) / (kFpThreads / 32);
    const long long grid = std::max<long long>(1, std::min<long long>((long long)sms * std::max(per_sm, 1), ctas));
    fullpass_kernel<NP><<<(unsigned)grid, kFpThreads, smem, st>>>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2,
                                                                   incumbent);
    return cudaGetLastError();
}

cudaError_t launch_tcx_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                                const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                                int incumbent, int sms, cudaStream_t st);

// Which implementation full passes use: 0 = by shape (below), 1 = the
// FP32-ALU pass, 2 = the tensor-core pass where it applies (else FP32-ALU).
// All give identical labels and objective (same definition, certified).
static std::atomic<int> g_fullpass_impl{0};
static thread_local int g_last_impl = 0;
void set_fullpass_impl(int impl) { g_fullpass_impl.store(impl); }
int last_fullpass_impl() { return g_last_impl; }
int fullpass_impl_setting() { return g_fullpass_impl.load(); }
// By shape: the FP32-ALU pass costs about k NP / 2 packed FMAs per row, the
// tensor-core pass a fixed epilogue per row and centroid column, so the
// tensor cores win once the contraction per row is large.  Measured on GB300
// (10^6 x 16 and 4 10^6 x 32): the lean pass (NP <= 32) wins from NP k = 800
// (n = 16, k = 50: 55 against 67 us; n = 32, k = 25: 201 against 264 us) and
// loses at NP k <= 400 (n = 16, k = 25: 49 against 43 us); the NP = 64 pass
// from NP k > 1600.
bool fullpass_prefers_tensor(int np, int k) { return (long long)np * k > (np <= 32 ? 512 : 1600); }
cudaError_t launch_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                            const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                            int incumbent, int sms, cudaStream_t st) {
    int impl = g_fullpass_impl.load();
    if (impl == 0) impl = fullpass_prefers_tensor(np, k) ? 2 : 1;
    if (impl == 2) {
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
