// Full-data pass of Algorithm 1 (its last step, Y <- nearest centroid of every
// x in X) and the objective f(C, X) of Eq. (1); plus the input prepass.
//
// The pass streams X once: a persistent grid of CTAs walks row tiles, each
// thread assigns RT rows against the centroids held in shared memory with the
// certified FP32 expanded form, re-scores uncertain rows in the FP32 direct
// form, stores labels and accumulates the exact objective in 128-bit fixed
// point.  CTA partials go to global memory as 32-bit chunks added into four
// 64-bit words; the last CTA to finish rounds the total once to double.
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

// mode: selection of the centroid set.
//   sel_f == nullptr: use C directly (k x NP, padded).
//   otherwise: C = Cw + w* k NP with w* = argmin sel_f[0..W) (lowest index).
// incumbent: when set, f_incumbent = min(f_incumbent, f) and best_worker = w*.
template <int NP>
__global__ void __launch_bounds__(kThreads, 1)
fullpass_kernel(const float* __restrict__ X, long long m, int n, const float* __restrict__ Cw,
                int k, const double* sel_f, int W, int* __restrict__ labels, Globals* g,
                float gB, float gp2, int incumbent) {
    constexpr int RT = (64 / NP) > 8 ? 8 : ((64 / NP) < 1 ? 1 : 64 / NP);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Cs = reinterpret_cast<float*>(smem_raw);                       // k * NP
    float* CC = Cs + (size_t)k * NP;                                      // k
    __shared__ unsigned __int128 red128[kWarps];
    __shared__ unsigned long long red64[kWarps];
    __shared__ unsigned int redu[kWarps];
    __shared__ CertC cert;
    __shared__ int wsel;
    __shared__ bool last;

    if (g->nonfinite) return;
    if (threadIdx.x == 0) {
        int best = 0;
        if (sel_f)
            for (int w = 1; w < W; ++w)
                if (sel_f[w] < sel_f[best]) best = w;
        wsel = best;
    }
    __syncthreads();
    const float* C = Cw + (sel_f ? (long long)wsel * k * NP : 0ll);
    for (int e = threadIdx.x; e < k * NP; e += kThreads) Cs[e] = C[e];
    __syncthreads();
    unsigned int mx = 0;
    for (int j = threadIdx.x; j < k; j += kThreads) {
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
    const unsigned int mm = block_max_u32(mx, redu);
    if (threadIdx.x == 0) { cert.cmax2 = __uint_as_float(mm); cert.cmax = __fsqrt_ru(cert.cmax2); }
    __syncthreads();
    const CertC cc = cert;
    const Grids gr = grids_from_maxbits(g->maxbits);

    unsigned __int128 facc = 0;
    unsigned int inex = 0, resc = 0;
    const long long rows_per_cta_iter = (long long)kThreads * RT;
    for (long long base0 = (long long)blockIdx.x * rows_per_cta_iter; base0 < m;
         base0 += (long long)gridDim.x * rows_per_cta_iter) {
        const long long base = base0 + (long long)threadIdx.x;     // rows base + r*kThreads
        float m2x[RT][NP];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const long long row = base + (long long)r * kThreads;
            const float* xr = X + row * (long long)n;
#pragma unroll
            for (int d = 0; d < NP; ++d) m2x[r][d] = (row < m && d < n) ? -2.f * __ldg(xr + d) : 0.f;
        }
        float g1[RT], g2[RT];
        int j1[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) { g1[r] = __int_as_float(0x7f800000); g2[r] = g1[r]; j1[r] = 0; }
        for (int j = 0; j < k; ++j) {
            const float* cj = Cs + (size_t)j * NP;
            const float ccj = CC[j];
            float e[RT];
#pragma unroll
            for (int r = 0; r < RT; ++r) e[r] = ccj;
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                const float4 cv = reinterpret_cast<const float4*>(cj)[q];
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    e[r] = __fmaf_rn(m2x[r][4 * q + 0], cv.x, e[r]);
                    e[r] = __fmaf_rn(m2x[r][4 * q + 1], cv.y, e[r]);
                    e[r] = __fmaf_rn(m2x[r][4 * q + 2], cv.z, e[r]);
                    e[r] = __fmaf_rn(m2x[r][4 * q + 3], cv.w, e[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                g2[r] = fminf(g2[r], fmaxf(g1[r], e[r]));
                j1[r] = (e[r] < g1[r]) ? j : j1[r];
                g1[r] = fminf(g1[r], e[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const long long row = base + (long long)r * kThreads;
            if (row >= m) continue;
            float x[NP];
            float xn2 = 0.f;
#pragma unroll
            for (int d = 0; d < NP; ++d) {
                x[d] = -0.5f * m2x[r][d];
                xn2 = __fmaf_ru(x[d], x[d], xn2);
            }
            const float xn = __fsqrt_ru(xn2);
            int lab;
            float dv;
            if (certified(g1[r], g2[r], xn2, xn, cc, gB, gp2)) {
                lab = j1[r];
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
    const unsigned __int128 F = block_sum_u128(facc, red128);
    const unsigned long long I = block_sum<unsigned long long>(inex, red64);
    const unsigned long long R = block_sum<unsigned long long>(resc, red64);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) {
            const unsigned long long chunk = (unsigned long long)((F >> (32 * i)) & 0xffffffffu);
            if (chunk) atomicAdd(&g->obj_words[i], chunk);
        }
        if (I) atomicAdd(&g->inexact, I);
        if (R) atomicAdd(&g->rescored, R);
        __threadfence();
        const unsigned int prev = atomicAdd(&g->done_ctas, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
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
size_t fullpass_smem_bytes(int np, int k) { return (size_t)k * np * 4 + (size_t)k * 4; }

template <int NP>
static cudaError_t launch_fullpass_t(const float* X, long long m, int n, const float* C, int k,
                                     const double* sel_f, int W, int* labels, Globals* g, float gB,
                                     float gp2, int incumbent, int grid, cudaStream_t st) {
    const size_t smem = fullpass_smem_bytes(NP, k);
    cudaError_t e = cudaFuncSetAttribute(fullpass_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    fullpass_kernel<NP><<<grid, kThreads, smem, st>>>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent);
    return cudaGetLastError();
}

cudaError_t launch_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                            const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                            int incumbent, int grid, cudaStream_t st) {
    switch (np) {
        case 4: return launch_fullpass_t<4>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, grid, st);
        case 8: return launch_fullpass_t<8>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, grid, st);
        case 16: return launch_fullpass_t<16>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, grid, st);
        case 32: return launch_fullpass_t<32>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, grid, st);
        case 64: return launch_fullpass_t<64>(X, m, n, C, k, sel_f, W, labels, g, gB, gp2, incumbent, grid, st);
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
