#pragma once
// Fused Big-means worker kernel (template body; instantiated per padded
// width NP in bm_worker_np*.cu): one thread-block cluster per competing
// worker of Algorithm 1 (arXiv 2403.18766, Sec. 4.2-4.3).
//
// The samples of a round are drawn and gathered beforehand by the sampling
// kernel.  A worker's sample is split into contiguous row slices, one per CTA
// of its cluster.  Per pass the cluster re-seeds degenerate centroids with
// greedy K-means++ (a3), runs Lloyd's iterations (a4-a6) and applies the
// incumbent rule.  Cross-CTA exchange goes through distributed shared memory;
// every cross-CTA dependency is separated by a hardware cluster barrier
// (barrier.cluster, no spinning in this code).  All control flow that reaches
// a cluster barrier is cluster-uniform: it only depends on kernel arguments
// and on values every CTA reads after a barrier from the same place, so all
// CTAs execute the same sequence of barriers.
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "bm_device.cuh"
#include "bm_worker.cuh"

namespace bm {

template <int NP>
struct Sm {
    float* Ccur;          // k * NP  centroids of the current step
    float* Cnext;         // k * NP  next centroids, pushed by their owners
    float* CC;            // k       fl(||c||^2) FMA chain
    long long* OACC;      // owned slots * NP * kAccWords: exact coordinate sums of owned clusters
    int* ocnt;            // owned slots: member counts of owned clusters
    int* lcnt;            // k: this CTA's member counts, then bucket cursors
    int* lstart;          // k + 1: bucket starts of this CTA's rows sorted by label
    unsigned char* deg;   // k       worker's degenerate flags (identical copies)
    unsigned char* emptyall;  // k   empties of the last assignment, pushed by the owners
    Xch* x;
    ObjPart* inbox;       // kMaxCluster: objective partials of every CTA (used on rank 0)
    Decision* dec;        // rank 0's decision of the current step
    unsigned __int128* red128;    // one per warp (kMaxWarps)
    long long* red64;             // one per warp, + 1
    unsigned int* redu;           // one per warp
    CertC* cert;
    long long* bcast;             // broadcast slots: 0 f, 1 stop, 2 M/pick, 3 base,
                                  // 4 total, 5-7 candidates, 8 deadline flag
    unsigned short* labs;         // rows_cta: label of each row of the CTA (first assignment)
    unsigned short* rowlist;      // rows_cta: the CTA's row offsets sorted by label
};

template <int NP>
__device__ inline Sm<NP> carve(int k, int rows_cta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* p = smem_raw;
    Sm<NP> s;
    s.Ccur = (float*)p;            p += align16((size_t)k * NP * 4);
    s.Cnext = (float*)p;           p += align16((size_t)k * NP * 4);
    s.CC = (float*)p;              p += align16((size_t)k * 4);
    s.OACC = (long long*)p;        p += align16((size_t)k * NP * kAccWords * 8);
    s.ocnt = (int*)p;              p += align16((size_t)k * 4);
    s.lcnt = (int*)p;              p += align16((size_t)k * 4);
    s.lstart = (int*)p;            p += align16((size_t)(k + 1) * 4);
    s.deg = p;                     p += align16((size_t)k);
    s.emptyall = p;                p += align16((size_t)k);
    s.x = (Xch*)p;                 p += align16(sizeof(Xch));
    s.inbox = (ObjPart*)p;         p += align16(sizeof(ObjPart) * kMaxCluster);
    s.dec = (Decision*)p;          p += align16(sizeof(Decision));
    s.red128 = (unsigned __int128*)p; p += align16(sizeof(unsigned __int128) * kMaxWarps);
    s.red64 = (long long*)p;       p += align16(8 * (kMaxWarps + 1));
    s.redu = (unsigned int*)p;     p += align16(4 * kMaxWarps);
    s.cert = (CertC*)p;            p += align16(sizeof(CertC));
    s.bcast = (long long*)p;       p += align16(8 * 16);
    s.labs = (unsigned short*)p;
    s.rowlist = s.labs + rows_cta;
    return s;
}

template <int NP>
struct RowsPerThread { static constexpr int v = (64 / NP) > 8 ? 8 : ((64 / NP) < 1 ? 1 : 64 / NP); };

// ---------------------------------------------------------------- the CTA
// TPB: threads per CTA (256, or 512 for the largest clusters).
template <int NP, int TPB>
struct Worker {
    const WorkerArgs& a;
    cg::cluster_group cl;
    Sm<NP> sm;
    int rank, cs, w, k, n;
    int gi, G, ctaW, nW;    // cluster gi of the worker's G clusters; CTA ctaW of its nW
    int xpar = 0;           // parity of the next group exchange
    unsigned gepoch = 0;    // group barriers passed (thread 0)
    Grids g;
    float* S;               // current sample (padded rows), set per pass
    float* D2; float* Cw_mine;
    int* lab_prev;          // label of each sample row in the previous assignment

    __device__ Worker(const WorkerArgs& args, cg::cluster_group c) : a(args), cl(c) {
        cs = a.cs;
        rank = (int)cl.block_rank();
        const int ci = blockIdx.x / cs;
        if (a.ncl > 0) {
            const unsigned e = a.cmap[ci];
            w = (int)(e & 0xfffu);
            gi = (int)((e >> 16) & 0xffu);
            G = (int)(e >> 24);
        } else {
            w = a.worker_base + ci;
            gi = 0;
            G = 1;
        }
        ctaW = gi * cs + rank;
        nW = G * cs;
        k = a.k;
        n = a.n;
        sm = carve<NP>(k, a.rows_cta);
        g = grids_from_maxbits(a.glob->maxbits);
        S = a.S;
        D2 = a.D2 + (long long)w * a.D2_stride;
        lab_prev = a.lab + (long long)w * a.D2_stride;
        Cw_mine = a.Cw_cta + ((long long)w * kMaxCluster + rank) * (long long)k * NP;
    }

    __device__ Xch* rx(int q) { return cl.map_shared_rank(sm.x, q); }

    // Phase trace: rank 0, thread 0 adds elapsed SM cycles to glob->trace[i].
    __device__ bool tracer() const { return gi == 0 && rank == 0 && threadIdx.x == 0; }
    __device__ void trace_add(int i, long long t0) const {
        if (tracer()) atomicAdd(&a.glob->trace[i], (unsigned long long)(clock64() - t0));
    }

    // Sample of job (worker, slot) drawn by the sampling kernel; returns its size.
    __device__ long long use_sample(int slot) {
        const long long job = (long long)w * (a.P + 1) + slot;
        S = a.S + job * a.S_stride;
        return a.job_s[job];
    }

    // Rows of this CTA: its share of the worker's G * cs CTAs.
    __device__ void slice(long long s, long long& lo, long long& hi) const {
        lo = s * ctaW / nW;
        hi = s * (ctaW + 1) / nW;
    }
    // Rows of this CTA in K-means++, which cluster 0 of the group runs alone.
    __device__ void kslice(long long s, long long& lo, long long& hi) const {
        lo = s * rank / cs;
        hi = s * (rank + 1) / cs;
    }
    __device__ bool lead() const { return gi == 0 && rank == 0; }     // records the worker's counters

    // ------------------------------------------------ group of clusters
    // Barrier among every CTA of the worker's G clusters (G > 1): a counter
    // in global memory that each CTA increments once per barrier; a CTA waits
    // until it reaches (barriers passed) x (CTAs of the group).  The wait is
    // bounded: when it runs out, or when another CTA of the group gave up,
    // the group's abort flag is raised, every later wait of the group returns
    // at once and the launch reports a timeout (results are then discarded).
    __device__ void gsync() {
        if (G == 1) return;
        __syncthreads();
        if (threadIdx.x == 0) {
            ++gepoch;
            __threadfence();
            atomicAdd(a.xbar + w, 1u);
            const unsigned target = gepoch * (unsigned)nW;
            const volatile unsigned* bar = a.xbar + w;
            const volatile int* ab = a.xabort + w;
            for (unsigned polls = 0; *bar < target; ++polls) {
                if (*ab) break;
                if (polls >= (1u << 22)) {
                    atomicExch(a.xabort + w, 1);
                    atomicOr(&a.glob->err, kErrTimeout);
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        __syncthreads();
    }
    __device__ bool group_aborted() const { return G > 1 && *(const volatile int*)(a.xabort + w) != 0; }
    // Offsets of this worker's exchange slots (parity par, cluster q).
    __device__ size_t xslot(int par, int q) const { return ((size_t)w * 2 + par) * kMaxGroup + q; }

    // cluster barrier that also orders global-memory writes
    __device__ void csync_global() {
        __threadfence();
        cl.sync();
    }

    // ------------------------------------------------------ centroid prep
    __device__ void load_centroids(const float* src) {
        for (int e = threadIdx.x; e < k * NP; e += TPB) sm.Ccur[e] = src[e];
        __syncthreads();
    }
    __device__ void store_centroids(float* dst) {
        for (int e = threadIdx.x; e < k * NP; e += TPB) dst[e] = sm.Ccur[e];
        __syncthreads();
    }
    // fl(||c_j||^2) as an FMA chain and the certificate's upper bounds.
    __device__ void prep_centroids() {
        unsigned int mx = 0;
        for (int j = threadIdx.x; j < k; j += TPB) {
            const float* c = sm.Ccur + (size_t)j * NP;
            float acc = 0.f, up = 0.f;
#pragma unroll
            for (int d = 0; d < NP; ++d) {
                acc = __fmaf_rn(c[d], c[d], acc);
                up = __fmaf_ru(c[d], c[d], up);
            }
            sm.CC[j] = acc;
            mx = max(mx, __float_as_uint(up));
        }
        const unsigned int m = block_max_u32(mx, sm.redu);
        if (threadIdx.x == 0) {
            sm.cert->cmax2 = __uint_as_float(m);
            sm.cert->cmax = __fsqrt_ru(__uint_as_float(m));
        }
        __syncthreads();
    }

    // ------------------------------------------- exact sums at the owners
    // Additions to another CTA's shared memory are fire-and-forget reductions
    // (red, relaxed, cluster scope) on its shared::cluster address; the
    // cluster barrier that follows orders them before the owner reads.
    __device__ static unsigned cluster_addr(const void* local, int q) {
        unsigned r;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(local)), "r"(q));
        return r;
    }
    __device__ static void red_u64(unsigned addr, unsigned long long v) {
        asm volatile("red.relaxed.cluster.shared::cluster.add.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
    }
    __device__ static void red_s32(unsigned addr, int v) {
        asm volatile("red.relaxed.cluster.shared::cluster.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
    }
    // Words of (cluster j, dimension d) in the owner CTA's shared memory.
    __device__ unsigned owner_words(int j, int d) {
        return cluster_addr(sm.OACC + ((size_t)(j / cs) * NP + d) * kAccWords, j % cs);
    }
    __device__ unsigned owner_count(int j) { return cluster_addr(sm.ocnt + j / cs, j % cs); }
    // Add a signed 128-bit value to three int64 words (w0 + w1 2^32 + w2 2^64).
    __device__ static void add_words(unsigned wd, __int128 v) {
        if (v == 0) return;
        const unsigned long long lo = (unsigned long long)v;
        const unsigned long long w0 = lo & 0xffffffffull, w1 = lo >> 32;
        const unsigned long long w2 = (unsigned long long)(long long)(v >> 64);
        if (w0) red_u64(wd, w0);
        if (w1) red_u64(wd + 8, w1);
        if (w2) red_u64(wd + 16, w2);
    }
    // Move one row (held as m2x = -2 x) from cluster `from` (-1: none) to
    // `to` at their owners, this lane alone.
    __device__ bool move_row_lane(const float2 (&m2x)[NP / 2], int from, int to, unsigned int& inex) {
        bool ok = true;
        red_s32(owner_count(to), 1);
        if (from >= 0) red_s32(owner_count(from), -1);
#pragma unroll
        for (int d = 0; d < NP; ++d) {
            if (d < n) {
                __int128 v;
                ok &= fixed_of(-0.5f * ((d & 1) ? m2x[d >> 1].y : m2x[d >> 1].x), g.gx, inex, v);
                add_words(owner_words(to, d), v);
                if (from >= 0) add_words(owner_words(from, d), -v);
            }
        }
        return ok;
    }

    // The CTA's rows of the first assignment of a Lloyd run, summed per
    // cluster without per-element atomics: the rows are bucketed by label
    // (counting sort of 16-bit row offsets in shared memory), each warp walks
    // an equal share of the sorted rows with its lanes over (row, dimension),
    // in batches whose loads are issued one batch ahead, keeps the exact sum
    // in registers (two int64 parts of 48-bit-aligned pieces) and adds it to
    // the owner's words once per cluster it meets.
    __device__ bool bucket_sums(long long lo, long long hi, unsigned int& inex) {
        const int nrows = (int)(hi - lo);
        __syncthreads();                                   // labs and lcnt complete
        // counts to the owners; exclusive scan of the counts (warp 0)
        for (int j = threadIdx.x; j < k; j += TPB)
            if (sm.lcnt[j]) red_s32(owner_count(j), sm.lcnt[j]);
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int run = 0;
            for (int j0 = 0; j0 < k; j0 += 32) {
                const int j = j0 + lane;
                const int c = j < k ? sm.lcnt[j] : 0;
                int x = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (j < k) sm.lstart[j] = run + x - c;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) sm.lstart[k] = run;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < k; j += TPB) sm.lcnt[j] = sm.lstart[j];   // cursors
        __syncthreads();
        for (int i = threadIdx.x; i < nrows; i += TPB)
            sm.rowlist[atomicAdd(&sm.lcnt[sm.labs[i]], 1)] = (unsigned short)i;
        __syncthreads();
        constexpr int LPR = NP < 32 ? NP : 32;             // lanes per row
        constexpr int RPS = 32 / LPR;                      // rows per warp step
        constexpr int DPL = NP / LPR;                      // dimensions per lane (2 for NP = 64)
        constexpr int U = 4;                               // steps per batch
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int sub = lane / LPR, d0 = lane % LPR;
        const int b0 = (int)((long long)nrows * wid / (TPB / 32));
        const int b1 = (int)((long long)nrows * (wid + 1) / (TPB / 32));
        const float* Sl = S + lo * NP;
        bool ok = true;
        int cur = -1;                                      // cluster of this lane's running sum
        long long shi[DPL], slo[DPL];
#pragma unroll
        for (int t = 0; t < DPL; ++t) shi[t] = slo[t] = 0;
        // x 2^-gx as two exact power-of-two factors (each at most 2^127)
        const int eg = -g.gx;
        const int e1 = eg > 127 ? 127 : eg;
        const float s1 = __int_as_float((unsigned)(e1 + 127) << 23);
        const float s2 = __int_as_float((unsigned)(eg - e1 + 127) << 23);
        // the rows of a batch (values and labels); the next batch is loaded
        // while this one is converted and added
        auto load_batch = [&](int q0, float (&xv)[U][DPL], int (&jl)[U]) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = q0 + u * RPS;
                const int r = p < b1 ? sm.rowlist[p] : 0;
                jl[u] = p < b1 ? (int)sm.labs[r] : -1;
#pragma unroll
                for (int t = 0; t < DPL; ++t) {
                    const int d = d0 + t * LPR;
                    xv[u][t] = (p < b1 && d < n) ? Sl[(long long)r * NP + d] : 0.f;
                }
            }
        };
        float xn[U][DPL];
        int jn[U];
        load_batch(b0 + sub, xn, jn);
        for (int p0 = b0 + sub; p0 < b1; p0 += U * RPS) {
            long long hv[U][DPL], lv[U][DPL];
            int jv[U];
            // the batch's coordinates on the grid, all at once, without
            // branches: y = x 2^-gx exactly (|y| < 2^96 by the choice of gx),
            // y = hf 2^48 + lf with hf an integer and lf the exact remainder,
            // whose bits below the grid are truncated (and counted): the
            // integer fixed_of gives, split at 2^48
#pragma unroll
            for (int u = 0; u < U; ++u) {
                jv[u] = jn[u];
#pragma unroll
                for (int t = 0; t < DPL; ++t) {
                    const float y = __fmul_rn(__fmul_rn(xn[u][t], s1), s2);
                    const float hf = truncf(__fmul_rn(y, 0x1p-48f));
                    const float lf = __fmaf_rn(-hf, 0x1p48f, y);
                    const float lt = truncf(lf);
                    inex += (lf != lt) ? 1u : 0u;
                    ok &= fabsf(y) < 0x1p96f;
                    hv[u][t] = __float2ll_rz(hf);
                    lv[u][t] = __float2ll_rz(lt);
                }
            }
            if (p0 + U * RPS < b1) load_batch(p0 + U * RPS, xn, jn);
            // rows are sorted by cluster: a running sum per lane, added to the
            // owner's words when the cluster changes
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jv[u] < 0) break;                      // past this warp's rows
                if (jv[u] != cur) {
                    if (cur >= 0)
#pragma unroll
                        for (int t = 0; t < DPL; ++t) {
                            add_words(owner_words(cur, d0 + t * LPR),
                                      ((__int128)shi[t] << 48) + (__int128)slo[t]);
                            shi[t] = slo[t] = 0;
                        }
                    cur = jv[u];
                }
#pragma unroll
                for (int t = 0; t < DPL; ++t) {
                    shi[t] += hv[u][t];
                    slo[t] += lv[u][t];
                }
            }
        }
        if (cur >= 0)
#pragma unroll
            for (int t = 0; t < DPL; ++t)
                add_words(owner_words(cur, d0 + t * LPR), ((__int128)shi[t] << 48) + (__int128)slo[t]);
        return ok;
    }

    // --------------------------------------------- a4/a5: assign + accumulate
    // Assign the CTA's rows against Ccur and push the CTA partial objective to
    // rank 0's inbox.  mode 0: no sums (objective only); mode 1: first
    // assignment of a Lloyd run (the owners' sums start from zero, see
    // lloyd); mode 2: incremental -- the sums are exact integers, so only rows
    // whose label changed since the previous assignment move from their old
    // cluster to the new one.
    __device__ void assign_slice(long long s, int mode) {
        constexpr int RT = RowsPerThread<NP>::v;
        long long lo, hi;
        slice(s, lo, hi);
        if (mode == 1)
            for (int e = threadIdx.x; e < k; e += TPB) sm.lcnt[e] = 0;
        __syncthreads();
        const long long t_loop = clock64();
        const CertC cc = *sm.cert;
        const float gB = a.gB, gp2 = a.gp2;
        const int gf = g.gf;
        unsigned __int128 facc = 0;
        unsigned int inex = 0, resc = 0;
        bool ok = true;
        const int lane = threadIdx.x & 31;
        // warp-uniform trip count (the move step below uses warp ballots)
        for (long long base0 = lo + (long long)(threadIdx.x & ~31) * RT; base0 < hi;
             base0 += (long long)TPB * RT) {
            const long long base = base0 + (long long)lane * RT;
            float2 m2x[RT][NP / 2];                          // -2 x, dimension pairs
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const long long row = base + r;
                if (row < hi) {
                    const float4* p = reinterpret_cast<const float4*>(S + row * NP);
#pragma unroll
                    for (int q = 0; q < NP / 4; ++q) {
                        const float4 v = p[q];
                        m2x[r][2 * q + 0] = make_float2(-2.f * v.x, -2.f * v.y);
                        m2x[r][2 * q + 1] = make_float2(-2.f * v.z, -2.f * v.w);
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < NP / 2; ++d) m2x[r][d] = make_float2(0.f, 0.f);
                }
            }
            int oldlab[RT];
#pragma unroll
            for (int r = 0; r < RT; ++r)
                oldlab[r] = (mode == 2 && base + r < hi) ? lab_prev[base + r] : -1;
            {   // start the L2 -> L1 fetch of this thread's rows of the next trip
                const long long nb = base + (long long)TPB * RT;
                if (nb < hi) {
                    const char* pn = reinterpret_cast<const char*>(S + nb * NP);
#pragma unroll
                    for (int o = 0; o < RT * NP * 4; o += 128)
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(pn + o));
                    if (mode == 2) asm volatile("prefetch.global.L1 [%0];" ::"l"(lab_prev + nb));
                }
            }
            float g1[RT], g2[RT];
            int j1[RT];
#pragma unroll
            for (int r = 0; r < RT; ++r) { g1[r] = __int_as_float(0x7f800000); g2[r] = g1[r]; j1[r] = 0; }
            for (int j = 0; j < k; ++j) {
                // g_j = ||c_j||^2 - 2 x.c_j as two interleaved partial sums
                // (even and odd dimensions, packed FP32 FMA), then added:
                // NP + 1 terms in another order, inside the certificate's
                // gamma_{2NP+2} bound.
                const float* cj = sm.Ccur + (size_t)j * NP;
                const float ccj = sm.CC[j];
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
                float e[RT];
#pragma unroll
                for (int r = 0; r < RT; ++r) e[r] = __fadd_rn(e2[r].x, e2[r].y);
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    g2[r] = fminf(g2[r], fmaxf(g1[r], e[r]));
                    j1[r] = (e[r] < g1[r]) ? j : j1[r];
                    g1[r] = fminf(g1[r], e[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const long long row = base + r;
                const bool valid = row < hi;
                const float xn2 = xnorm2_up_m2x<NP>(m2x[r]);
                const float xn = __fsqrt_ru(xn2);
                int lab = 0;
                float dv = 0.f;
                if (valid) {
                    if (certified(g1[r], g2[r], xn2, xn, cc, gB, gp2)) {
                        lab = j1[r];
                        dv = d32_m2x<NP>(m2x[r], sm.Ccur + (size_t)lab * NP);
                    } else {
                        resc++;
                        dv = d32_m2x<NP>(m2x[r], sm.Ccur);
                        for (int j = 1; j < k; ++j) {
                            const float dj = d32_m2x<NP>(m2x[r], sm.Ccur + (size_t)j * NP);
                            if (dj < dv) { dv = dj; lab = j; }
                        }
                    }
                    acc_obj(facc, dv, gf, inex);
                }
                if (mode == 1) {
                    if (valid) {
                        lab_prev[row] = lab;
                        sm.labs[row - lo] = (unsigned short)lab;
                        atomicAdd(&sm.lcnt[lab], 1);
                    }
                } else if (mode == 2) {
                    // Move rows whose label changed between clusters.  Many
                    // movers: each lane moves its own row.  Few movers (later
                    // iterations): the warp moves them one at a time, lanes
                    // over dimensions, so the warp does not walk the move path
                    // with one or two lanes active.
                    const bool moved = valid && oldlab[r] != lab;
                    const unsigned mv = __ballot_sync(0xffffffffu, moved);
                    if (__popc(mv) > 8) {
                        if (moved) {
                            // the row is in registers (x = -m2x / 2, exact)
                            ok &= move_row_lane(m2x[r], oldlab[r], lab, inex);
                            lab_prev[row] = lab;
                        }
                    } else {
                        unsigned rem = mv;
                        while (rem) {
                            const int src = __ffs(rem) - 1;
                            rem &= rem - 1u;
                            const long long srow = __shfl_sync(0xffffffffu, row, src);
                            const int snew = __shfl_sync(0xffffffffu, lab, src);
                            const int sold = __shfl_sync(0xffffffffu, oldlab[r], src);
                            if (lane == src) {
                                red_s32(owner_count(snew), 1);
                                red_s32(owner_count(sold), -1);
                                lab_prev[srow] = snew;
                            }
                            const float* xr = S + srow * NP;
                            for (int d = lane; d < n; d += 32) {
                                __int128 v;
                                ok &= fixed_of(xr[d], g.gx, inex, v);
                                add_words(owner_words(snew, d), v);
                                add_words(owner_words(sold, d), -v);
                            }
                        }
                    }
                }
            }
        }
        if (mode == 1) {
            if (tracer()) atomicAdd(&a.glob->trace[15], (unsigned long long)(clock64() - t_loop));
            ok &= bucket_sums(lo, hi, inex);
        }
        if (!ok) atomicOr(&a.glob->err, kErrDigits);
        const long long t_red = clock64();
        if (mode) trace_add(mode == 1 ? 14 : 8, t_loop);   // 14: first assignment of a run
        // one fused CTA reduction: objective (128-bit) and the two counters,
        // pushed into rank 0's inbox
        unsigned __int128 F = warp_sum_u128(facc);
        const unsigned long long IR = warp_sum(((unsigned long long)inex << 32) | resc);
        const int wid = threadIdx.x >> 5;
        if (lane == 0) { sm.red128[wid] = F; sm.red64[wid] = (long long)IR; }
        __syncthreads();
        if (threadIdx.x < 32) {
            F = (lane < (TPB / 32)) ? sm.red128[lane] : (unsigned __int128)0;
            unsigned long long ir = (lane < (TPB / 32)) ? (unsigned long long)sm.red64[lane] : 0ull;
            F = warp_sum_u128(F);
            ir = warp_sum(ir);
            if (lane == 0) {
                ObjPart* dst = cl.map_shared_rank(sm.inbox, 0) + rank;
                dst->f_lo = (unsigned long long)F;
                dst->f_hi = (unsigned long long)(F >> 64);
                dst->inexact = ir >> 32;
                dst->rescored = ir & 0xffffffffull;
            }
        }
        if (mode) trace_add(9, t_red);
    }

    // After a barrier, on rank 0, warp 0: the CTA partials of the inbox
    // combined into the cluster's partial (exact; valid in lane 0).
    __device__ void cluster_objective_warp(unsigned __int128& F, unsigned long long& I, unsigned long long& R) {
        const int lane = threadIdx.x & 31;
        F = 0; I = 0; R = 0;
        for (int q = lane; q < cs; q += 32) {
            const ObjPart& p = sm.inbox[q];
            F += ((unsigned __int128)p.f_hi << 64) | (unsigned __int128)p.f_lo;
            I += p.inexact;
            R += p.rescored;
        }
        F = warp_sum_u128(F);
        I = warp_sum(I);
        R = warp_sum(R);
    }
    // The worker's objective from partials (F, I, R) of every cluster: with
    // one cluster these are the partials themselves; with a group, rank 0 of
    // each cluster publishes its partial (before the group barrier) and adds
    // up all of them (after it).  f = the exact sum rounded once (lane 0);
    // the counters are recorded once per worker.
    __device__ void publish_objective(const unsigned __int128& F, unsigned long long I, unsigned long long R) {
        if (G > 1 && (threadIdx.x & 31) == 0) {
            unsigned long long* o = a.xobj + xslot(xpar, gi) * 4;
            o[0] = (unsigned long long)F;
            o[1] = (unsigned long long)(F >> 64);
            o[2] = I;
            o[3] = R;
        }
    }
    __device__ double total_objective(unsigned __int128 F, unsigned long long I, unsigned long long R) {
        if (G > 1) {
            F = 0; I = 0; R = 0;
            for (int q = 0; q < G; ++q) {
                const volatile unsigned long long* o = a.xobj + xslot(xpar, q) * 4;
                F += ((unsigned __int128)o[1] << 64) | (unsigned __int128)o[0];
                I += o[2];
                R += o[3];
            }
        }
        if ((threadIdx.x & 31) == 0 && gi == 0) {
            if (I) atomicAdd(&a.glob->inexact, I);
            if (R) atomicAdd(&a.glob->rescored, R);
        }
        return u128_to_double(F, g.gf);
    }
    // Owners publish their clusters' partial sums and counts (group only).
    __device__ void publish_sums() {
        if (G == 1) return;
        const int nOwned = (k - rank + cs - 1) / cs;
        long long* dst = a.xpart + xslot(xpar, gi) * (size_t)k * NP * kAccWords;
        int* dcnt = a.xcnt + xslot(xpar, gi) * (size_t)k;
        for (int e = threadIdx.x; e < nOwned * NP; e += TPB) {
            const int slot = e / NP, d = e % NP, j = rank + slot * cs;
            const long long* wd = sm.OACC + (size_t)e * kAccWords;
            long long* o = dst + ((size_t)j * NP + d) * kAccWords;
            o[0] = wd[0]; o[1] = wd[1]; o[2] = wd[2];
            if (d == 0) dcnt[j] = sm.ocnt[slot];
        }
    }
    // Rank 0, one thread: the decision to every CTA of the cluster.
    __device__ void push_decision(double f, int stop) {
        for (int q = 0; q < cs; ++q) {
            Decision* d = cl.map_shared_rank(sm.dec, q);
            d->f = f;
            d->stop = stop;
        }
    }

    // Zero the owned sums and counts (before a Lloyd run; a cluster barrier
    // must follow before any CTA adds to them).
    __device__ void zero_owned() {
        const int nOwned = (k - rank + cs - 1) / cs;
        for (int e = threadIdx.x; e < nOwned * NP * kAccWords; e += TPB) sm.OACC[e] = 0;
        for (int e = threadIdx.x; e < nOwned; e += TPB) sm.ocnt[e] = 0;
    }

    // a6 (owner part): new centroid of each owned cluster j (j % cs == rank):
    // float(double(exact sum) / count); an empty cluster keeps its centroid.
    // The sums are complete in this CTA's shared memory; the new centroids
    // and the empty flags are pushed into every CTA's Cnext / emptyall.
    __device__ void owner_update() {
        const int nOwned = (k - rank + cs - 1) / cs;
        const int total = nOwned * NP;
        for (int e = threadIdx.x; e < total; e += TPB) {
            const int slot = e / NP, d = e % NP;
            const int j = rank + slot * cs;
            __int128 V = 0;
            long long cntj = 0;
            if (G == 1) {
                const long long* wd = sm.OACC + (size_t)e * kAccWords;
                V = (__int128)wd[0] + ((__int128)wd[1] << 32) + ((__int128)wd[2] << 64);
                cntj = sm.ocnt[slot];
            } else {                                 // the group's partials, in global memory
                for (int q = 0; q < G; ++q) {
                    const volatile long long* wd =
                        a.xpart + (xslot(xpar, q) * (size_t)k * NP + (size_t)j * NP + d) * kAccWords;
                    V += (__int128)wd[0] + ((__int128)wd[1] << 32) + ((__int128)wd[2] << 64);
                    cntj += ((const volatile int*)a.xcnt)[xslot(xpar, q) * (size_t)k + j];
                }
            }
            float c = sm.Ccur[(size_t)j * NP + d];
            if (cntj > 0 && d < n) {
                c = __double2float_rn(__ddiv_rn(i128_to_double(V, g.gx), (double)cntj));
            }
            const unsigned char em = (cntj == 0) ? 1 : 0;
            for (int q = 0; q < cs; ++q) {
                cl.map_shared_rank(sm.Cnext, q)[(size_t)j * NP + d] = c;
                if (d == 0) cl.map_shared_rank(sm.emptyall, q)[j] = em;
            }
        }
    }

    // f(Ccur, S) without updating centroids (recompute of f_hat_w, recheck).
    __device__ double eval(long long s) {
        assign_slice(s, 0);
        cl.sync();                                       // partials in rank 0's inbox
        unsigned __int128 F = 0;
        unsigned long long I = 0, R = 0;
        if (rank == 0 && threadIdx.x < 32) {
            cluster_objective_warp(F, I, R);
            publish_objective(F, I, R);
        }
        gsync();                                         // every cluster's partial published
        if (rank == 0 && threadIdx.x < 32) {
            const double f = total_objective(F, I, R);
            if (threadIdx.x == 0) push_decision(f, 1);
        }
        xpar ^= 1;
        cl.sync();                                       // decision in every CTA
        const double f = sm.dec->f;
        if (lead() && threadIdx.x == 0) atomicAdd(&a.glob->eval_rows, (unsigned long long)s);
        return f;
    }

    // Lloyd from Ccur (Sec. 4.1; Sec. 5 stop rule).  On return Ccur holds the
    // result C_a, emptyall its empty clusters, `iters` the number of updates.
    __device__ double lloyd(long long s, int& iters) {
        zero_owned();
        cl.sync();                                       // no CTA adds before the owners cleared
        double f_prev = 0.0;
        int it = 0;
        for (;;) {
            const long long t_a = clock64();
            assign_slice(s, it == 0 ? 1 : 2);
            trace_add(1, t_a);
            if (tracer()) atomicAdd(&a.glob->trace[6], 1ull);
            const long long t_x = clock64();
            cl.sync();                                       // sums and partials at their owners
            trace_add(10, t_x);
            const long long t_o = clock64();
            unsigned __int128 F = 0;
            unsigned long long I = 0, R = 0;
            if (G > 1) {                                     // partials of every cluster of the group
                publish_sums();
                if (rank == 0 && threadIdx.x < 32) {
                    cluster_objective_warp(F, I, R);
                    publish_objective(F, I, R);
                }
                gsync();
            } else if (rank == 0 && threadIdx.x < 32) {
                cluster_objective_warp(F, I, R);
            }
            owner_update();
            if (rank == 0 && threadIdx.x < 32) {
                const double f = total_objective(F, I, R);
                if (threadIdx.x == 0) {
                    int stop;
                    if (it == 0) stop = (a.max_lloyd <= 0);
                    else stop = (__dsub_rn(f_prev, f) <= __dmul_rn(a.tol, f_prev)) || (it >= a.max_lloyd);
                    if (group_aborted()) stop = 1;
                    push_decision(f, stop);
                }
            }
            xpar ^= 1;
            trace_add(11, t_o);
            const long long t_b2 = clock64();
            cl.sync();                                       // updates + decision in every CTA
            trace_add(12, t_b2);
            const long long t_p = clock64();
            const double f = sm.dec->f;
            const int stop = sm.dec->stop;
            if (stop) {
                trace_add(2, t_x);
                iters = it;
                return f;
            }
            for (int e = threadIdx.x; e < k * NP; e += TPB) sm.Ccur[e] = sm.Cnext[e];
            __syncthreads();
            prep_centroids();
            trace_add(13, t_p);
            trace_add(2, t_x);
            f_prev = f;
            ++it;
        }
    }

    // ------------------------------------------------ a3: greedy K-means++
    __device__ static int frexp_exp(unsigned int mb) {   // M = f * 2^E, f in [0.5, 1)
        const unsigned ef = mb >> 23;
        if (ef) return (int)ef - 126;
        return (32 - __clz((int)(mb & 0x7fffff))) - 149;
    }
    __device__ static long long quant(float v, int E) {   // floor(v * 2^(31 - E))
        const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
        if (!b) return 0;
        uint32_t mant; int e2;
        f32_parts(b, mant, e2);
        const int sh = e2 + 31 - E;
        if (sh >= 0) return (long long)mant << sh;
        if (-sh >= 32) return 0;
        return (long long)(mant >> (-sh));
    }

    __device__ void load_row(long long i, float (&x)[NP]) const {
        const float4* p = reinterpret_cast<const float4*>(S + i * NP);
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) {
            const float4 v = p[q];
            x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
        }
    }

    __device__ void kmeanspp(long long s, unsigned long long k1) {
        long long lo, hi;
        kslice(s, lo, hi);
        bool any_live = false;
        for (int j = 0; j < k; ++j) any_live |= (sm.deg[j] == 0);
        unsigned int mloc = 0;
        if (any_live) {
            for (long long i = lo + threadIdx.x; i < hi; i += TPB) {
                float x[NP];
                load_row(i, x);
                float dm = __int_as_float(0x7f800000);
                for (int j = 0; j < k; ++j)
                    if (!sm.deg[j]) dm = fminf(dm, d32<NP>(x, sm.Ccur + (size_t)j * NP));
                D2[i] = dm;
                mloc = max(mloc, __float_as_uint(dm));
            }
        }
        __syncthreads();
        const int trials = a.trials < 1 ? 1 : (a.trials > 3 ? 3 : a.trials);
        const long long ch = (hi - lo + TPB - 1) / TPB;
        const long long c0 = lo + ch * threadIdx.x, c1 = min(hi, c0 + ch);
        for (int j = 0; j < k; ++j) {
            if (!sm.deg[j]) continue;
            long long pick;
            if (!any_live) {
                pick = (long long)draw_below(a.seed, k1, 0, (unsigned long long)j, (unsigned long long)s);
            } else {
                const unsigned int mb = block_max_u32(mloc, sm.redu);
                if (threadIdx.x == 0) sm.x->maxbits = mb;
                cl.sync();                                                   // [A]
                if (threadIdx.x == 0) {
                    unsigned int M = 0;
                    for (int q = 0; q < cs; ++q) M = max(M, rx(q)->maxbits);
                    sm.bcast[2] = M;
                }
                __syncthreads();
                const unsigned int M = (unsigned int)sm.bcast[2];
                if (M == 0) {
                    pick = (long long)draw_below(a.seed, k1, 0, (unsigned long long)j, (unsigned long long)s);
                } else {
                    const int E = frexp_exp(M);
                    long long wmine = 0;
                    for (long long i = c0; i < c1; ++i) wmine += quant(D2[i], E);
                    long long ctaTot;
                    const long long excl = block_exscan(wmine, sm.red64, &ctaTot);
                    if (threadIdx.x == 0) sm.x->wsum = ctaTot;
                    cl.sync();                                               // [B]
                    if (threadIdx.x < 4) sm.x->cand[threadIdx.x] = -1;
                    if (threadIdx.x == 0) {
                        long long base = 0, tot = 0;
                        for (int q = 0; q < cs; ++q) {
                            const long long v = rx(q)->wsum;
                            if (q < rank) base += v;
                            tot += v;
                        }
                        sm.bcast[3] = base;
                        sm.bcast[4] = tot;
                    }
                    __syncthreads();
                    const long long base = sm.bcast[3];
                    const unsigned long long Wtot = (unsigned long long)sm.bcast[4];
                    for (int l = 0; l < trials; ++l) {
                        const unsigned long long u = draw_below(a.seed, k1, (unsigned long long)l,
                                                                (unsigned long long)j, Wtot);
                        const long long lo_w = base + excl;
                        if ((long long)u >= lo_w && (long long)u < lo_w + wmine) {
                            long long run = lo_w;
                            for (long long i = c0; i < c1; ++i) {
                                run += quant(D2[i], E);
                                if (run > (long long)u) { sm.x->cand[l] = (int)i; break; }
                            }
                        }
                    }
                    cl.sync();                                               // [C]
                    if (threadIdx.x < trials) {
                        int c = -1;
                        for (int q = 0; q < cs; ++q) c = max(c, rx(q)->cand[threadIdx.x]);
                        sm.bcast[5 + threadIdx.x] = c;
                    }
                    __syncthreads();
                    int cand[3];
#pragma unroll
                    for (int l = 0; l < 3; ++l) {
                        cand[l] = (l < trials) ? (int)sm.bcast[5 + l] : 0;
                        if (cand[l] < 0 || cand[l] >= s) {          // cannot happen: prefix covers [0, W)
                            if (threadIdx.x == 0) atomicOr(&a.glob->err, kErrArgs);
                            cand[l] = 0;
                        }
                    }
                    long long pot[3] = {0, 0, 0};
                    for (long long i = lo + threadIdx.x; i < hi; i += TPB) {
                        float x[NP];
                        load_row(i, x);
                        const float d2 = D2[i];
#pragma unroll
                        for (int l = 0; l < 3; ++l) {
                            if (l < trials) {
                                const float dc = d32<NP>(x, S + (long long)cand[l] * NP);
                                pot[l] += quant(fminf(d2, dc), E);
                            }
                        }
                    }
#pragma unroll
                    for (int l = 0; l < 3; ++l) {
                        if (l < trials) {
                            const long long t = block_sum<long long>(pot[l], sm.red64);
                            if (threadIdx.x == 0) sm.x->pot[l] = t;
                        }
                    }
                    cl.sync();                                               // [D]
                    if (threadIdx.x == 0) {
                        long long best = 0;
                        int bl = 0;
                        for (int l = 0; l < trials; ++l) {
                            long long t = 0;
                            for (int q = 0; q < cs; ++q) t += rx(q)->pot[l];
                            if (l == 0 || t < best) { best = t; bl = l; }
                        }
                        sm.bcast[2] = cand[bl];
                    }
                    __syncthreads();
                    pick = sm.bcast[2];
                    __syncthreads();
                }
            }
            // centroid j = S[pick]
            if (lead() && threadIdx.x == 0) atomicAdd(&a.glob->reseeded, 1ull);
            for (int d = threadIdx.x; d < NP; d += TPB) sm.Ccur[(size_t)j * NP + d] = S[pick * NP + d];
            __syncthreads();
            mloc = 0;
            for (long long i = lo + threadIdx.x; i < hi; i += TPB) {
                float x[NP];
                load_row(i, x);
                const float dj = d32<NP>(x, sm.Ccur + (size_t)j * NP);
                const float v = any_live ? fminf(D2[i], dj) : dj;
                D2[i] = v;
                mloc = max(mloc, __float_as_uint(v));
            }
            __syncthreads();
            any_live = true;
        }
    }
};

// trials > 3 would need more broadcast slots; the host caps it at 3.

// BATCH: a launch for several fits, whose arguments are read from device
// memory (p.batch[fit of the cluster]); otherwise the kernel parameter itself.
template <int NP, int TPB, bool BATCH>
__global__ void __launch_bounds__(TPB, 512 / TPB) worker_kernel(const __grid_constant__ WorkerArgs p) {
    // The launch must have the cluster shape and grid the arguments describe
    // (every exchange addresses the other CTAs of the cluster by rank): if
    // not, record the error and leave before any barrier or remote access.
    if (cg::this_cluster().num_blocks() != (unsigned)p.cs || gridDim.x % (unsigned)p.cs != 0 ||
        (p.ncl > 0 && gridDim.x != (unsigned)(p.ncl * p.cs))) {
        if (threadIdx.x == 0) atomicOr(&p.glob->err, kErrArgs);
        return;
    }
    const WorkerArgs& a = BATCH ? p.batch[(p.cmap[blockIdx.x / p.cs] >> 12) & 0xfu] : p;
    Worker<NP, TPB> W(a, cg::this_cluster());
    if (a.glob->nonfinite) return;            // uniform: read before any barrier
    const int w = W.w;

    if (a.mode == kModeStepKpp || a.mode == kModeStepLloyd) {
        // S (padded) and C (padded, in a.Cw) were staged by the host.
        W.load_centroids(a.Cw);
        for (int j = threadIdx.x; j < W.k; j += TPB) W.sm.deg[j] = a.deg[j];
        __syncthreads();
        W.cl.sync();
        if (a.mode == kModeStepKpp) {
            W.kmeanspp(a.step_s, stream_k1(kPurposeKpp, a.step_worker, a.step_round, a.step_pass));
        } else {
            W.prep_centroids();
            int iters = 0;
            const double f = W.lloyd(a.step_s, iters);
            if (W.rank == 0 && threadIdx.x == 0) { *a.step_f = f; *a.step_iters = iters; }
            if (W.rank == 0)
                for (int j = threadIdx.x; j < W.k; j += TPB) a.step_empty[j] = W.sm.emptyall[j];
        }
        if (W.rank == 0) W.store_centroids(a.Cw);
        W.csync_global();
        return;
    }

    // worker state for this launch
    const long long t_kernel = clock64();
    for (int j = threadIdx.x; j < W.k; j += TPB) W.sm.deg[j] = a.deg[(long long)w * W.k + j];
    for (int e = threadIdx.x; e < W.k * NP; e += TPB)
        W.Cw_mine[e] = a.Cw[(long long)w * W.k * NP + e];
    __syncthreads();
    double fhat = a.fhat[w];

    if (a.mode == kModeFinalEval) {
        // the common sample S (job 0 of the final sampling launch)
        W.S = a.S;
        const long long s_opt = a.job_s[0];
        W.load_centroids(W.Cw_mine);
        W.prep_centroids();
        const double f = W.eval(s_opt);
        if (W.rank == 0 && threadIdx.x == 0) a.f_final[w] = f;
        W.cl.sync();
        return;
    }

    // ---------------------------------------------------- Algorithm 1 round
    // Samples of this round were drawn and gathered by the sampling kernel:
    // slots 0..P-1 are the passes, slot P the f_hat recompute sample.
    bool failed = false, out_of_time = false;
    int rounds_completed = 0;
    for (int t = a.round_begin; t < a.round_end && !failed && !out_of_time; ++t) {
        const long long s_w = W.use_sample(a.P);
        if (s_w <= 0) { failed = true; break; }
        bool all_deg = true;
        for (int j = 0; j < W.k; ++j) all_deg &= (W.sm.deg[j] != 0);
        if (!all_deg) {                                  // recompute f_hat_w with the new s_w
            const long long t_e = clock64();
            W.load_centroids(W.Cw_mine);
            W.prep_centroids();
            fhat = W.eval(s_w);
            W.trace_add(3, t_e);
        }
        for (int p = 0; p < a.P; ++p) {
            if (a.deadline_ns) {
                // the lead CTA reads the clock; its decision reaches every CTA
                // of the cluster (and, for a group, every cluster)
                if (W.lead() && threadIdx.x == 0) {
                    unsigned long long now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                    const int late = (now >= a.deadline_ns) ? 1 : 0;
                    W.sm.x->flag = late;
                    if (W.G > 1) a.xflag[(size_t)w * 2 + W.xpar] = late;
                }
                if (W.G > 1) {
                    W.gsync();
                    if (threadIdx.x == 0) W.sm.bcast[8] = *(const volatile int*)(a.xflag + (size_t)w * 2 + W.xpar);
                    W.xpar ^= 1;
                } else {
                    W.cl.sync();
                    if (threadIdx.x == 0) W.sm.bcast[8] = W.rx(0)->flag;
                }
                __syncthreads();
                const bool late = W.sm.bcast[8] != 0;
                W.cl.sync();
                if (late) { out_of_time = true; break; }
            }
            W.use_sample(p);
            W.load_centroids(W.Cw_mine);
            bool any_deg = false;
            for (int j = 0; j < W.k; ++j) any_deg |= (W.sm.deg[j] != 0);
            if (any_deg) {
                // re-seeding is in place (Alg. 1); a group's cluster 0 runs it
                // over the whole sample and hands the centroids to the others
                const long long t_k = clock64();
                if (W.gi == 0) W.kmeanspp(s_w, stream_k1(kPurposeKpp, w, t, p));
                if (W.G > 1) {
                    if (W.gi == 0 && W.rank == 0) W.store_centroids(a.xC + (size_t)w * W.k * NP);
                    W.gsync();
                    if (W.gi > 0) W.load_centroids(a.xC + (size_t)w * W.k * NP);
                }
                W.store_centroids(W.Cw_mine);
                W.trace_add(0, t_k);
            }
            W.prep_centroids();
            int iters = 0;
            const double f = W.lloyd(s_w, iters);
            if (f < fhat) {                              // incumbent rule
                fhat = f;
                for (int j = threadIdx.x; j < W.k; j += TPB) W.sm.deg[j] = W.sm.emptyall[j];
                W.store_centroids(W.Cw_mine);
                if (W.lead() && threadIdx.x == 0) {
                    const unsigned long long pos = atomicAdd(&a.glob->accepts, 1ull);
                    atomicAdd(&a.glob->L_sum, (unsigned long long)s_w);
                    if ((long long)pos < a.L_cap) a.L_buf[pos] = s_w;
                }
            }
            __syncthreads();
            if (W.lead() && threadIdx.x == 0) {
                atomicAdd(&a.glob->passes, 1ull);
                atomicAdd(&a.glob->lloyd_iters, (unsigned long long)iters);
                atomicAdd(&a.glob->assign_rows, (unsigned long long)(s_w * (iters + 1)));
            }
        }
        if (!failed && !out_of_time) ++rounds_completed;
    }
    if (failed && W.lead() && threadIdx.x == 0) atomicOr(&a.glob->err, kErrSample);
    // persist worker state
    if (W.lead()) {
        for (int e = threadIdx.x; e < W.k * NP; e += TPB)
            a.Cw[(long long)w * W.k * NP + e] = W.Cw_mine[e];
        for (int j = threadIdx.x; j < W.k; j += TPB) a.deg[(long long)w * W.k + j] = W.sm.deg[j];
        if (threadIdx.x == 0) {
            a.fhat[w] = fhat;
            atomicMin(&a.glob->rounds_done, a.round_begin + rounds_completed);
            const unsigned long long dt = (unsigned long long)(clock64() - t_kernel);
            atomicAdd(&a.glob->trace[4], dt);
            atomicMax(&a.glob->trace[5], dt);
            atomicAdd(&a.glob->trace[7], 1ull);
        }
    }
    W.csync_global();
}

template <int NP>
int worker_max_cluster_t(int k) {
    const size_t smem = worker_smem_bytes<NP>(k);
    if (allow_max_smem((const void*)worker_kernel<NP, 256, false>) != cudaSuccess ||
        allow_max_smem((const void*)worker_kernel<NP, 512, false>) != cudaSuccess ||
        cudaFuncSetAttribute(worker_kernel<NP, 256, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(worker_kernel<NP, 512, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, worker_kernel<NP, 256, false>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    return nclusters > 0 ? 16 : 8;
}

template <int NP>
int worker_active_clusters_t(int cs, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, size_t>, int> memo;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(cs, smem);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    if (allow_max_smem((const void*)worker_kernel<NP, 256, false>) != cudaSuccess ||
        (cs > 8 && cudaFuncSetAttribute(worker_kernel<NP, 256, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, worker_kernel<NP, 256, false>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        ncl = 0;
    }
    memo[key] = ncl;
    return ncl;
}

template <int NP, int TPB, bool BATCH>
cudaError_t launch_worker_tpb(const WorkerArgs& a, int clusters, cudaStream_t st) {
    const size_t smem = worker_smem_bytes<NP>(a.k_smem > 0 ? a.k_smem : a.k) + bucket_smem_bytes(a.rows_cta);
    cudaError_t e = allow_max_smem((const void*)worker_kernel<NP, TPB, BATCH>);
    if (e != cudaSuccess) return e;
    if (a.cs > 8) {
        e = cudaFuncSetAttribute(worker_kernel<NP, TPB, BATCH>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * a.cs), 1, 1);
    cfg.blockDim = dim3(TPB, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.coop ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, worker_kernel<NP, TPB, BATCH>, a);
}

// a.tpb = 512 runs the worker with 512-thread CTAs (one per SM), else 256.
template <int NP>
cudaError_t launch_worker_t(const WorkerArgs& a, int clusters, cudaStream_t st) {
    if (a.batch) return launch_worker_tpb<NP, 256, true>(a, clusters, st);
    return a.tpb == 512 ? launch_worker_tpb<NP, 512, false>(a, clusters, st)
                        : launch_worker_tpb<NP, 256, false>(a, clusters, st);
}

}  // namespace bm
