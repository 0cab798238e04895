// Inline-PTX wrappers for the sm_103a tensor-core passes: mbarriers, bulk and
// tensor (TMA) copies, tcgen05 MMA / commit / tensor-memory loads, and the
// shared-memory and instruction descriptors they take.
#pragma once
#include <cstdint>

#include "bm_device.cuh"

namespace bm {
namespace tc {

__device__ __forceinline__ unsigned s_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(b)) : "memory");
}
__device__ __forceinline__ bool try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(s_addr(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// try_wait that may suspend the thread for up to `ns` nanoseconds while the
// phase is incomplete (it returns as soon as the phase completes).
__device__ __forceinline__ bool try_wait_sleep(unsigned long long* b, unsigned parity, unsigned ns) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(s_addr(b)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Limits of the bounded waits: `polls` polls, each suspending the thread for
// at most `ns` nanoseconds (0: a plain poll).  The default, 2^18 polls of at
// most 20 us, ends a wait after about 5 s; bm_debug_set_wait_limit sets
// smaller values for a test that makes a wait run out.
struct WaitLimit { unsigned polls, ns; };
constexpr WaitLimit kDefaultWait = {1u << 18, 20000u};

// Bounded wait.  Gives up when `abort` is raised by another role of the CTA,
// or once the limit is spent (then it raises `abort` and the timeout flag),
// so that no role of a CTA can wait forever on another.
__device__ __forceinline__ bool wait(unsigned long long* b, unsigned parity, volatile int* abort, Globals* g,
                                     WaitLimit lim) {
    for (unsigned i = 0; i < lim.polls; ++i) {
        if (lim.ns ? try_wait_sleep(b, parity, lim.ns) : try_wait(b, parity)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    atomicOr(&g->err, kErrTimeout);
    return false;
}

// 1-D bulk copy global -> shared (addresses and size multiples of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_addr(dst)),
                 "l"(src), "r"(bytes), "r"(s_addr(b))
                 : "memory");
}
// 2-D tiled tensor copy global -> shared through a tensor map; (x, y) is the
// box origin in elements (x * element size must be a multiple of 16 bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(s_addr(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(s_addr(b))
        : "memory");
}

// 64-bit shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// groups 1024 bytes apart, descriptor version 1.
__device__ __forceinline__ unsigned long long desc_sw128(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);          // start address
    d |= (unsigned long long)1u << 16;                          // leading byte offset (unused here)
    d |= (unsigned long long)(1024u >> 4) << 32;                // stride byte offset
    d |= (unsigned long long)1u << 46;                          // version
    d |= (unsigned long long)2u << 61;                          // 128-byte swizzle
    return d;
}
// Instruction descriptors: FP32 accumulate, A and B K-major, M x N.
//   kind::f16 with BF16 operands (format 1); kind::tf32 (format 2).
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__host__ __device__ constexpr unsigned idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `b` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void commit(unsigned long long* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(b))
                 : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// Generic-proxy writes to shared memory made visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor-memory allocation (whole warp); the address lands in *slot.
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(slot)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 32 lanes x 16 columns of 32-bit tensor-memory cells -> 16 registers per
// thread (no wait; pair with wait_ld).
__device__ __forceinline__ void ld16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------- epilogue helpers (g top-2)
// Both tensor-core passes read, per row, g_j = fl(ccb_j - 2 acc_j) from the
// accumulator columns in chunks of 16 and keep the two least g (pass 1),
// then a bit mask of the columns with g <= lim (pass 2).

// 16 tensor-memory columns in flight into r: the wait for them takes r as
// operands, so that no use of r can be scheduled before the wait.
__device__ __forceinline__ void wait_ld16(unsigned (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// g of the columns c0 + 4 q .. c0 + 4 q + 3 from 16 accumulator cells:
// fl(ccb - 2 acc).
__device__ __forceinline__ void g_quad(float (&e)[4], const unsigned (&va)[16], const float* ccb, int c0, int q) {
    const float4 cq = *reinterpret_cast<const float4*>(ccb + c0 + 4 * q);
    const float2 e01 = __ffma2_rn(make_float2(-2.f, -2.f),
                                  make_float2(__uint_as_float(va[4 * q]), __uint_as_float(va[4 * q + 1])),
                                  make_float2(cq.x, cq.y));
    const float2 e23 = __ffma2_rn(make_float2(-2.f, -2.f),
                                  make_float2(__uint_as_float(va[4 * q + 2]), __uint_as_float(va[4 * q + 3])),
                                  make_float2(cq.z, cq.w));
    e[0] = e01.x;
    e[1] = e01.y;
    e[2] = e23.x;
    e[3] = e23.y;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// Pass 1 over the columns c0 .. c0 + 15 (the first `nv` of them when PART):
// four chains of the least and second least g.  Each pair of columns is
// sorted (lo, hi) and merged: t2 = min(t2, hi, max(t1, lo)), t1 = min(t1, lo).
template <bool PART>
__device__ __forceinline__ void min2_chunk(float (&t1)[4], float (&t2)[4], const unsigned (&va)[16], const float* ccb,
                                           int c0, int nv) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (PART && 4 * q >= nv) break;
        float e[4];
        g_quad(e, va, ccb, c0, q);
        if (PART)                                   // columns past k: +inf
#pragma unroll
            for (int i = 0; i < 4; ++i) e[i] = (4 * q + i < nv) ? e[i] : __int_as_float(0x7f800000);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int c = (2 * q + p) & 3;
            const float lo = fminf(e[2 * p], e[2 * p + 1]), hi = fmaxf(e[2 * p], e[2 * p + 1]);
            t2[c] = min3f(t2[c], hi, fmaxf(t1[c], lo));
            t1[c] = fminf(t1[c], lo);
        }
    }
}
// Pass 2 over the columns c0 .. c0 + 15 (the first `nv` when PART): bit i
// set where g of column c0 + i is <= lim.
template <bool PART>
__device__ __forceinline__ unsigned le_mask16(const unsigned (&va)[16], const float* ccb, int c0, float lim, int nv) {
    unsigned mk = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (PART && 4 * q >= nv) break;
        float e[4];
        g_quad(e, va, ccb, c0, q);
#pragma unroll
        for (int i = 0; i < 4; ++i) mk |= (e[i] <= lim) ? (1u << (4 * q + i)) : 0u;
    }
    return PART ? mk & ((1u << nv) - 1u) : mk;
}

// Round to TF32 (10 explicit mantissa bits), to nearest, ties away from zero.
__device__ __forceinline__ float to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace bm
