// bm_assign_noalloc: the full-data pass of bm_assign without any device
// memory allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// full-data assignment: services that reserve all of their device memory in
// their own pool at start-up, or loops with a fixed memory budget in which an
// allocation could fail or wait for the device at an unpredictable moment.
// For them this entry point keeps its scratch (the accumulators and the
// padded centroids) in a fixed-size array inside the library.  Every GPU that
// loads the library holds that array until the process exits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/bigmeans.h"
#include "bm_device.cuh"

namespace bm {
bm_status set_error(bm_status s, const char* msg);
size_t fullpass_smem_bytes(int np, int k, int n);
cudaError_t launch_fullpass(int np, const float* X, long long m, int n, const float* C, int k,
                            const double* sel_f, int W, int* labels, Globals* g, float gB, float gp2,
                            int incumbent, int grid, cudaStream_t st);
cudaError_t launch_prepass(const float* v, long long count, Globals* g, int grid, cudaStream_t st);
cudaError_t launch_pad(const float* src, long long rows, int n, int np, float* dst, cudaStream_t st);
bm_status status_from_flags(const Globals& h);
}  // namespace bm

namespace {

constexpr long long kMaxCentroidFloats = 16384;          // k * padded n, 64 KiB
constexpr size_t kGlobalsBytes = (sizeof(bm::Globals) + 255) & ~(size_t)255;
constexpr size_t kScratchBytes = kGlobalsBytes + (size_t)kMaxCentroidFloats * 4;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

bm_status err(bm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return bm::set_error(s, buf);
}

int padded(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64; }

float gamma_up(int q) {
    const double u = std::ldexp(1.0, -24);
    return std::nextafter((float)(q * u / (1.0 - q * u)), INFINITY);
}

}  // namespace

// The scratch itself: accumulators (a Globals record) followed by the
// centroids padded to the kernel's width.  Host code must not use this name
// as a device address; it uses the address looked up below.
static __device__ __align__(256) unsigned char bm_noalloc_scratch[kScratchBytes];

extern "C" bm_status bm_assign_noalloc(const float* X_dev, int64_t m, int32_t n, const float* C_dev,
                                       int32_t k, int32_t* labels_out_dev, double* f_out_host,
                                       void* stream) {
    if (m < 1 || m >= (1ll << 31)) return err(BM_EINVAL, "m = %lld out of range [1, 2^31)", (long long)m);
    if (n < 1 || n > 64) return err(BM_EINVAL, "n = %d out of range [1, 64]", n);
    if (k < 1) return err(BM_EINVAL, "k = %d must be >= 1", k);
    const int np = padded(n);
    if ((long long)k * np > kMaxCentroidFloats)
        return err(BM_EINVAL, "k * padded n = %lld exceeds the fixed scratch of %lld floats "
                              "(bm_assign has no such limit)", (long long)k * np, kMaxCentroidFloats);
    if (bm::fullpass_smem_bytes(np, k, n) > 227 * 1024)
        return err(BM_EINVAL, "k = %d with n = %d needs more shared memory than the full pass has", k, n);
    if (!X_dev || ((uintptr_t)X_dev & 15)) return err(BM_EINVAL, "X_dev is NULL or not 16-byte aligned");
    if (!C_dev) return err(BM_EINVAL, "C_dev is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(BM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(BM_EINVAL, "device %d beyond the supported %d", dev, kMaxDevices);
    void* base = nullptr;
    {
        // Set-up, once per device and with that device current: find the
        // device address of the scratch array.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            e = cudaGetSymbolAddress(&g_scratch_addr[dev], bm_noalloc_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return err(BM_ECUDA, "cudaGetSymbolAddress of the scratch: %s", cudaGetErrorString(e));
            }
        }
        base = g_scratch_addr[dev];
    }
    bm::Globals* g = (bm::Globals*)base;
    float* Cp = (float*)((char*)base + kGlobalsBytes);
    cudaStream_t st = (cudaStream_t)stream;
    const float gB = std::nextafter(gamma_up(2 * np + 2) * (1.0f + 1e-6f), INFINITY);
    const float gp2 = std::nextafter((float)(2.0 * (1.0 + std::ldexp(1.0, -14)) * (double)gamma_up(np + 2)) *
                                         (1.0f + 1e-6f), INFINITY);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // The scratch keeps the previous call's contents: clear the accumulators.
    if ((e = cudaMemsetAsync(g, 0, sizeof(bm::Globals), st)) ||
        (e = bm::launch_pad(C_dev, k, n, np, Cp, st)) ||
        (e = bm::launch_prepass(X_dev, (long long)m * n, g, 2 * sms, st)) ||
        (e = bm::launch_prepass(C_dev, (long long)k * n, g, 1, st)) ||
        (e = bm::launch_fullpass(np, X_dev, m, n, Cp, k, nullptr, 1, labels_out_dev, g, gB, gp2, 0, sms, st)))
        return err(BM_ECUDA, "full pass launch: %s", cudaGetErrorString(e));
    bm::Globals h;
    if ((e = cudaMemcpyAsync(&h, g, sizeof h, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return err(BM_ECUDA, "full pass: %s", cudaGetErrorString(e));
    const bm_status fs = bm::status_from_flags(h);      // the same statuses as bm_assign
    if (fs != BM_OK) return fs;
    if (f_out_host) *f_out_host = h.f_full;
    return BM_OK;
}
