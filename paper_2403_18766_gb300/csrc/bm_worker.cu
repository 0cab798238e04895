// Dispatch of the fused worker kernel over the padded width NP.
#include <map>
#include <mutex>

#include <cooperative_groups.h>

#include "bm_worker.cuh"

namespace bm {

template <int NP>
cudaError_t launch_worker_t(const WorkerArgs& a, int clusters, cudaStream_t st);
template <int NP>
int worker_max_cluster_t(int k);
template <int NP>
int worker_active_clusters_t(int cs, size_t smem);

// Whether a cooperative launch keeps its cluster shape on this device and in
// this process (a launch of 2 clusters of 2 CTAs that report what they see).
// Checked once per device: some tools that intercept launches were seen to
// drop the cluster dimension of cooperative launches.  The probe's name
// starts like the worker kernel's, so that a profiler told to intercept the
// worker kernel by name intercepts the probe as well.
__global__ void worker_kernel_launch_probe(int* out) {
    if (threadIdx.x == 0) atomicAdd(out, (int)cg::this_cluster().num_blocks());
}
bool cooperative_clusters_ok() {
    static std::mutex mu;
    static std::map<int, bool> memo;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    std::lock_guard<std::mutex> lk(mu);
    const auto it = memo.find(dev);
    if (it != memo.end()) return it->second;
    bool ok = false;
    int* d = nullptr;
    int h = 0;
    if (cudaMalloc(&d, sizeof(int)) == cudaSuccess && cudaMemset(d, 0, sizeof(int)) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(4, 1, 1);
        cfg.blockDim = dim3(32, 1, 1);
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeCooperative;
        attr[1].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        if (cudaLaunchKernelEx(&cfg, worker_kernel_launch_probe, d) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
            cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
            ok = (h == 8);                               // 4 CTAs, each in a cluster of 2
    }
    if (d) cudaFree(d);
    cudaGetLastError();
    memo[dev] = ok;
    return ok;
}

int worker_active_clusters(int np, int cs, size_t smem) {
    switch (np) {
        case 4: return worker_active_clusters_t<4>(cs, smem);
        case 8: return worker_active_clusters_t<8>(cs, smem);
        case 16: return worker_active_clusters_t<16>(cs, smem);
        case 32: return worker_active_clusters_t<32>(cs, smem);
        case 64: return worker_active_clusters_t<64>(cs, smem);
    }
    return 0;
}

int worker_max_cluster(int np, int k) {
    switch (np) {
        case 4: return worker_max_cluster_t<4>(k);
        case 8: return worker_max_cluster_t<8>(k);
        case 16: return worker_max_cluster_t<16>(k);
        case 32: return worker_max_cluster_t<32>(k);
        case 64: return worker_max_cluster_t<64>(k);
    }
    return 8;
}

size_t worker_smem(int np, int k) {
    switch (np) {
        case 4: return worker_smem_bytes<4>(k);
        case 8: return worker_smem_bytes<8>(k);
        case 16: return worker_smem_bytes<16>(k);
        case 32: return worker_smem_bytes<32>(k);
        case 64: return worker_smem_bytes<64>(k);
    }
    return 0;
}

cudaError_t launch_worker(int np, const WorkerArgs& a, int clusters, cudaStream_t st) {
    switch (np) {
        case 4: return launch_worker_t<4>(a, clusters, st);
        case 8: return launch_worker_t<8>(a, clusters, st);
        case 16: return launch_worker_t<16>(a, clusters, st);
        case 32: return launch_worker_t<32>(a, clusters, st);
        case 64: return launch_worker_t<64>(a, clusters, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bm
