// Dispatch of the fused worker kernel over the padded width NP.
#include "bm_worker.cuh"

namespace bm {

template <int NP>
cudaError_t launch_worker_t(const WorkerArgs& a, int clusters, cudaStream_t st);
template <int NP>
int worker_max_cluster_t(int k);
template <int NP>
int worker_active_clusters_t(int cs, size_t smem);

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
