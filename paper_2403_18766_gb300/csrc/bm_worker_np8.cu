// Worker kernel instantiated for padded width NP = 8.
#include "bm_worker_impl.cuh"

namespace bm {
template cudaError_t launch_worker_t<8>(const WorkerArgs&, int, cudaStream_t);
template int worker_max_cluster_t<8>(int);
template int worker_active_clusters_t<8>(int, size_t);
}  // namespace bm
