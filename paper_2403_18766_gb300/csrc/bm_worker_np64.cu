// Worker kernel instantiated for padded width NP = 64.
#include "bm_worker_impl.cuh"

namespace bm {
template cudaError_t launch_worker_t<64>(const WorkerArgs&, int, cudaStream_t);
template int worker_max_cluster_t<64>(int);
template int worker_active_clusters_t<64>(int, size_t);
}  // namespace bm
