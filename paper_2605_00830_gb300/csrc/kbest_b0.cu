// kbest_b0.cu -- K-Best kernel instances for unlabelled edges.
#include "kbest_warp.cuh"

namespace fastged {
template cudaError_t launch_kbest_bk<0>(int, bool, bool, bool, const KParams &, int, int,
                                          size_t, cudaStream_t);
template cudaError_t kbest_occupancy_bk<0>(int, bool, bool, bool, int, size_t, int *);
template cudaError_t launch_kbest_cluster_bk<0>(int, bool, const KParams &, int, int, size_t, int,
                                                  cudaStream_t);
template cudaError_t kbest_cluster_occupancy_bk<0>(int, bool, int, size_t, int, int *);
template cudaError_t launch_kbest_warp_bk<0>(bool, const KParams &, int, int, size_t,
                                              cudaStream_t);
template cudaError_t kbest_warp_occupancy_bk<0>(bool, int, size_t, int *);
}  // namespace fastged
