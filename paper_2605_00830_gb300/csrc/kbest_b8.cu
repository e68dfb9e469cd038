// kbest_b8.cu -- K-Best kernel instances for up to eight edge-label bit-planes.
#include "kbest_warp.cuh"

namespace fastged {
template cudaError_t launch_kbest_bk<8>(int, bool, bool, bool, const KParams &, int, int,
                                          size_t, cudaStream_t);
template cudaError_t kbest_occupancy_bk<8>(int, bool, bool, bool, int, size_t, int *);
template cudaError_t launch_kbest_cluster_bk<8>(int, bool, const KParams &, int, int, size_t, int,
                                                  cudaStream_t);
template cudaError_t kbest_cluster_occupancy_bk<8>(int, bool, int, size_t, int, int *);
template cudaError_t launch_kbest_warp_bk<8>(bool, const KParams &, int, int, size_t,
                                              cudaStream_t);
template cudaError_t kbest_warp_occupancy_bk<8>(bool, int, size_t, int *);
}  // namespace fastged
