// kbest_kernels.cu -- the S0 packing kernel and the host-side dispatch onto the K-Best
// kernel instances.
//
//   pack_kernel   S0: edge lists -> adjacency bitsets and edge-label bit-planes
//   launch_kbest / kbest_occupancy / launch_kbest_cluster / kbest_cluster_occupancy /
//   launch_kbest_warp / kbest_warp_occupancy:
//                 pick the instance (words per bitset, map entry width, all-shared-memory or
//                 not, label planes) of the S1-S5 kernels in kbest_impl.cuh (one-CTA and
//                 cluster teams) and kbest_warp.cuh (one-warp teams), which are compiled in
//                 kbest_b0.cu, kbest_b2.cu and kbest_b8.cu.
//
// Method: Algorithm 1 of Dabah & Herten (branching Sec. 4.1.1, evaluation Sec. 4.1.2 and
// Algorithm 2, selection Sec. 4.2, leaf insertions Sec. 4.4); kbest_impl.cuh states how the
// implied edge costs are computed from bitsets.
#include "kbest_warp.cuh"

namespace fastged {

// ------------------------------------------------------------------------------------
// S0: pack edge lists into bitsets (one warp per graph, lanes over its edges).
// ------------------------------------------------------------------------------------
__global__ void pack_kernel(const PackParams pp)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g < pp.n_graphs; g += nwarps) {
        const GraphMeta mt = pp.gmeta[g];
        uint64_t *A = pp.adj + mt.adj_off;
        for (int k = lane; k < mt.m; k += 32) {
            const int64_t e = mt.edge_off + k;
            const int u = pp.edges[2 * e], v = pp.edges[2 * e + 1];
            const unsigned long long bu = 1ull << (u & 63), bv = 1ull << (v & 63);
            const unsigned long long old =
                atomicOr((unsigned long long *)&A[(int64_t)u * mt.W + (v >> 6)], bv);
            if (old & bv) atomicOr(pp.err, kErrDuplicateEdge);
            atomicOr((unsigned long long *)&A[(int64_t)v * mt.W + (u >> 6)], bu);
            if (pp.elabel) {
                const int lab = pp.elabel[e];
                for (int b = 0; b < pp.B; ++b) {
                    if (!((lab >> b) & 1)) continue;
                    uint64_t *Pl = pp.planes + mt.plane_off + (int64_t)b * mt.n * mt.W;
                    atomicOr((unsigned long long *)&Pl[(int64_t)u * mt.W + (v >> 6)], bv);
                    atomicOr((unsigned long long *)&Pl[(int64_t)v * mt.W + (u >> 6)], bu);
                }
            }
        }
    }
}


bool kbest_has_smem_variant(int W, bool wide, bool w32) { return w32 || (W <= 4 && !wide); }

// the K-Best instances are compiled in kbest_b0.cu, kbest_b2.cu and kbest_b8.cu (one
// translation unit per label-plane count, built in parallel); none are instantiated here
#define FASTGED_EXTERN_BK(BK)                                                                  \
    extern template cudaError_t launch_kbest_bk<BK>(int, bool, bool, bool, const KParams &, int, \
                                                    int, size_t, cudaStream_t);                \
    extern template cudaError_t kbest_occupancy_bk<BK>(int, bool, bool, bool, int, size_t,      \
                                                       int *);                                 \
    extern template cudaError_t launch_kbest_cluster_bk<BK>(int, bool, const KParams &, int, int, \
                                                            size_t, int, cudaStream_t);        \
    extern template cudaError_t kbest_cluster_occupancy_bk<BK>(int, bool, int, size_t, int, int *); \
    extern template cudaError_t launch_kbest_warp_bk<BK>(bool, const KParams &, int, int,       \
                                                         size_t, cudaStream_t);                \
    extern template cudaError_t kbest_warp_occupancy_bk<BK>(bool, int, size_t, int *);
FASTGED_EXTERN_BK(0)
FASTGED_EXTERN_BK(2)
FASTGED_EXTERN_BK(8)
#undef FASTGED_EXTERN_BK

// bk: edge-label planes of the instance (0, 2 or 8; see solve_pair)
cudaError_t launch_kbest(int W, bool wide_map, bool w32, bool sm, int bk, const KParams &p,
                         int grid, int block, size_t smem, cudaStream_t st)
{
    if (bk == 0) return launch_kbest_bk<0>(W, wide_map, w32, sm, p, grid, block, smem, st);
    if (bk == 2) return launch_kbest_bk<2>(W, wide_map, w32, sm, p, grid, block, smem, st);
    return launch_kbest_bk<8>(W, wide_map, w32, sm, p, grid, block, smem, st);
}

cudaError_t kbest_occupancy(int W, bool wide_map, bool w32, bool sm, int bk, int block,
                            size_t smem, int *out)
{
    if (bk == 0) return kbest_occupancy_bk<0>(W, wide_map, w32, sm, block, smem, out);
    if (bk == 2) return kbest_occupancy_bk<2>(W, wide_map, w32, sm, block, smem, out);
    return kbest_occupancy_bk<8>(W, wide_map, w32, sm, block, smem, out);
}

template <int BK>
cudaError_t launch_kbest_cluster_bk(int W, bool wide, const KParams &p, int grid, int block, size_t smem,
                                    int cluster, cudaStream_t st);
template <int BK>
cudaError_t kbest_cluster_occupancy_bk(int W, bool wide, int block, size_t smem, int cluster, int *out);

bool kbest_has_cluster_variant(int W, bool wide, bool w32)
{
    return !w32 && ((wide && W >= 4) || ((W == 2 || W == 4) && !wide));
}

cudaError_t launch_kbest_cluster(int W, bool wide, int bk, const KParams &p, int grid, int block,
                                 size_t smem, int cluster, cudaStream_t st)
{
    if (bk == 0) return launch_kbest_cluster_bk<0>(W, wide, p, grid, block, smem, cluster, st);
    if (bk == 2) return launch_kbest_cluster_bk<2>(W, wide, p, grid, block, smem, cluster, st);
    return launch_kbest_cluster_bk<8>(W, wide, p, grid, block, smem, cluster, st);
}

cudaError_t kbest_cluster_occupancy(int W, bool wide, int bk, int block, size_t smem, int cluster,
                                    int *out)
{
    if (bk == 0) return kbest_cluster_occupancy_bk<0>(W, wide, block, smem, cluster, out);
    if (bk == 2) return kbest_cluster_occupancy_bk<2>(W, wide, block, smem, cluster, out);
    return kbest_cluster_occupancy_bk<8>(W, wide, block, smem, cluster, out);
}

// one-warp teams (kbest_warp.cuh): w32 = one 32-bit bitset word, else one 64-bit word
cudaError_t launch_kbest_warp(bool w32, int bk, const KParams &p, int grid, int block,
                              size_t smem, cudaStream_t st)
{
    if (bk == 0) return launch_kbest_warp_bk<0>(w32, p, grid, block, smem, st);
    if (bk == 2) return launch_kbest_warp_bk<2>(w32, p, grid, block, smem, st);
    return launch_kbest_warp_bk<8>(w32, p, grid, block, smem, st);
}

cudaError_t kbest_warp_occupancy(bool w32, int bk, int block, size_t smem, int *out)
{
    if (bk == 0) return kbest_warp_occupancy_bk<0>(w32, block, smem, out);
    if (bk == 2) return kbest_warp_occupancy_bk<2>(w32, block, smem, out);
    return kbest_warp_occupancy_bk<8>(w32, block, smem, out);
}

cudaError_t launch_pack(const PackParams &pp, int n_graphs, cudaStream_t st)
{
    const int block = 256;
    int grid = (n_graphs * 32 + block - 1) / block;
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    pack_kernel<<<grid, block, 0, st>>>(pp);
    return cudaGetLastError();
}

// upper bound of the kernels' static shared memory (the team's scalars)
size_t team_shared_static_bytes() { return sizeof(TeamShared) + 256; }
size_t team_shared_cluster_bytes() { return sizeof(TeamSharedCl); }

}  // namespace fastged
