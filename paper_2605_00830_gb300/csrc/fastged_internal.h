// fastged_internal.h -- data layout shared by the sm_103a kernels and the host runtime.
//
// Device data of one batch (all resident in HBM):
//   GraphMeta table        one entry per graph
//   vlabel pool  int32     vertex labels, graph g at lab_off
//   edge pool    int32x2   raw edge list, graph g at edge_off (packed into bitsets on device)
//   elabel pool  int32     edge labels (absent when the batch is unlabelled)
//   adj pool     uint64    adjacency bitsets, graph g: n rows of W words, row-major [v][w]
//   plane pool   uint64    edge-label bit-planes, graph g: B planes of n x W words; bit u of
//                          row v of plane b is bit b of the label of edge (v, u)
//
// One team (a CTA) solves one pair at a time. Its working set is split into regions; the
// host planner puts each region in shared memory or in the team's slice of a global
// scratch buffer (the same kernel code addresses both through generic pointers).
#pragma once
#include <cstdint>

namespace fastged {

constexpr int kMaxWords = 16;       // 1024 vertices
constexpr int kHistMax = 32;        // PED histogram buckets (one per lane)
constexpr int kMaxB = 8;            // edge-label bit-planes (labels 0..255)
constexpr int kMaxWarps = 16;       // 512 threads per CTA
constexpr int kMaxClusterWarps = 256; // 16 CTAs of 512 threads

struct CostModel {
    int32_t vsub, vdel, vins, esub, edel, eins;
};

struct GraphMeta {
    int32_t n, m, W, pad;
    int64_t adj_off;     // uint64 words into the adj pool
    int64_t plane_off;   // uint64 words into the plane pool
    int64_t lab_off;     // int32 index into the vlabel pool
    int64_t edge_off;    // edge index into the edge / elabel pools
};

enum Region : int {
    RG_HIST = 0, RG_ALPHA2, RG_A2T, RG_L2T, RG_SBASE, RG_PED0, RG_PED1, RG_SEL, RG_SELPED,
    RG_KLIST, RG_KPED, RG_NOFF, RG_NBR, RG_IMG0, RG_IMG1, RG_P, RG_PL,
    RG_CAND, RG_MAP0, RG_MAP1, RG_IMGL, RG_CROW,
    RG_COUNT
};



struct Layout {
    int64_t off[RG_COUNT];     // byte offset inside shared memory or the global slice
    uint32_t smem_mask;        // bit r set: region r lives in shared memory
    int32_t kmax;              // slots per beam buffer
    int32_t kloc;              // node slots a CTA prepares (kmax, or its share of a cluster)
    int32_t n1max, n2max;      // largest graphs of the class
    int32_t n2s;               // row stride (elements) of the transposed g2 tables
    int32_t mrow;              // bytes per stored vertex map
    int32_t fs;                // successors per node at most (n2max + 1)
    int32_t word_bytes;        // 4 or 8: bytes per bitset word
    int32_t B;                 // edge-label planes
    int32_t pk;                // 1: successors packed as PED << 16 | slot << jbits | j
    int64_t smem_bytes;        // dynamic shared memory per CTA
    int64_t slice_bytes;       // global scratch bytes per team (CTA or cluster)
    int64_t team_off;          // cluster teams: offset of the team scalars in the slice
    // cluster teams: per-CTA tables that did not fit shared memory live in a block of the
    // slice per CTA (at cta_off + cluster rank * cta_bytes; their off[] is inside the block)
    uint32_t cta_mask;
    int64_t cta_off, cta_bytes;
    int64_t rsize[RG_COUNT];   // bytes of every region (bounds-checked builds check against it)
};

// One-warp teams (kbest_warp_kernel): every warp of a CTA solves its own pair in its own
// block of shared memory; the two vertex-map buffers are in that block too, or in the warp's
// block of global scratch (gmap). Offsets are in bytes from the start of the block.
enum WarpRegion : int {
    WR_TGT = 0,   // g2 records: adjacency word, label planes, cost-row entry (n2 + 2 of them)
    WR_LAB2,      // g2 vertex labels, int32[n2]
    WR_NOFF,      // g1 prior-neighbour list offsets, int32[n1 + 1]
    WR_NBR,       // g1 prior-neighbour lists, int32[m1]: k | edge label << 16
    WR_IMG0, WR_IMG1,     // Img bitset of every kept node, Word[K], two beam buffers
    WR_PED0, WR_PED1,     // PED of every kept node, int32[K]
    WR_E20, WR_E21,       // g2 edges with both ends in Img, uint16[K]
    WR_ENT,       // successor entries of a level in enumeration order, uint16[K * (n2 + 1)]
    WR_NODEOFF,   // first entry of every node, uint16[K + 1]
    WR_KLIST,     // kept successors, uint32[K]: PED offset << 16 | entry index
    WR_SEL,       // selected children in key order, int32[K]: parent slot << 8 | j (one-warp
                  // kernel: record index j, 1 + target vertex or n2 + 1 for the deletion)
    WR_SELPED,    // their PEDs, int32[K]
    WR_MAP0, WR_MAP1,     // vertex maps of the kept nodes, uint8[K][mrow]
    WR_COUNT
};

// bytes of one target record of the one-warp kernel: one bitset word for the adjacency, npl
// label planes and the 32-bit cost-row entry, padded to 16 bytes (vector loads)
constexpr int warp_rec_bytes(bool w32, int npl)
{
    return ((w32 ? 4 : 8) * (1 + npl) + 4 + 15) / 16 * 16;
}

struct WarpLayout {
    int32_t off[WR_COUNT];
    int32_t warp_bytes;   // shared memory per warp
    int32_t gmap;         // 1: WR_MAP0 / WR_MAP1 are offsets into the warp's global block
    int32_t gmap_bytes;   // bytes of that global block (0 when the maps are in shared memory)
    int32_t mrow;         // bytes per stored vertex map (a multiple of 16)
    int32_t size[WR_COUNT];   // bytes of every region (bounds-checked builds check against it)
};

struct KParams {
    // batch inputs
    const GraphMeta *gmeta;
    const uint64_t *adj;
    const uint64_t *planes;
    const int32_t *vlab;
    const int32_t *pairs;        // [2 * n_pairs]
    const int32_t *order;        // pair indices of this class, heaviest first
    int32_t n_order;
    const int32_t *kpp;          // per-pair K or nullptr
    int32_t K;                   // K when kpp == nullptr
    int32_t hwin;                // histogram window (2..kHistMax)
    int32_t variant;
    CostModel cost;
    // work queue and status
    int32_t *queue_head;
    int32_t *err;
    // outputs
    int32_t *out_cost;
    int32_t *out_map;
    const int64_t *map_off;      // [n_pairs] offset of each pair's map in out_map
    int64_t *out_nevals;         // may be nullptr
    // scratch
    uint8_t *gscratch;
    Layout lay;
    WarpLayout wl;               // one-warp teams only
    // per-phase cycle counters; profiling builds only (nullptr otherwise)
    unsigned long long *phase_cycles;
    // element counts of the batch arrays (bounds-checked builds check every index against them)
    int64_t n_graphs, n_pairs, n_vlab, adj_words, plane_words, map_total;
};

struct PackParams {
    const GraphMeta *gmeta;
    int32_t n_graphs;
    const int32_t *edges;
    const int32_t *elabel;       // nullptr: unlabelled
    int32_t B;
    uint64_t *adj;
    uint64_t *planes;
    int32_t *err;
};

// error bits written by kernels into *err
constexpr int32_t kErrDuplicateEdge = 1;
// bounds-checked builds (FASTGED_BOUNDS_CHECK): an index left its array; err[2] holds the
// source line of the first such access (the access itself went to the array's element 0)
constexpr int32_t kErrBounds = 4;

#ifdef FASTGED_BOUNDS_CHECK
__device__ __forceinline__ int64_t fg_bound(int64_t i, int64_t n, int line, int32_t *err)
{
    if (i >= 0 && i < n) return i;
    atomicOr(err, kErrBounds);
    atomicCAS(err + 2, 0, line);
    return 0;
}
// element i of array a that holds n elements (n counted in elements)
#define FG_AT(a, i, n) ((a)[fg_bound((int64_t)(i), (int64_t)(n), __LINE__, p.err)])
#else
#define FG_AT(a, i, n) ((a)[(i)])
#endif
// elements of type T in a region of `bytes` bytes
#define FG_N(T, bytes) ((int64_t)(bytes) / (int64_t)sizeof(T))

}  // namespace fastged
