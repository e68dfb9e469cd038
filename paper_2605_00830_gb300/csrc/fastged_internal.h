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
    // per-phase cycle counters; profiling builds only (nullptr otherwise)
    unsigned long long *phase_cycles;
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

}  // namespace fastged
