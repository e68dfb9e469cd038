// fastged_runtime.h -- host-side objects behind the opaque handles of include/fastged.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fastged.h"
#include "fastged_internal.h"

namespace fastged {

constexpr int kMaxClasses = 16;

// Grow-only device buffer. Growth is stream-ordered on the owner's stream (it waits for that
// stream only, never for the whole device); with headroom = true it takes half again the
// old capacity as well (rounded to 1 MiB), so that a handle serving batches of growing size
// re-allocates rarely.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t n, cudaStream_t st, bool headroom);   // returns a fastged status
    void release();
};

// Grow-only pinned host buffer (the same headroom rule).
struct PinBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t n, bool headroom);
    void release();
};

// One size class: pairs whose g2 bitsets need W words and whose stored vertex-map entries
// are 8 (wide = false) or 16 bits wide.
struct ClassPlan {
    int W = 1;
    bool wide = false;
    bool w32 = false;             // one 32-bit word per bitset (every g2 has <= 32 vertices)
    bool pk = false;              // successors packed into one 32-bit entry (see packable)
    bool all_smem = false;        // every region of a team fits in shared memory
    int cluster = 1;              // CTAs per team (> 1: a thread-block cluster per pair)
    bool warp = false;            // one warp per pair (kbest_warp_kernel; W == 1, small K)
    WarpLayout wl{};              // layout of one warp's working set (warp classes)
    int n1max = 0, n2max = 0, m1max = 0, kmax = 1;
    std::vector<int32_t> order;   // pair indices, heaviest first
    int64_t order_off = 0;        // offset of this class's order in the device order array
    Layout lay{};
    int block = 256;
    int grid = 1;
    size_t smem = 0;
    size_t scratch_off = 0;       // offset of this class's scratch in the scratch area
};

// A validated, flattened batch: staging offsets (input region) and device work offsets.
struct Batch {
    int n_graphs = 0, n_pairs = 0, K = 1, B = 0;
    bool labelled = false;
    bool has_kpp = false;
    fastged_options opt{};
    std::vector<GraphMeta> meta;
    std::vector<int64_t> map_off;
    // FASTGED_ORDER_DEGREE: for map entry map_off[p] + k, the source vertex branched at level
    // k (empty in index order)
    std::vector<int32_t> perm;
    int64_t n_vlab = 0, n_edges = 0, adj_words = 0, plane_words = 0, map_total = 0;
    std::vector<ClassPlan> classes;
    // input region (pinned staging == device input buffer)
    size_t off_meta = 0, off_vlab = 0, off_edges = 0, off_elab = 0, off_pairs = 0,
           off_order = 0, off_mapoff = 0, off_kpp = 0, in_bytes = 0;
    // work region
    size_t woff_err = 0, woff_cost = 0, woff_nev = 0, woff_map = 0, out_bytes = 0,
           woff_queue = 0, woff_pool = 0, woff_scratch = 0, work_bytes = 0;
};

int set_error(int code, const std::string &msg);
int set_error(int code, const char *msg);
// splits a team's working set into shared-memory and global-scratch regions (budget bytes of
// shared memory, filled in order of access frequency)
void plan_layout(ClassPlan &cp, int B, int block, size_t budget);
// lays out one warp's working set for a one-warp class; gmap puts the vertex maps in global
// scratch. Returns the shared-memory bytes per warp.
size_t plan_warp_layout(ClassPlan &cp, int B, bool gmap);
// one-warp teams: largest K, largest source graph, and largest target graph (of the 64-bit and
// of the 32-bit word instance): a node's successors are a bitset of its free target vertices
// with the deletion as the bit after the last vertex
constexpr int kWarpMaxK = 128;
constexpr int kWarpMaxN = 64;
constexpr int kWarpMaxN2 = 63;
constexpr int kWarpMaxN2Word32 = 31;
// default histogram window of the one-warp kernel: sixteen 4-bit counters per lane, of which
// offsets 0-14 from the anchor decide the threshold
constexpr int kWarpHist = 16;
// kernel instance serving B edge-label planes (0, 2 or 8)
int label_instance(int B);
// One-shot host-side fault injection (fastged_inject_fault): true when the armed fault of
// this kind fires now.
bool inject_fire(int kind);
// An NVTX range for timeline tools (Nsight Systems); free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
// Packed classes store a successor as PED << 16 | parent slot << jbits | j with
// jbits = bit length of n2 (j runs over 0..n2): a pair may be packed only if no PED reaches
// 2^16 and its K fits the remaining 16 - jbits bits. The single-word kernels are always
// packed; a single-word pair that is not packable is solved by the two-word kernels.
inline int jbits_of(int n2)
{
    int b = 0;
    while (b < 31 && (1 << b) <= n2) ++b;
    return b;
}
inline bool packable(long long ped_bound, long long k, int n2)
{
    const int jb = jbits_of(n2);
    return ped_bound < 65536 && jb <= 16 && k <= (1LL << (16 - jb));
}
void clear_error();
int flatten(fastged_handle *h, const fastged_pair_list *pl, int32_t K,
            const fastged_options &opt, Batch &b);
int enqueue(fastged_handle *h, const Batch &b, uint8_t *in, uint8_t *wk, cudaStream_t st,
            int *launches, cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr,
            bool capturing = false);
int finish_outputs(const Batch &b, const uint8_t *host_out, int32_t *out_cost,
                   int32_t *out_mapping, int64_t *out_nevals);
// asynchronous halves of fastged_batch_ex: enqueue everything (flatten, upload, kernels,
// download into the handle's staging buffer) on h->stream; after the stream has finished,
// copy the results out of the staging buffer
int batch_enqueue(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                  const fastged_options &o);
int batch_results(fastged_handle *h, int32_t *out_cost, int32_t *out_mapping,
                  int64_t *out_nevals);
fastged_options default_options();

}  // namespace fastged

struct fastged_handle {
    fastged_cost_model cost{};
    int device = 0;
    int sm_count = 1;
    int smem_optin = 48 * 1024;
    int smem_per_sm = 100 * 1024;
    cudaStream_t stream = nullptr;
    cudaStream_t class_stream[fastged::kMaxClasses] = {};
    cudaEvent_t ev[fastged::kMaxClasses + 1] = {};
    fastged::DevBuf dev_in, dev_work;
    fastged::PinBuf pin;
    fastged::Batch batch;
    int32_t timeout_ms = 0;         // 0: fastged_batch_ex waits without a bound
    bool inflight = false;          // a timed-out batch may still be running on `stream`
    cudaEvent_t done = nullptr;     // recorded after a batch, polled under a timeout
};

struct fastged_plan {
    fastged_handle *h = nullptr;
    fastged::Batch b;
    fastged::DevBuf dev_in, dev_work;
    fastged::PinBuf pin_out;
    cudaStream_t stream = nullptr;
    cudaStream_t last_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    int launches = 0;
    cudaEvent_t t0 = nullptr, t1 = nullptr;   // bracket the K-Best launches of a run
};
