// noalloc.cu -- a K-Best batch entry point that allocates no memory.
//
// Some callers cannot allocate device memory: code embedded in a host application that owns
// every device allocation through its own pool, plugins that are handed a fixed device budget,
// or runtimes where a cudaMalloc at an arbitrary point is forbidden. fastged_batch_noalloc
// serves them: the caller passes device inputs and device outputs, and every piece of scratch
// the path needs (graph table, work queue, status word, bitset pools, per-team working sets)
// lives in one file-scope __device__ array of FASTGED_NOALLOC_SCRATCH_BYTES. The array is part
// of the loaded module, so every GPU that loads the library holds it until the process exits.
//
// Host code may not use the array's name as a device address (it is a host-side stand-in).
// The first call on a device, with that device current, resolves the real address with
// cudaGetSymbolAddress; later calls reuse it while the device's context is the same one (a
// new context, after cudaDeviceReset for instance, may load the module elsewhere, so the
// address is resolved again).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/fastged.h"
#include "fastged_internal.h"
#include "fastged_runtime.h"

namespace fastged {
cudaError_t launch_kbest(int W, bool wide_map, bool w32, bool sm, int bk, const KParams &p,
                         int grid, int block, size_t smem, cudaStream_t st);
cudaError_t kbest_occupancy(int W, bool wide_map, bool w32, bool sm, int bk, int block,
                            size_t smem, int *out);
bool kbest_has_smem_variant(int W, bool wide, bool w32);
cudaError_t launch_pack(const PackParams &pp, int n_graphs, cudaStream_t st);
size_t team_shared_static_bytes();

static __device__ __align__(256) unsigned char g_noalloc_scratch[FASTGED_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, with the id of the context it was resolved
// in (0: not yet).
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    unsigned long long ctx = 0;
    void *addr = nullptr;
};
static ScratchAddr g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Id of the calling thread's current context (unique over the process's lifetime), from the
// driver entry points; 0 when it cannot be read (the address is then resolved on every call).
static unsigned long long current_context_id()
{
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (GetIdFn)f;
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c ||
        get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Bit-set row of every graph: an exclusive prefix sum of the vertex counts (one block, the
// graphs in chunks of its size), so graphs whose label ranges overlap still get rows of
// their own. Negative counts count as 0 here (noalloc_prepare rejects them).
__global__ void noalloc_rows(const int32_t *graph_n, int n_graphs, int64_t *row)
{
    __shared__ int64_t part[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int g0 = 0; g0 < n_graphs; g0 += blockDim.x) {
        const int g = g0 + (int)threadIdx.x;
        const int64_t v = g < n_graphs ? (int64_t)max(graph_n[g], 0) : 0;
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) part[wid] = incl;
        __syncthreads();
        int64_t before = carry;
        for (int w = 0; w < wid; ++w) before += part[w];
        if (g < n_graphs) row[g] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t t = 0;
            for (int w = 0; w < nw; ++w) t += part[w];
            carry += t;
        }
        __syncthreads();
    }
}

// Builds the graph table (graph g gets Wg-word bit-set rows from row[g]), the identity pair
// order, and validates what the packing and K-Best kernels rely on before any of them runs:
// vertex and edge counts, label and edge ranges, bit-set rows within total_vertices, edge
// endpoints, edge labels, pair indices and map ranges. Any violation sets bit kErrInvalid of
// *err (and the edges of a graph whose ranges are invalid are not read).
constexpr int32_t kErrInvalid = 2;

__global__ void noalloc_prepare(const fastged_device_batch b, int Wg, int B, int max_m,
                                const int64_t *row, GraphMeta *meta, int32_t *order,
                                int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g < b.n_graphs; g += nwarps) {
        const int n = b.graph_n[g], m = b.graph_m[g];
        const int64_t lo = b.vlabel_off[g], eo = b.edge_off[g], r = row[g];
        const bool ok = n >= 0 && n <= b.max_n && m >= 0 && m <= max_m && lo >= 0 && eo >= 0 &&
                        lo + n <= b.total_vertices && eo + m <= b.total_edges &&
                        r + n <= b.total_vertices;
        if (lane == 0) {
            GraphMeta mt;
            mt.n = n;
            mt.m = m;
            mt.W = Wg;
            mt.pad = 0;
            mt.adj_off = r * Wg;
            mt.plane_off = r * Wg * B;
            mt.lab_off = lo;
            mt.edge_off = eo;
            meta[g] = mt;
            if (!ok) atomicOr(err, kErrInvalid);
        }
        if (!ok) continue;
        for (int k = lane; k < m; k += 32) {
            const int u = b.edges[2 * (eo + k)], v = b.edges[2 * (eo + k) + 1];
            const int lab = b.elabel ? b.elabel[eo + k] : 0;
            if (u < 0 || v < 0 || u >= n || v >= n || u == v || lab < 0 || lab > b.max_elabel)
                atomicOr(err, kErrInvalid);
        }
    }
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = t; p < b.n_pairs; p += gridDim.x * blockDim.x) {
        order[p] = p;
        const int a = b.pairs[2 * p], d = b.pairs[2 * p + 1];
        if (a < 0 || d < 0 || a >= b.n_graphs || d >= b.n_graphs) {
            atomicOr(err, kErrInvalid);
            continue;
        }
        const int64_t mo = b.map_off[p];
        if (mo < 0 || mo + max(b.graph_n[a], 0) > b.map_len) atomicOr(err, kErrInvalid);
    }
}

}  // namespace fastged

using namespace fastged;

static size_t na_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

extern "C" int fastged_batch_noalloc(const fastged_cost_model *cost,
                                     const fastged_device_batch *b, int32_t K,
                                     int32_t *out_cost, int32_t *out_mapping,
                                     int64_t *out_nevals, void *stream)
{
    clear_error();
    if (!cost || !b || !out_cost || !out_mapping)
        return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    const int32_t *cv = &cost->v_sub;
    for (int k = 0; k < 6; ++k)
        if (cv[k] < 0) return set_error(FASTGED_ERR_INVALID_ARG, "negative cost");
    if (K < 1 || K > FASTGED_MAX_K) return set_error(FASTGED_ERR_INVALID_ARG, "K out of range");
    if (b->n_graphs < 0 || b->n_pairs < 0 || b->max_n < 1 || b->max_n > FASTGED_MAX_N ||
        b->max_m < 0 || (int64_t)b->max_m > (int64_t)b->max_n * (b->max_n - 1) / 2 ||
        b->max_elabel < 0 || b->max_elabel > FASTGED_MAX_ELABEL || b->total_vertices < 0 ||
        b->total_edges < 0 || b->map_len < 0)
        return set_error(FASTGED_ERR_INVALID_ARG, "batch limits out of range");
    if (b->n_pairs == 0) return FASTGED_OK;
    if (!b->graph_n || !b->graph_m || !b->vlabel_off || !b->edge_off || !b->pairs ||
        !b->map_off || (b->total_vertices > 0 && !b->vlabel) || (b->total_edges > 0 && !b->edges))
        return set_error(FASTGED_ERR_INVALID_ARG, "null device array");
    {
        const long long n = b->max_n, m = b->max_m;
        const long long bound = n * std::max(cost->v_sub, cost->v_del) + n * cost->v_ins +
                                m * std::max(cost->e_sub, cost->e_del) + m * cost->e_ins;
        if (bound >= (long long)INT32_MAX)
            return set_error(FASTGED_ERR_INVALID_ARG, "costs can overflow int32");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(FASTGED_ERR_CUDA, "no usable current device");
    uint8_t *base = nullptr;
    {
        const unsigned long long ctx = current_context_id();
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        ScratchAddr &sa = g_scratch_addr[dev];
        if (ctx == 0 || sa.ctx != ctx || !sa.addr) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                char msg[160];
                snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return set_error(FASTGED_ERR_CUDA, msg);
            }
            sa.addr = ptr;
            sa.ctx = ctx;
        }
        base = (uint8_t *)sa.addr;
    }
    cudaStream_t st = (cudaStream_t)stream;

    // one size class covering every graph of the batch
    int B = 0;
    while ((1 << B) <= b->max_elabel) ++B;
    if (B == 1) B = 2;   // served by the two-plane kernel (second plane all zero)
    const int Wg = (b->max_n + 63) / 64;
    ClassPlan cp;
    cp.W = Wg <= 1 ? 1 : Wg <= 2 ? 2 : Wg <= 4 ? 4 : Wg <= 8 ? 8 : 16;
    const long long ped_bound =
        (long long)b->max_n * std::max(cost->v_sub, cost->v_del) +
        (long long)b->max_m * (std::max(cost->e_sub, cost->e_del) + cost->e_ins);
    cp.pk = packable(ped_bound, K, b->max_n);
    if (cp.W == 1 && !cp.pk) cp.W = 2;
    cp.w32 = cp.W == 1 && b->max_n <= 32;
    cp.wide = b->max_n >= 255 || cp.W >= 8;
    cp.n1max = b->max_n;
    cp.n2max = b->max_n;
    cp.m1max = b->max_m;
    cp.kmax = K;
    const int block = K <= 32 ? 128 : 256;
    int smem_per_sm = 0, optin = 0, sms = 0;
    cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t stat = team_shared_static_bytes() + 1024;
    const size_t max_dyn = (size_t)optin - team_shared_static_bytes();
    plan_layout(cp, B, block, (size_t)1 << 40);
    const size_t total = (size_t)cp.lay.smem_bytes;
    size_t budget = (total + stat <= (size_t)smem_per_sm / 2 && total <= max_dyn)
                        ? total
                        : std::min(max_dyn, (size_t)smem_per_sm / 2 - stat);
    plan_layout(cp, B, block, budget);
    cp.all_smem = cp.lay.slice_bytes == 0 && kbest_has_smem_variant(cp.W, cp.wide, cp.w32);
    int occ = 0;
    cudaError_t e = kbest_occupancy(cp.W, cp.wide, cp.w32, cp.all_smem, label_instance(B), block,
                                    (size_t)cp.lay.smem_bytes, &occ);
    if (e != cudaSuccess || occ < 1)
        return set_error(FASTGED_ERR_CUDA, "team does not fit on an SM");

    // carve the scratch array: status | graph table | bit-set rows | pair order | bitset
    // pools | teams
    const size_t off_status = 0;
    const size_t off_meta = 256;
    const size_t off_row = na_align(off_meta + sizeof(GraphMeta) * (size_t)b->n_graphs, 256);
    const size_t off_order = na_align(off_row + 8 * (size_t)b->n_graphs, 256);
    const size_t off_pool = na_align(off_order + 4 * (size_t)b->n_pairs, 256);
    const size_t adj_words = (size_t)b->total_vertices * (size_t)Wg;
    const size_t pool_bytes = 8 * adj_words * (size_t)(1 + B);
    const size_t off_teams = na_align(off_pool + pool_bytes, 256);
    if (off_teams > FASTGED_NOALLOC_SCRATCH_BYTES)
        return set_error(FASTGED_ERR_INVALID_ARG,
                         "batch does not fit the fastged_batch_noalloc scratch array");
    int64_t grid = (int64_t)sms * occ;
    grid = std::min<int64_t>(grid, b->n_pairs);
    if (cp.lay.slice_bytes > 0)
        grid = std::min<int64_t>(grid, (int64_t)((FASTGED_NOALLOC_SCRATCH_BYTES - off_teams) /
                                                 (size_t)cp.lay.slice_bytes));
    if (grid < 1)
        return set_error(FASTGED_ERR_INVALID_ARG,
                         "one team's working set does not fit the fastged_batch_noalloc scratch");

    int32_t *status = (int32_t *)(base + off_status);   // [0] error bits, [1] queue head
    GraphMeta *meta = (GraphMeta *)(base + off_meta);
    int64_t *row = (int64_t *)(base + off_row);
    int32_t *order = (int32_t *)(base + off_order);
    uint64_t *pool = (uint64_t *)(base + off_pool);

#define NA_CK(call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            char msg_[200];                                                                 \
            snprintf(msg_, sizeof(msg_), "%s: %s", #call, cudaGetErrorString(e_));          \
            return set_error(FASTGED_ERR_CUDA, msg_);                                       \
        }                                                                                   \
    } while (0)

    // validate and build the tables, then check before any kernel trusts the edges
    int32_t host_err = 0;
    NA_CK(cudaMemsetAsync(status, 0, 256, st));
    {
        const int pblock = 256;
        int pgrid = (int)std::min<int64_t>(4096, ((int64_t)std::max(b->n_graphs, b->n_pairs) * 32 +
                                                  pblock - 1) / pblock);
        pgrid = std::max(pgrid, 1);
        if (b->n_graphs > 0) {
            noalloc_rows<<<1, 1024, 0, st>>>(b->graph_n, b->n_graphs, row);
            NA_CK(cudaGetLastError());
        }
        noalloc_prepare<<<pgrid, pblock, 0, st>>>(*b, Wg, B, b->max_m, row, meta, order, status);
        NA_CK(cudaGetLastError());
    }
    NA_CK(cudaMemcpyAsync(&host_err, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (host_err) return set_error(FASTGED_ERR_INVALID_ARG, "invalid graph, edge, label or pair index");

    // bitset pools start at zero; pack (S0), then the K-Best teams (S1-S5)
    if (pool_bytes) NA_CK(cudaMemsetAsync(pool, 0, pool_bytes, st));
    PackParams pp;
    pp.gmeta = meta;
    pp.n_graphs = b->n_graphs;
    pp.edges = b->edges;
    pp.elabel = b->elabel;
    pp.B = B;
    pp.adj = pool;
    pp.planes = pool + adj_words;
    pp.err = status;
    if (b->n_graphs > 0) NA_CK(launch_pack(pp, b->n_graphs, st));

    KParams p;
    memset(&p, 0, sizeof(p));
    p.gmeta = meta;
    p.adj = pool;
    p.planes = pool + adj_words;
    p.vlab = b->vlabel;
    p.pairs = b->pairs;
    p.order = order;
    p.n_order = b->n_pairs;
    p.kpp = nullptr;
    p.K = K;
    p.hwin = kHistMax;
    p.variant = 0;
    p.cost.vsub = cost->v_sub;
    p.cost.vdel = cost->v_del;
    p.cost.vins = cost->v_ins;
    p.cost.esub = cost->e_sub;
    p.cost.edel = cost->e_del;
    p.cost.eins = cost->e_ins;
    p.queue_head = status + 1;
    p.err = status;
    p.out_cost = out_cost;
    p.out_map = out_mapping;
    p.map_off = b->map_off;
    p.out_nevals = out_nevals;
    p.gscratch = base + off_teams;
    p.lay = cp.lay;
    p.n_graphs = b->n_graphs;
    p.n_pairs = b->n_pairs;
    p.n_vlab = b->total_vertices;
    p.adj_words = (int64_t)adj_words;
    p.plane_words = (int64_t)adj_words * B;
    p.map_total = b->map_len;
    NA_CK(launch_kbest(cp.W, cp.wide, cp.w32, cp.all_smem, label_instance(B), p, (int)grid, block,
                       (size_t)cp.lay.smem_bytes, st));
    NA_CK(cudaMemcpyAsync(&host_err, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (host_err & kErrDuplicateEdge)
        return set_error(FASTGED_ERR_INVALID_ARG, "duplicate edge in a graph");
    if (host_err & kErrBounds) return set_error(FASTGED_ERR_CUDA, "device bounds check failed");
    if (host_err) return set_error(FASTGED_ERR_CUDA, "device error flag set");
    return FASTGED_OK;
}
