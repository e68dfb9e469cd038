// fastged_runtime.cu -- host runtime behind the C ABI of include/fastged.h.
//
// A call flows as: validate + flatten the caller's graphs into one pinned staging buffer
// -> one host-to-device copy -> zero the bitset pools -> pack kernel (S0) -> one persistent
// K-Best launch per size class, each on its own stream, pulling pairs heaviest-first from
// a device work queue (S1-S5) -> one device-to-host copy of costs, evaluation counts,
// vertex maps and the error flag.
//
// Size classes group pairs by the number of 64-bit words a g2 bitset needs (1, 2, 4, 8, 16)
// and by the width of a stored vertex-map entry (8 or 16 bits). Each class gets a region
// plan: the per-team working set is split into regions placed in shared memory in order
// of access frequency; what does not fit goes to a per-team slice of global scratch.
// Pairs of single-word classes with small graphs and beams (n1 <= 64, n2 <= 63, K <= 128) form
// their own classes solved by one warp per pair (several warps per CTA, each with its own
// block of shared memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <functional>
#include <map>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fastged.h"
#include "fastged_internal.h"
#include "fastged_runtime.h"

namespace fastged {
cudaError_t launch_kbest(int W, bool wide_map, bool w32, bool sm, int bk, const KParams &p,
                         int grid, int block, size_t smem, cudaStream_t st);
cudaError_t kbest_occupancy(int W, bool wide_map, bool w32, bool sm, int bk, int block,
                            size_t smem, int *out);
bool kbest_has_smem_variant(int W, bool wide, bool w32);
bool kbest_has_cluster_variant(int W, bool wide, bool w32);
cudaError_t launch_kbest_cluster(int W, bool wide, int bk, const KParams &p, int grid, int block,
                                 size_t smem, int cluster, cudaStream_t st);
cudaError_t kbest_cluster_occupancy(int W, bool wide, int bk, int block, size_t smem, int cluster,
                                    int *out);
size_t team_shared_cluster_bytes();
cudaError_t launch_pack(const PackParams &pp, int n_graphs, cudaStream_t st);
size_t team_shared_static_bytes();
cudaError_t launch_kbest_warp(bool w32, int bk, const KParams &p, int grid, int block,
                              size_t smem, cudaStream_t st);
cudaError_t kbest_warp_occupancy(bool w32, int bk, int block, size_t smem, int *out);
}  // namespace fastged

using namespace fastged;

// ------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------
// per-thread message of the last failed call (a fixed buffer: storing it never allocates)
static thread_local char g_err[512];

int fastged::set_error(int code, const char *msg)
{
    snprintf(g_err, sizeof(g_err), "%s", msg ? msg : "");
    return code;
}

int fastged::set_error(int code, const std::string &msg) { return set_error(code, msg.c_str()); }

void fastged::clear_error() { g_err[0] = '\0'; }

static int cuda_fail(cudaError_t e, const char *what)
{
    const int code = (e == cudaErrorMemoryAllocation) ? FASTGED_ERR_OOM : FASTGED_ERR_CUDA;
    return set_error(code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

// ------------------------------------------------------------------------------------
// buffers
// ------------------------------------------------------------------------------------
static size_t grown(size_t n, size_t cap, bool headroom)
{
    if (!headroom) return n;
    const size_t g = std::max(n, cap + cap / 2);
    return (g + ((size_t)1 << 20) - 1) >> 20 << 20;
}

int DevBuf::ensure(size_t n, cudaStream_t st, bool headroom)
{
    if (n <= cap) return 0;
    if (inject_fire(FASTGED_INJECT_ALLOC))
        return set_error(FASTGED_ERR_OOM, "injected device allocation failure");
    const size_t want = grown(n, cap, headroom);
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    cap = 0;
    if (n == 0) return 0;
    cudaError_t e = cudaMallocAsync(&p, want, st);
    size_t got = want;
    if (e != cudaSuccess && want > n) {   // no room for the headroom: the exact size
        cudaGetLastError();
        e = cudaMallocAsync(&p, n, st);
        got = n;
    }
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return cuda_fail(e, "cudaMallocAsync");
    }
    cap = got;
    return 0;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

int PinBuf::ensure(size_t n, bool headroom)
{
    if (n <= cap) return 0;
    if (inject_fire(FASTGED_INJECT_ALLOC))
        return set_error(FASTGED_ERR_OOM, "injected pinned allocation failure");
    const size_t want = grown(n, cap, headroom);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (n == 0) return 0;
    cudaError_t e = cudaMallocHost(&p, want);
    size_t got = want;
    if (e != cudaSuccess && want > n) {
        cudaGetLastError();
        e = cudaMallocHost(&p, n);
        got = n;
    }
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return cuda_fail(e, "cudaMallocHost");
    }
    cap = got;
    return 0;
}

void PinBuf::release()
{
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// kernel instance for B edge-label planes: 0, exactly 2, or up to 8
int fastged::label_instance(int B) { return B == 0 ? 0 : (B == 2 ? 2 : 8); }

// ------------------------------------------------------------------------------------
// host thread pool for the batch flattening (validation and staging copies)
// ------------------------------------------------------------------------------------
// A process-wide pool of worker threads, created on first use. parallel_for(n, grain, f)
// runs f(lo, hi) over [0, n) in chunks of `grain` on the workers and the calling thread and
// returns when every chunk is done; a call made while another one is running (from another
// host thread) runs serially in the caller instead. The passes of one batch follow each other
// within microseconds, so an idle worker polls for the next job for a short while (yielding
// its core) before it sleeps, and the caller polls for the workers to finish before it
// sleeps; a job is still taken up and released under the mutex, so no worker can run a job
// whose call has returned.
class HostPool {
public:
    static HostPool &get()
    {
        static HostPool pool;
        return pool;
    }

    // threads that run a parallel_for: the workers and the caller
    int64_t threads() const { return (int64_t)workers_.size() + 1; }

    void parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)> &f)
    {
        grain = std::max<int64_t>(grain, 1);
        if (n <= grain || workers_.empty() || !busy_.try_lock()) {
            for (int64_t lo = 0; lo < n; lo += grain) f(lo, std::min(n, lo + grain));
            return;
        }
        {
            std::lock_guard<std::mutex> g(mu_);
            job_ = &f;
            n_ = n;
            grain_ = grain;
            next_.store(0);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        run(&f, n, grain);
        poll_until([&] { return active_.load(std::memory_order_acquire) == 0; });
        {
            std::unique_lock<std::mutex> lk(mu_);
            done_cv_.wait(lk, [&] { return active_.load() == 0; });
            job_ = nullptr;
        }
        busy_.unlock();
    }

private:
    static constexpr int kPollUs = 200;

    // FASTGED_HOST_THREADS (read once, at first use) sets the threads of a parallel_for,
    // the caller included: 1 runs everything in the caller; by default up to 16
    HostPool()
    {
        const unsigned hw = std::thread::hardware_concurrency();
        int nw = (int)std::min(15u, hw > 1 ? hw - 1 : 0u);
        if (const char *e = getenv("FASTGED_HOST_THREADS")) {
            const long t = strtol(e, nullptr, 10);
            if (t >= 1) nw = (int)std::min(t - 1, 63L);
        }
        for (int k = 0; k < nw; ++k) workers_.emplace_back([this] { loop(); });
    }
    ~HostPool()
    {
        {
            std::lock_guard<std::mutex> g(mu_);
            quit_.store(true);
        }
        cv_.notify_all();
        for (auto &t : workers_) t.join();
    }
    template <typename Pred>
    static void poll_until(Pred done)
    {
        const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(kPollUs);
        while (!done() && std::chrono::steady_clock::now() < until) std::this_thread::yield();
    }
    void run(const std::function<void(int64_t, int64_t)> *f, int64_t n, int64_t grain)
    {
        for (;;) {
            const int64_t lo = next_.fetch_add(grain);
            if (lo >= n) break;
            (*f)(lo, std::min(n, lo + grain));
        }
    }
    void loop()
    {
        uint64_t seen = 0;
        for (;;) {
            poll_until([&] { return gen_.load(std::memory_order_acquire) != seen || quit_.load(); });
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [&] { return quit_.load() || (gen_.load() != seen && job_ != nullptr); });
            if (quit_.load()) return;
            seen = gen_.load();
            const auto *f = job_;
            const int64_t n = n_, grain = grain_;
            active_.fetch_add(1);
            lk.unlock();
            run(f, n, grain);
            lk.lock();
            if (active_.fetch_sub(1, std::memory_order_acq_rel) == 1) done_cv_.notify_all();
        }
    }

    std::vector<std::thread> workers_;
    std::mutex mu_, busy_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int64_t, int64_t)> *job_ = nullptr;   // guarded by mu_
    int64_t n_ = 0, grain_ = 1;                                     // guarded by mu_
    std::atomic<int64_t> next_{0};
    std::atomic<uint64_t> gen_{0};   // written under mu_, polled without it
    std::atomic<int> active_{0};     // workers inside run(); changed under mu_
    std::atomic<bool> quit_{false};
};

// The error of the lowest index among those reported from parallel chunks.
struct FirstError {
    std::mutex mu;
    int64_t idx = INT64_MAX;
    std::string msg;
    void put(int64_t i, std::string m)
    {
        std::lock_guard<std::mutex> g(mu);
        if (i < idx) {
            idx = i;
            msg = std::move(m);
        }
    }
    int report() const { return set_error(FASTGED_ERR_INVALID_ARG, msg); }
};

// ------------------------------------------------------------------------------------
// host-side fault injection (tests) and the handle's wait bound
// ------------------------------------------------------------------------------------
static std::atomic<int> g_inject[3];   // countdown per kind; 0 = disarmed

bool fastged::inject_fire(int kind)
{
    int c = g_inject[kind].load();
    while (c > 0)
        if (g_inject[kind].compare_exchange_weak(c, c - 1)) return c == 1;
    return false;
}

extern "C" int fastged_inject_fault(int32_t kind, int32_t countdown)
{
    clear_error();
    if (kind < 0 || kind > 2 || countdown < 0)
        return set_error(FASTGED_ERR_INVALID_ARG, "fault kind or countdown out of range");
    g_inject[kind].store(countdown);
    return FASTGED_OK;
}

extern "C" int fastged_set_timeout(fastged_handle *h, int32_t ms)
{
    clear_error();
    if (!h || ms < 0) return set_error(FASTGED_ERR_INVALID_ARG, "null handle or negative timeout");
    h->timeout_ms = ms;
    return FASTGED_OK;
}

static int words_class(int n)
{
    const int w = (n + 63) / 64;
    if (w <= 1) return 1;
    if (w <= 2) return 2;
    if (w <= 4) return 4;
    if (w <= 8) return 8;
    return 16;
}

// ------------------------------------------------------------------------------------
// handle
// ------------------------------------------------------------------------------------
extern "C" int fastged_version(void) { return FASTGED_VERSION; }

extern "C" const char *fastged_last_error(const fastged_handle *) { return g_err; }

extern "C" int fastged_create(const fastged_cost_model *cost, fastged_handle **out)
{
    clear_error();
    if (!cost || !out) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    const int32_t *cv = &cost->v_sub;
    for (int k = 0; k < 6; ++k)
        if (cv[k] < 0) return set_error(FASTGED_ERR_INVALID_ARG, "negative cost");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    fastged_handle *h = new fastged_handle();
    h->cost = *cost;
    h->device = dev;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // the class streams are created when a batch first has several size classes: the
    // device maps streams onto a few hardware queues, and a process with many handles (a
    // server's lanes) keeps its main streams on queues of their own that way
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    for (int k = 0; k < kMaxClasses + 1 && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&h->ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fastged_destroy(h);
        return cuda_fail(e, "stream/event creation");
    }
    *out = h;
    return FASTGED_OK;
}

extern "C" void fastged_destroy(fastged_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int k = 0; k < kMaxClasses; ++k)
        if (h->class_stream[k]) {
            cudaStreamSynchronize(h->class_stream[k]);
            cudaStreamDestroy(h->class_stream[k]);
        }
    for (int k = 0; k < kMaxClasses + 1; ++k)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    if (h->done) cudaEventDestroy(h->done);
    if (h->stream) cudaStreamDestroy(h->stream);
    h->dev_in.release();
    h->dev_work.release();
    h->pin.release();
    delete h;
}

// ------------------------------------------------------------------------------------
// flattening + validation
// ------------------------------------------------------------------------------------
fastged_options fastged::default_options()
{
    fastged_options o;
    memset(&o, 0, sizeof(o));
    o.use_cuda_graph = 1;
    return o;
}

void fastged::plan_layout(ClassPlan &cp, int B, int block, size_t budget)
{
    Layout &L = cp.lay;
    const int NW = (block / 32) * cp.cluster;   // warps of the whole team
    const int W = cp.W;
    const size_t msz = cp.wide ? 2 : 1;
    const size_t wb = cp.w32 ? 4 : 8;
    L.kmax = cp.kmax;
    L.n1max = cp.n1max;
    L.n2max = cp.n2max;
    L.n2s = (int)align_up((size_t)std::max(cp.n2max, 1) + 1, 4);
    L.mrow = (int)align_up((size_t)std::max(cp.n1max, 1) * msz, 16);
    L.fs = cp.n2max + 1;
    L.word_bytes = (int)wb;
    L.B = B;
    size_t sz[RG_COUNT];
    const size_t km = (size_t)cp.kmax;
    const size_t ncand = km * ((size_t)cp.n2max + 1);
    // node slots a CTA prepares: all of them, or its share of a cluster team
    const size_t kl = cp.cluster > 1 ? (km + cp.cluster - 1) / cp.cluster + 1 : km;
    L.kloc = (int32_t)kl;
    sz[RG_HIST] = (size_t)kHistMax * NW * 4;
    sz[RG_ALPHA2] = (size_t)L.n2s * 4;
    sz[RG_CROW] = (size_t)2 * L.n2s * 4;
    sz[RG_A2T] = (size_t)W * L.n2s * wb;
    sz[RG_L2T] = (size_t)B * W * L.n2s * wb;
    sz[RG_SBASE] = kl * 4;
    sz[RG_PED0] = km * 4;
    sz[RG_PED1] = km * 4;
    sz[RG_SEL] = km * 4;
    sz[RG_SELPED] = km * 4;
    sz[RG_KLIST] = km * 4;
    sz[RG_KPED] = km * 4;
    sz[RG_NOFF] = ((size_t)cp.n1max + 1) * 4;
    sz[RG_NBR] = (size_t)std::max(cp.m1max, 1) * 4;
    sz[RG_IMG0] = km * W * wb;
    sz[RG_IMG1] = km * W * wb;
    sz[RG_P] = kl * W * wb;
    sz[RG_PL] = (size_t)B * kl * W * wb;
    sz[RG_IMGL] = cp.cluster > 1 ? kl * W * wb : 0;
    // single-word classes pack the successor ids into the PED entries
    // one entry per successor: 32 bits when packed, else 64 (PED, parent slot, j)
    const bool packed = cp.pk && cp.cluster == 1;
    L.pk = packed ? 1 : 0;
    sz[RG_CAND] = ncand * (packed ? 4 : 8);
    sz[RG_MAP0] = km * L.mrow;
    sz[RG_MAP1] = km * L.mrow;
    // shared memory is filled in order of access frequency; the rest goes to global scratch
    static const int prio[RG_COUNT] = {RG_HIST, RG_CROW, RG_ALPHA2, RG_SBASE, RG_PED0, RG_PED1,
                                       RG_SEL, RG_SELPED, RG_KLIST, RG_KPED, RG_NOFF,
                                       RG_A2T, RG_L2T, RG_IMG0, RG_IMG1, RG_P, RG_PL,
                                       RG_CAND, RG_NBR, RG_MAP0, RG_MAP1, RG_IMGL};
    // cluster teams: the per-CTA tables the CTA writes (P, PL, sbase, staged Img) must be in
    // shared memory, so they come first
    static const int prio_cl[RG_COUNT] = {RG_SBASE, RG_P, RG_PL, RG_IMGL, RG_CROW, RG_ALPHA2,
                                          RG_NOFF,
                                          RG_A2T, RG_L2T, RG_NBR, RG_HIST, RG_PED0, RG_PED1,
                                          RG_SEL, RG_SELPED, RG_KLIST, RG_KPED, RG_IMG0,
                                          RG_IMG1, RG_CAND, RG_MAP0, RG_MAP1};
    // a cluster team shares only global memory: its CTAs keep private shared-memory copies
    // of the read-only target-graph tables and neighbour lists, everything else is global
    auto cta_local = [](int r) {
        return r == RG_ALPHA2 || r == RG_A2T || r == RG_L2T || r == RG_NOFF || r == RG_NBR ||
               r == RG_P || r == RG_PL || r == RG_SBASE || r == RG_IMGL || r == RG_CROW;
    };
    for (int r = 0; r < RG_COUNT; ++r) L.rsize[r] = (int64_t)align_up(sz[r], 16);
#ifdef FASTGED_BOUNDS_CHECK
    // tests of the checked build: declare the selection list four entries long (the buffer
    // keeps its real size), so that the kernels' own accesses trip the check
    if (getenv("FASTGED_CHECK_SHRINK_SEL")) L.rsize[RG_SEL] = 16;
#endif
    size_t s_used = 0, g_used = 0, c_used = 0;
    L.smem_mask = 0;
    L.cta_mask = 0;
    for (int k = 0; k < RG_COUNT; ++k) {
        const int r = cp.cluster > 1 ? prio_cl[k] : prio[k];
        const size_t a = align_up(sz[r], 16);
        if (s_used + a <= budget && (cp.cluster == 1 || cta_local(r))) {
            L.off[r] = (int64_t)s_used;
            L.smem_mask |= 1u << r;
            s_used += a;
        } else if (cp.cluster > 1 && cta_local(r)) {
            L.off[r] = (int64_t)c_used;   // one copy per CTA of the cluster
            L.cta_mask |= 1u << r;
            c_used += a;
        } else {
            L.off[r] = (int64_t)g_used;
            g_used += a;
        }
    }
    L.team_off = (int64_t)align_up(g_used, 256);
    L.cta_off = 0;
    L.cta_bytes = 0;
    if (cp.cluster > 1) {
        g_used = (size_t)L.team_off + team_shared_cluster_bytes();
        L.cta_off = (int64_t)align_up(g_used, 256);
        L.cta_bytes = (int64_t)align_up(c_used, 256);
        g_used = (size_t)L.cta_off + (size_t)cp.cluster * (size_t)L.cta_bytes;
    }
    L.smem_bytes = (int64_t)s_used;
    L.slice_bytes = (int64_t)align_up(g_used, 256);
}

size_t fastged::plan_warp_layout(ClassPlan &cp, int B, bool gmap)
{
    WarpLayout &wl = cp.wl;
    const int npl = label_instance(B);
    const size_t rec = (size_t)warp_rec_bytes(cp.w32, npl);
    const size_t wb = cp.w32 ? 4 : 8;
    const size_t km = (size_t)cp.kmax, n2 = (size_t)cp.n2max, n1 = (size_t)cp.n1max;
    wl.mrow = (int32_t)align_up(std::max<size_t>(n1, 1), 16);
    size_t sz[WR_COUNT];
    sz[WR_TGT] = (n2 + 2) * rec;   // records 1..n2 the vertices, n2 + 1 the deletion, 0 the stand-in
    sz[WR_LAB2] = std::max<size_t>(n2, 1) * 4;
    sz[WR_NOFF] = (n1 + 1) * 4;
    sz[WR_NBR] = (size_t)std::max(cp.m1max, 1) * 4;
    sz[WR_IMG0] = sz[WR_IMG1] = km * wb;
    sz[WR_PED0] = sz[WR_PED1] = km * 4;
    sz[WR_E20] = sz[WR_E21] = km * 2;
    sz[WR_ENT] = km * (n2 + 1) * 2;
    sz[WR_NODEOFF] = (km + 1) * 2;
    sz[WR_KLIST] = km * 4;
    sz[WR_SEL] = km * 4;
    sz[WR_SELPED] = km * 4;
    sz[WR_MAP0] = sz[WR_MAP1] = km * (size_t)wl.mrow;
    size_t sh = 0, gl = 0;
    for (int r = 0; r < WR_COUNT; ++r) {
        const size_t a = align_up(sz[r], 16);
        wl.size[r] = (int32_t)a;
        if (gmap && (r == WR_MAP0 || r == WR_MAP1)) {
            wl.off[r] = (int32_t)gl;
            gl += a;
        } else {
            wl.off[r] = (int32_t)sh;
            sh += a;
        }
    }
#ifdef FASTGED_BOUNDS_CHECK
    if (getenv("FASTGED_CHECK_SHRINK_SEL")) wl.size[WR_SEL] = 16;   // see plan_layout
#endif
    wl.warp_bytes = (int32_t)sh;
    wl.gmap = gmap ? 1 : 0;
    wl.gmap_bytes = gmap ? (int32_t)align_up(gl, 256) : 0;
    cp.lay.B = B;
    cp.lay.kmax = cp.kmax;
    cp.lay.n1max = cp.n1max;
    cp.lay.n2max = cp.n2max;
    cp.lay.word_bytes = (int32_t)wb;
    cp.lay.pk = 1;
    return sh;
}

static size_t layout_total(const ClassPlan &cp, int B, int block)
{
    ClassPlan t = cp;
    plan_layout(t, B, block, (size_t)1 << 40);
    return (size_t)t.lay.smem_bytes;
}

// ------------------------------------------------------------------------------------
// tuning table: size-class shape -> team shape (threads per CTA, CTAs per cluster)
// ------------------------------------------------------------------------------------
struct TuneChoice {
    int block = 0;
    int cluster = 1;
    int gmap = -1;   // one-warp classes: 1 = vertex maps in global scratch, 0 = shared memory
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune;
static bool g_tune_loaded = false;
static TuneChoice g_tune_force;   // set only while the autotuner times a candidate
static bool g_tune_forcing = false;

static int pow2_ceil(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

static std::string class_key(const ClassPlan &cp, int B, int npairs, int sm_count)
{
    char buf[128];
    snprintf(buf, sizeof(buf), "%sw%d%s%s%s_b%d_k%d_n%d_%s", cp.warp ? "warp_" : "", cp.W,
             cp.wide ? "x" : "", cp.w32 ? "h" : "", cp.pk ? "p" : "", label_instance(B),
             pow2_ceil(cp.kmax), pow2_ceil(cp.n2max), npairs < sm_count ? "few" : "many");
    return buf;
}

static void tune_load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("FASTGED_AUTOTUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    // one entry per line: key, threads per CTA, CTAs per team, map placement, time in ms
    char line[256], key[128];
    while (fgets(line, sizeof(line), f)) {
        int block = 0, cluster = 1, gmap = -1;
        if (sscanf(line, "%127s %d %d %d", key, &block, &cluster, &gmap) != 4) continue;
        TuneChoice c;
        c.block = block;
        c.cluster = cluster;
        c.gmap = gmap;
        g_tune[key] = c;
    }
    fclose(f);
}

static bool tune_lookup(const std::string &key, TuneChoice *out)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    if (g_tune_forcing) {
        *out = g_tune_force;
        return true;
    }
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

static void tune_store(const std::string &key, const TuneChoice &c, double ms)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    g_tune[key] = c;
    const char *path = getenv("FASTGED_AUTOTUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %.4f\n", key.c_str(), c.block, c.cluster, c.gmap, ms);
    fclose(f);
}

extern "C" int fastged_autotune_entries(void)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    return (int)g_tune.size();
}

extern "C" void fastged_autotune_clear(void)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.clear();
    g_tune_loaded = true;
}

// A class whose pairs are fewer than the SMs may give each pair a cluster of CTAs: classes of
// large graphs (four or more words), and two-word classes whose beam holds at least 2^16
// successors per level.
static bool cluster_eligible(const ClassPlan &cp, int npairs, int sm_count)
{
    if (!kbest_has_cluster_variant(cp.W, cp.wide, cp.w32) || npairs >= sm_count) return false;
    return cp.W >= 4 || (int64_t)cp.kmax * (cp.n2max + 1) >= 65536;
}

// CTAs per cluster without a tuning entry: about 20,000 successors of a level (K times the
// target's vertices and the deletion) per CTA, between 2 and 8 CTAs (16 for a handful of
// very wide pairs), then halved while the class's teams would take more than two waves of
// the GPU (smaller teams spend fewer cluster barriers per successor).
static int cluster_rule(const ClassPlan &cp, int npairs, int sm_count)
{
    const int64_t succ = (int64_t)cp.kmax * (cp.n2max + 1);
    int cl = succ <= 40000 ? 2 : succ <= 160000 ? 4 : 8;
    if (succ >= 2000000 && (int64_t)npairs * 16 <= sm_count) cl = 16;
    while (cl > 2 && (int64_t)npairs * cl > 2 * (int64_t)sm_count) cl >>= 1;
    return cl;
}

// The resident teams of a class capped to max_sms SMs (0 = no cap): whole clusters, or as
// many teams as fit that many SMs at per_sm teams each; at least one team.
static void cap_grid(ClassPlan &cp, int max_sms, int per_sm)
{
    if (max_sms <= 0) return;
    const int teams = cp.grid / cp.cluster;
    const int cap = cp.cluster > 1 ? std::max(1, max_sms / cp.cluster)
                                   : std::max(1, max_sms * std::max(1, per_sm));
    cp.grid = std::min(teams, cap) * cp.cluster;
}

// Chooses the team shape of a class (threads, CTAs per team) and its shared-memory budget.
// Classes of large pairs that are too few to fill the GPU one pair per CTA get a cluster of
// CTAs per pair.
// One-warp classes: warps per CTA (threads / 32, at most 4) and where the vertex maps live.
// Without a tuning entry the maps stay in shared memory when that still leaves room for 16
// warps per SM, and CTAs hold 4 warps.
static int tune_warp_class(fastged_handle *h, ClassPlan &cp, int B, int forced_block,
                           int max_sms)
{
    const int npairs = (int)std::max<size_t>(cp.order.size(), 1);
    TuneChoice tc;
    const bool tuned = tune_lookup(class_key(cp, B, npairs, h->sm_count), &tc);
    int block = forced_block ? forced_block : (tuned && tc.block ? tc.block : 128);
    bool gmap;
    if (tuned && tc.gmap >= 0) {
        gmap = tc.gmap != 0;
    } else {
        const size_t shared_maps = plan_warp_layout(cp, B, false);
        gmap = (size_t)h->smem_per_sm / std::max<size_t>(shared_maps, 1) < 16;
    }
    const size_t wbytes = plan_warp_layout(cp, B, gmap);
    // at most 4 warps per CTA (the kernel's launch bound is 128 threads)
    int wpc = std::min(4, std::max(1, block / 32));
    while (wpc > 1 && (size_t)wpc * wbytes > (size_t)h->smem_optin) wpc >>= 1;
    if ((size_t)wpc * wbytes > (size_t)h->smem_optin)
        return set_error(FASTGED_ERR_CUDA, "a one-warp team does not fit shared memory");
    block = wpc * 32;
    int occ = 0;
    cudaError_t e = kbest_warp_occupancy(cp.w32, label_instance(B), block, (size_t)wpc * wbytes,
                                         &occ);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ < 1) return set_error(FASTGED_ERR_CUDA, "one-warp teams do not fit on an SM");
    cp.block = block;
    cp.smem = (size_t)wpc * wbytes;
    cp.all_smem = !gmap;
    cp.lay.smem_bytes = (int64_t)cp.smem;
    cp.lay.slice_bytes = gmap ? (int64_t)wpc * cp.wl.gmap_bytes : 0;
    const int64_t need = ((int64_t)cp.order.size() + wpc - 1) / wpc;
    cp.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sm_count * occ, need));
    cap_grid(cp, max_sms, occ);
    return FASTGED_OK;
}

static int tune_class(fastged_handle *h, ClassPlan &cp, int B, int forced_block, int max_sms,
                      int forced_cluster)
{
    if (cp.warp) return tune_warp_class(h, cp, B, forced_block, max_sms);
    const size_t stat = team_shared_static_bytes() + 1024;   // + per-block reservation
    const size_t per_sm = (size_t)h->smem_per_sm;
    const size_t max_dyn = (size_t)h->smem_optin - team_shared_static_bytes();
    const int npairs = (int)std::max<size_t>(cp.order.size(), 1);
    TuneChoice tc;
    const bool tuned = forced_block == 0 &&
                       tune_lookup(class_key(cp, B, npairs, h->sm_count), &tc);
    if (tuned) forced_block = tc.block;
    if (cluster_eligible(cp, npairs, h->sm_count)) {
        const char *env = getenv("FASTGED_CLUSTER");
        int cl = env ? atoi(env)
                     : forced_cluster ? forced_cluster
                                      : (tuned ? tc.cluster : cluster_rule(cp, npairs, h->sm_count));
        if (cl == 1 || cl == 2 || cl == 4 || cl == 8 || cl == 16) {
            cp.cluster = cl;
        }
    }
    if (cp.cluster > 1) {
        plan_layout(cp, B, forced_block ? forced_block : 512, max_dyn);
        const int block = cp.block = forced_block ? forced_block : 512;
        int nclu = 0;
        cudaError_t e = kbest_cluster_occupancy(cp.W, cp.wide, label_instance(B), block,
                                                (size_t)cp.lay.smem_bytes, cp.cluster, &nclu);
        if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
        if (nclu < 1) return set_error(FASTGED_ERR_CUDA, "a cluster team does not fit the GPU");
        cp.block = block;
        cp.smem = (size_t)cp.lay.smem_bytes;
        cp.all_smem = false;
        cp.grid = std::min(nclu, npairs) * cp.cluster;
        cap_grid(cp, max_sms, 1);
        return FASTGED_OK;
    }
    int block = forced_block;
    if (block == 0) block = cp.kmax <= 32 ? 128 : 256;
    const size_t total = layout_total(cp, B, block);
    size_t budget;
    if (total + stat <= per_sm / 2 && total <= max_dyn) {
        budget = total;                                   // all in shared memory
    } else {
        budget = std::min(max_dyn, per_sm / 2 - stat);    // keep two teams per SM
    }
    plan_layout(cp, B, block, budget);
    cp.all_smem = cp.lay.slice_bytes == 0 && kbest_has_smem_variant(cp.W, cp.wide, cp.w32);
    int occ = 0;
    cudaError_t e = kbest_occupancy(cp.W, cp.wide, cp.w32, cp.all_smem, label_instance(B), block,
                                    (size_t)cp.lay.smem_bytes, &occ);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ < 1) return set_error(FASTGED_ERR_CUDA, "team does not fit on an SM");
    cp.block = block;
    cp.smem = (size_t)cp.lay.smem_bytes;
    const int64_t want = (int64_t)h->sm_count * occ;
    cp.grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)cp.order.size()));
    cap_grid(cp, max_sms, occ);
    return FASTGED_OK;
}

// Source graphs relabelled so that vertex k is the k-th in descending-degree order (ties by
// index): every graph that is a pair's source gets a relabelled copy appended to the graph
// list, and the pairs point at the copies. perm of a copy maps new ids to original ids.
struct Reordered {
    fastged_pair_list list{};
    std::vector<fastged_graph> graphs;
    std::vector<std::vector<int32_t>> store;   // labels, edges and edge labels of the copies
    std::vector<int32_t> pairs;
    std::vector<int> copy_of;                  // graph -> index of its copy, or -1
    std::vector<std::vector<int32_t>> perm;    // per copy: new id -> original id
};

static bool reorder_sources(const fastged_pair_list *pl, Reordered &ro)
{
    const int ng = pl->n_graphs, np = pl->n_pairs;
    ro.graphs.assign(pl->graphs, pl->graphs + ng);
    ro.pairs.assign(pl->pairs, pl->pairs + 2 * (size_t)np);
    ro.copy_of.assign(ng, -1);
    for (int p = 0; p < np; ++p) {
        const int g = pl->pairs[2 * p];
        if (g < 0 || g >= ng) continue;   // reported by the pair validation
        if (ro.copy_of[g] < 0) {
            const fastged_graph &G = pl->graphs[g];
            if (G.n < 0 || G.n > FASTGED_MAX_N || G.m < 0 || (G.n > 0 && !G.vlabel) ||
                (G.m > 0 && !G.edges))
                continue;   // reported by the graph validation
            bool ok = true;
            std::vector<int> deg(G.n, 0);
            for (int k = 0; k < G.m && ok; ++k) {
                const int u = G.edges[2 * k], v = G.edges[2 * k + 1];
                if (u < 0 || v < 0 || u >= G.n || v >= G.n) ok = false;
                else { ++deg[u]; ++deg[v]; }
            }
            if (!ok) continue;
            std::vector<int32_t> perm(G.n), inv(G.n);
            for (int v = 0; v < G.n; ++v) perm[v] = v;
            std::stable_sort(perm.begin(), perm.end(),
                             [&](int a, int c) { return deg[a] > deg[c]; });
            for (int k = 0; k < G.n; ++k) inv[perm[k]] = k;
            std::vector<int32_t> lab(G.n), edg(2 * (size_t)G.m), el;
            for (int k = 0; k < G.n; ++k) lab[k] = G.vlabel[perm[k]];
            for (int k = 0; k < G.m; ++k) {
                edg[2 * k] = inv[G.edges[2 * k]];
                edg[2 * k + 1] = inv[G.edges[2 * k + 1]];
            }
            if (G.elabel) el.assign(G.elabel, G.elabel + G.m);
            ro.store.push_back(std::move(lab));
            ro.store.push_back(std::move(edg));
            ro.store.push_back(std::move(el));
            fastged_graph C = G;
            C.vlabel = ro.store[ro.store.size() - 3].data();
            C.edges = ro.store[ro.store.size() - 2].data();
            C.elabel = G.elabel ? ro.store[ro.store.size() - 1].data() : nullptr;
            ro.copy_of[g] = (int)ro.graphs.size();
            ro.graphs.push_back(C);
            ro.perm.push_back(std::move(perm));
        }
        ro.pairs[2 * p] = ro.copy_of[g];
    }
    ro.list.n_graphs = (int32_t)ro.graphs.size();
    ro.list.graphs = ro.graphs.data();
    ro.list.n_pairs = np;
    ro.list.pairs = ro.pairs.data();
    return true;
}

int fastged::flatten(fastged_handle *h, const fastged_pair_list *pl, int32_t K,
                     const fastged_options &opt, Batch &b)
{
    if (!pl) return set_error(FASTGED_ERR_INVALID_ARG, "null pair list");
    if (K < 1 || K > FASTGED_MAX_K) return set_error(FASTGED_ERR_INVALID_ARG, "K out of range");
    if (pl->n_graphs < 0 || pl->n_pairs < 0)
        return set_error(FASTGED_ERR_INVALID_ARG, "negative count");
    if ((pl->n_graphs > 0 && !pl->graphs) || (pl->n_pairs > 0 && !pl->pairs))
        return set_error(FASTGED_ERR_INVALID_ARG, "null graphs or pairs");
    if (opt.variant != 0 && opt.variant != 1)
        return set_error(FASTGED_ERR_INVALID_ARG, "variant must be 0 or 1");
    if (opt.hist_window != 0 && (opt.hist_window < 2 || opt.hist_window > kHistMax))
        return set_error(FASTGED_ERR_INVALID_ARG, "hist_window out of range");
    if (opt.block_threads != 0 && opt.block_threads != 128 && opt.block_threads != 256 &&
        opt.block_threads != 512)
        return set_error(FASTGED_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
    if (opt.vertex_order != FASTGED_ORDER_INDEX && opt.vertex_order != FASTGED_ORDER_DEGREE)
        return set_error(FASTGED_ERR_INVALID_ARG, "vertex_order must be 0 or 1");
    if (opt.team != FASTGED_TEAM_AUTO && opt.team != FASTGED_TEAM_CTA)
        return set_error(FASTGED_ERR_INVALID_ARG, "team must be 0 or 1");
    if (opt.max_sms < 0) return set_error(FASTGED_ERR_INVALID_ARG, "max_sms must be >= 0");
    if (opt.cluster != 0 && opt.cluster != 1 && opt.cluster != 2 && opt.cluster != 4 &&
        opt.cluster != 8 && opt.cluster != 16)
        return set_error(FASTGED_ERR_INVALID_ARG, "cluster must be 0, 1, 2, 4, 8 or 16");
    b.perm.clear();
    Reordered ro;
    if (opt.vertex_order == FASTGED_ORDER_DEGREE) {
        reorder_sources(pl, ro);
        pl = &ro.list;
    }

    const int ng = pl->n_graphs, np = pl->n_pairs;
    b.n_graphs = ng;
    b.n_pairs = np;
    b.K = K;
    b.opt = opt;
    b.has_kpp = opt.k_per_pair != nullptr;
    b.meta.resize(ng);
    HostPool &pool = HostPool::get();
    FirstError ferr;
    // Graphs and pairs are processed in fixed chunks on the host pool; each chunk keeps its
    // own partial results (sizes, maxima, class histograms) and a short serial step combines
    // them, so nothing depends on how many threads ran.
    const int64_t nthr = pool.threads();
    const int64_t gch = std::max<int64_t>(1024, (ng + 4 * nthr - 1) / (4 * nthr));
    const int64_t pch = std::max<int64_t>(2048, (np + 2 * nthr - 1) / (2 * nthr));
    const int ngc = (int)((ng + gch - 1) / gch), npc = (int)((np + pch - 1) / pch);

    // graphs: validation, words per row, edge-label range, sizes per chunk
    struct GraphChunk {
        int64_t nv = 0, ne = 0, adjw = 0;   // sizes of the chunk, then its base offsets
        int maxlab = 0;
        bool lab = false;
    };
    std::vector<GraphChunk> gcs(ngc);
    pool.parallel_for(ng, gch, [&](int64_t lo, int64_t hi) {
        GraphChunk &C = gcs[lo / gch];
        for (int g = (int)lo; g < (int)hi; ++g) {
            const fastged_graph &G = pl->graphs[g];
            auto where = [g] { return "graph " + std::to_string(g); };
            if (G.n < 0 || G.n > FASTGED_MAX_N) { ferr.put(g, where() + ": n out of range"); break; }
            if (G.m < 0 || (int64_t)G.m > (int64_t)G.n * (G.n - 1) / 2) { ferr.put(g, where() + ": m out of range"); break; }
            if ((G.n > 0 && !G.vlabel) || (G.m > 0 && !G.edges)) { ferr.put(g, where() + ": null array"); break; }
            GraphMeta &M = b.meta[g];
            M.n = G.n;
            M.m = G.m;
            M.W = std::max(1, (G.n + 63) / 64);
            M.pad = 0;
            C.nv += G.n;
            C.ne += G.m;
            C.adjw += (int64_t)G.n * M.W;
            if (G.elabel && G.m > 0) {
                C.lab = true;
                int ml = 0, lo_l = 0;
                for (int k = 0; k < G.m; ++k) {
                    ml = std::max(ml, G.elabel[k]);
                    lo_l = std::min(lo_l, G.elabel[k]);
                }
                if (lo_l < 0 || ml > FASTGED_MAX_ELABEL) { ferr.put(g, where() + ": edge label out of range"); break; }
                C.maxlab = std::max(C.maxlab, ml);
            }
        }
    });
    if (ferr.idx != INT64_MAX) return ferr.report();
    int64_t nv = 0, ne = 0, adjw = 0;
    int maxlab = 0;
    bool labelled = false;
    for (GraphChunk &C : gcs) {
        const GraphChunk t = C;
        C.nv = nv;
        C.ne = ne;
        C.adjw = adjw;
        nv += t.nv;
        ne += t.ne;
        adjw += t.adjw;
        maxlab = std::max(maxlab, t.maxlab);
        labelled = labelled || t.lab;
    }
    int B = 0;
    while ((1 << B) <= maxlab) ++B;   // planes needed for labels 0..maxlab
    if (B == 1) B = 2;                // served by the two-plane kernel (second plane all zero)
    b.B = B;
    b.labelled = labelled && B > 0;
    b.n_vlab = nv;
    b.n_edges = ne;
    b.adj_words = adjw;
    b.plane_words = adjw * B;

    // pairs: validation, size class and work bucket of each, with per-chunk class statistics
    // and (class, bucket) histograms. Classes are numbered in order of first appearance;
    // inside a class the pairs run heaviest first (longest-processing-time order, which only
    // shortens the tail: results do not depend on the order), by a work estimate
    // n1 * min(K, n1 n2 + 1) * (n2 + 1) bucketed at 1/16 of a power of two, ties by index.
    const fastged_cost_model &c = h->cost;
    const int32_t *kpp = opt.k_per_pair;
    b.map_off.resize(np);
    b.classes.clear();
    constexpr int kKeys = 32, kBuckets = 64 * 16;
    struct KeyClass {
        int first = INT_MAX;   // first pair of this class key
        int8_t W = 1, wide = 0, w32 = 0, pk = 0, warp = 0;
        int n1max = 0, n2max = 0, m1max = 0, kmax = 1;
        int bmin = kBuckets, bmax = -1;
    };
    struct PairChunk {
        int64_t maps = 0;                // map entries of the chunk, then its base offset
        KeyClass key[kKeys];
        std::vector<int32_t> hist;       // [key][bucket] counts, then output positions
    };
    std::vector<PairChunk> pcs(npc);
    std::vector<uint8_t> pkey((size_t)np);
    std::vector<uint16_t> pbk((size_t)np);
    pool.parallel_for(np, pch, [&](int64_t lo, int64_t hi) {
        PairChunk &C = pcs[lo / pch];
        C.hist.assign((size_t)kKeys * kBuckets, 0);
        for (int p = (int)lo; p < (int)hi; ++p) {
            const int a = pl->pairs[2 * p], d = pl->pairs[2 * p + 1];
            auto where = [p] { return "pair " + std::to_string(p); };
            if (a < 0 || a >= ng || d < 0 || d >= ng) { ferr.put(p, where() + ": graph index out of range"); break; }
            const int kp = kpp ? kpp[p] : K;
            if (kp < 1 || kp > K) { ferr.put(p, where() + ": per-pair K out of range"); break; }
            const GraphMeta &g1 = b.meta[a], &g2 = b.meta[d];
            const long long bound = (long long)g1.n * std::max(c.v_sub, c.v_del) +
                                    (long long)g2.n * c.v_ins +
                                    (long long)g1.m * std::max(c.e_sub, c.e_del) +
                                    (long long)g2.m * c.e_ins;
            if (bound >= (long long)INT32_MAX) { ferr.put(p, where() + ": costs can overflow int32"); break; }
            int W = words_class(g2.n);
            // packing (PED, parent slot, j) into 32 bits needs every PED below 2^16 (PEDs
            // never count vertex insertions, and at most the g2 edges among mapped vertices)
            // and K within the slot field
            const long long ped_bound = (long long)g1.n * std::max(c.v_sub, c.v_del) +
                                        (long long)g1.m * std::max(c.e_sub, c.e_del) +
                                        (long long)g2.m * c.e_ins;
            const bool pk = packable(ped_bound, kp, g2.n);
            if (W == 1 && !pk) W = 2;
            // one warp per pair: single-word, packable pairs with small source graphs and
            // beams, variant A
            const bool warp = opt.team == FASTGED_TEAM_AUTO && opt.variant == 0 && W == 1 &&
                              g1.n <= kWarpMaxN && g2.n <= kWarpMaxN2 && kp <= kWarpMaxK;
            const bool wide = g2.n >= 255,
                       w32 = W == 1 && g2.n <= (warp ? kWarpMaxN2Word32 : 32);
            const int key = warp ? 22 + (w32 ? 1 : 0) :
                (w32 ? 10 : (W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : W == 8 ? 3 : 4) * 2 + (wide ? 1 : 0)) * 2 +
                (pk ? 1 : 0);
            const double wt = (double)g1.n *
                              (double)std::min<long long>(kp, 1 + (long long)g2.n * g1.n) *
                              (double)(g2.n + 1);
            int q = wt < 1.0 ? 0 : (int)(std::log2(wt) * 16.0);
            q = std::min(std::max(q, 0), kBuckets - 1);
            const int bk = kBuckets - 1 - q;   // heavier first
            pkey[p] = (uint8_t)key;
            pbk[p] = (uint16_t)bk;
            ++C.hist[(size_t)key * kBuckets + bk];
            KeyClass &kc = C.key[key];
            if (kc.first == INT_MAX) {
                kc.first = p;
                kc.W = (int8_t)W;
                kc.wide = (int8_t)wide;
                kc.w32 = (int8_t)w32;
                kc.pk = (int8_t)pk;
                kc.warp = (int8_t)warp;
            }
            kc.n1max = std::max(kc.n1max, g1.n);
            kc.m1max = std::max(kc.m1max, g1.m);
            kc.n2max = std::max(kc.n2max, g2.n);
            kc.kmax = std::max(kc.kmax, kp);
            kc.bmin = std::min(kc.bmin, bk);
            kc.bmax = std::max(kc.bmax, bk);
            C.maps += g1.n;
        }
    });
    if (ferr.idx != INT64_MAX) return ferr.report();
    // combine: classes in order of first appearance, their statistics, and the output position
    // of every (chunk, class, bucket) run: buckets ascending, then chunks, then pair order
    int cls_of[kKeys];
    {
        KeyClass all[kKeys];
        for (const PairChunk &C : pcs)
            for (int k = 0; k < kKeys; ++k) {
                const KeyClass &x = C.key[k];
                if (x.first == INT_MAX) continue;
                KeyClass &y = all[k];
                if (x.first < y.first) {
                    y.first = x.first;
                    y.W = x.W;
                    y.wide = x.wide;
                    y.w32 = x.w32;
                    y.pk = x.pk;
                    y.warp = x.warp;
                }
                y.n1max = std::max(y.n1max, x.n1max);
                y.m1max = std::max(y.m1max, x.m1max);
                y.n2max = std::max(y.n2max, x.n2max);
                y.kmax = std::max(y.kmax, x.kmax);
                y.bmin = std::min(y.bmin, x.bmin);
                y.bmax = std::max(y.bmax, x.bmax);
            }
        int keys[kKeys], nk = 0;
        for (int k = 0; k < kKeys; ++k) {
            cls_of[k] = -1;
            if (all[k].first != INT_MAX) keys[nk++] = k;
        }
        std::sort(keys, keys + nk, [&](int x, int y) { return all[x].first < all[y].first; });
        for (int ci = 0; ci < nk; ++ci) {
            const int k = keys[ci];
            const KeyClass &y = all[k];
            cls_of[k] = ci;
            ClassPlan cp;
            cp.W = y.W;
            cp.wide = y.wide || y.W >= 8;
            cp.w32 = y.w32;
            cp.pk = y.pk;
            cp.warp = y.warp;
            cp.n1max = y.n1max;
            cp.m1max = y.m1max;
            cp.n2max = y.n2max;
            cp.kmax = y.kmax;
            int32_t run = 0;
            for (int bk = y.bmin; bk <= y.bmax; ++bk)
                for (PairChunk &C : pcs) {
                    int32_t &slot = C.hist[(size_t)k * kBuckets + bk];
                    const int32_t cnt = slot;
                    slot = run;
                    run += cnt;
                }
            cp.order.resize((size_t)run);
            b.classes.push_back(std::move(cp));
        }
    }
    int64_t mtot = 0;
    for (PairChunk &C : pcs) {
        const int64_t t = C.maps;
        C.maps = mtot;
        mtot += t;
    }
    b.map_total = mtot;
    for (auto &cp : b.classes) {
        int rc = tune_class(h, cp, B, opt.block_threads, opt.max_sms, opt.cluster);
        if (rc) return rc;
    }
    if ((int)b.classes.size() > kMaxClasses)
        return set_error(FASTGED_ERR_INVALID_ARG, "too many size classes");
    // very wide beams: fewer resident teams, so that their global scratch stays within half
    // of the free device memory (each team still solves its pairs one after another)
    {
        size_t fr = 0, tot = 0, need = 0;
        for (const auto &cp : b.classes)
            need += (size_t)cp.lay.slice_bytes * (size_t)(cp.grid / cp.cluster);
        if (need > 0 && cudaMemGetInfo(&fr, &tot) == cudaSuccess && need > fr / 2) {
            const double f = (double)(fr / 2) / (double)need;
            for (auto &cp : b.classes) {
                const int teams = std::max(1, (int)((double)(cp.grid / cp.cluster) * f));
                cp.grid = teams * cp.cluster;
            }
        }
    }

    // staging layout (one pinned buffer, one copy)
    size_t o = 0;
    b.off_meta = o;   o = align_up(o + sizeof(GraphMeta) * (size_t)ng, 256);
    b.off_vlab = o;   o = align_up(o + 4 * (size_t)nv, 256);
    b.off_edges = o;  o = align_up(o + 8 * (size_t)ne, 256);
    b.off_elab = o;   o = align_up(o + (b.labelled ? 4 * (size_t)ne : 0), 256);
    b.off_pairs = o;  o = align_up(o + 8 * (size_t)np, 256);
    b.off_order = o;  o = align_up(o + 4 * (size_t)np, 256);
    b.off_mapoff = o; o = align_up(o + 8 * (size_t)np, 256);
    b.off_kpp = o;    o = align_up(o + (kpp ? 4 * (size_t)np : 0), 256);
    b.in_bytes = o;
    // device work region: [status | cost | nevals | map] then pools, queues, scratch
    size_t w = 0;
    b.woff_err = w;    w = align_up(w + 16, 256);
    b.woff_cost = w;   w = align_up(w + 4 * (size_t)np, 256);
    b.woff_nev = w;    w = align_up(w + 8 * (size_t)np, 256);
    b.woff_map = w;    w = align_up(w + 4 * (size_t)mtot, 256);
    b.out_bytes = w;   // one device-to-host copy covers [0, out_bytes)
    b.woff_queue = w;  w = align_up(w + 4 * ((size_t)np + kMaxClasses), 256);
    b.woff_pool = w;   w = align_up(w + 8 * (size_t)(b.adj_words + b.plane_words), 256);
    size_t scratch = 0;
    int64_t q = 0;
    for (auto &cp : b.classes) {
        cp.scratch_off = scratch;
        scratch += align_up((size_t)cp.lay.slice_bytes * (size_t)(cp.grid / cp.cluster), 256);
        cp.order_off = q;
        q += (int64_t)cp.order.size();
    }
    b.woff_scratch = w; w += std::max<size_t>(scratch, 256);
    b.work_bytes = w;
    // the pinned staging buffer carries the inputs up and the results back
    int rc = h->pin.ensure(std::max<size_t>(std::max(b.in_bytes, b.out_bytes), 256), true);
    if (rc) return rc;
    uint8_t *S = (uint8_t *)h->pin.p;
    GraphMeta *smeta = (GraphMeta *)(S + b.off_meta);
    int32_t *vl = (int32_t *)(S + b.off_vlab);
    int32_t *ed = (int32_t *)(S + b.off_edges);
    int32_t *el = (int32_t *)(S + b.off_elab);
    int32_t *sord = (int32_t *)(S + b.off_order);
    int64_t *smo = (int64_t *)(S + b.off_mapoff);
    // one pass over every chunk: a pair chunk places its pairs in their class order and sets
    // their map offsets; a graph chunk sets the pool offsets of its graphs and stages their
    // labels and edges (checking every endpoint)
    pool.parallel_for((int64_t)npc + ngc, 1, [&](int64_t lo, int64_t hi) {
        for (int64_t u = lo; u < hi; ++u) {
            if (u < npc) {
                PairChunk &C = pcs[u];
                int64_t mo = C.maps;
                const int p1 = (int)std::min<int64_t>(np, (u + 1) * pch);
                for (int p = (int)(u * pch); p < p1; ++p) {
                    b.map_off[p] = mo;
                    smo[p] = mo;
                    mo += b.meta[pl->pairs[2 * p]].n;
                    const int key = pkey[p];
                    ClassPlan &cp = b.classes[cls_of[key]];
                    const int32_t pos = C.hist[(size_t)key * kBuckets + pbk[p]]++;
                    cp.order[pos] = p;
                    sord[cp.order_off + pos] = p;
                }
                continue;
            }
            const int64_t gi = u - npc;
            const GraphChunk &C = gcs[gi];
            int64_t lab = C.nv, eo = C.ne, aw = C.adjw;
            const int g1 = (int)std::min<int64_t>(ng, (gi + 1) * gch);
            for (int g = (int)(gi * gch); g < g1; ++g) {
                const fastged_graph &G = pl->graphs[g];
                GraphMeta &M = b.meta[g];
                M.lab_off = lab;
                M.edge_off = eo;
                M.adj_off = aw;
                M.plane_off = aw * B;
                lab += M.n;
                eo += M.m;
                aw += (int64_t)M.n * M.W;
                smeta[g] = M;
                if (G.n) memcpy(vl + M.lab_off, G.vlabel, 4 * (size_t)G.n);
                int32_t *dst = ed + 2 * M.edge_off;
                const unsigned n = (unsigned)G.n;
                bool bad = false;
                for (int k = 0; k < G.m; ++k) {
                    const int32_t x = G.edges[2 * k], y = G.edges[2 * k + 1];
                    bad |= ((unsigned)x >= n) | ((unsigned)y >= n) | (x == y);
                    dst[2 * k] = x;
                    dst[2 * k + 1] = y;
                }
                if (bad) {
                    ferr.put(g, "graph " + std::to_string(g) + ": bad edge endpoint or self-loop");
                    break;
                }
                if (b.labelled) {
                    if (G.elabel) memcpy(el + M.edge_off, G.elabel, 4 * (size_t)G.m);
                    else memset(el + M.edge_off, 0, 4 * (size_t)G.m);
                }
            }
        }
    });
    if (ferr.idx != INT64_MAX) return ferr.report();
    if (opt.vertex_order == FASTGED_ORDER_DEGREE) {
        b.perm.assign((size_t)mtot, 0);
        const int ng0 = (int)ro.copy_of.size();
        for (int p = 0; p < np; ++p) {
            const int cc = pl->pairs[2 * p] - ng0;
            if (cc < 0) continue;   // no copy: the source graph fails validation above
            std::copy(ro.perm[cc].begin(), ro.perm[cc].end(), b.perm.begin() + b.map_off[p]);
        }
    }
    memcpy(S + b.off_pairs, pl->pairs, 8 * (size_t)np);
    if (kpp) memcpy(S + b.off_kpp, kpp, 4 * (size_t)np);

    return FASTGED_OK;
}

#ifdef FASTGED_PHASE_TIMERS
// profiling builds only: per-phase cycle counters summed over every team
static unsigned long long *g_phase_dev = nullptr;

extern "C" int fastged_debug_phase_cycles(unsigned long long *out, int reset)
{
    if (!g_phase_dev) return -3;
    if (cudaMemcpy(out, g_phase_dev, 128, cudaMemcpyDeviceToHost) != cudaSuccess) return -3;
    if (reset) cudaMemset(g_phase_dev, 0, 128);
    return 0;
}
#endif

// Fills the kernel parameters of class k for a batch whose inputs sit at `in` and whose
// work region sits at `wk` on the device.
static KParams make_params(const fastged_handle *h, const Batch &b, int k, uint8_t *in,
                           uint8_t *wk)
{
    const ClassPlan &cp = b.classes[k];
    KParams p;
    memset(&p, 0, sizeof(p));
    p.gmeta = (const GraphMeta *)(in + b.off_meta);
    p.adj = (const uint64_t *)(wk + b.woff_pool);
    p.planes = (const uint64_t *)(wk + b.woff_pool) + b.adj_words;
    p.vlab = (const int32_t *)(in + b.off_vlab);
    p.pairs = (const int32_t *)(in + b.off_pairs);
    p.order = (const int32_t *)(in + b.off_order) + cp.order_off;
    p.n_order = (int32_t)cp.order.size();
    p.kpp = b.has_kpp ? (const int32_t *)(in + b.off_kpp) : nullptr;
    p.K = b.K;
    p.hwin = b.opt.hist_window ? b.opt.hist_window : (cp.warp ? kWarpHist : kHistMax);
    p.variant = b.opt.variant;
    p.cost.vsub = h->cost.v_sub;
    p.cost.vdel = h->cost.v_del;
    p.cost.vins = h->cost.v_ins;
    p.cost.esub = h->cost.e_sub;
    p.cost.edel = h->cost.e_del;
    p.cost.eins = h->cost.e_ins;
    p.queue_head = (int32_t *)(wk + b.woff_queue) + k;
    p.err = (int32_t *)(wk + b.woff_err);
    p.out_cost = (int32_t *)(wk + b.woff_cost);
    p.out_map = (int32_t *)(wk + b.woff_map);
    p.map_off = (const int64_t *)(in + b.off_mapoff);
    p.out_nevals = (int64_t *)(wk + b.woff_nev);
    p.gscratch = wk + b.woff_scratch + cp.scratch_off;
    p.lay = cp.lay;
    p.wl = cp.wl;
    p.n_graphs = b.n_graphs;
    p.n_pairs = b.n_pairs;
    p.n_vlab = b.n_vlab;
    p.adj_words = b.adj_words;
    p.plane_words = b.plane_words;
    p.map_total = b.map_total;
#ifdef FASTGED_PHASE_TIMERS
    if (!g_phase_dev && cudaMalloc(&g_phase_dev, 128) == cudaSuccess) cudaMemset(g_phase_dev, 0, 128);
    p.phase_cycles = g_phase_dev;
#endif
    return p;
}

// Creates the class streams a batch of nc size classes runs on (once per handle; never
// inside a stream capture).
static int ensure_class_streams(fastged_handle *h, int nc)
{
    if (nc < 2) return FASTGED_OK;
    for (int k = 0; k < nc && k < kMaxClasses; ++k) {
        if (h->class_stream[k]) continue;
        const cudaError_t e = cudaStreamCreateWithFlags(&h->class_stream[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            h->class_stream[k] = nullptr;
            return cuda_fail(e, "class stream creation");
        }
    }
    return FASTGED_OK;
}

// Enqueues the device path of a batch: zero pools and queues, pack, one launch per class.
int fastged::enqueue(fastged_handle *h, const Batch &b, uint8_t *in, uint8_t *wk,
                     cudaStream_t st, int *launches, cudaEvent_t t0, cudaEvent_t t1,
                     bool capturing)
{
    // inside stream capture the timing events must become graph nodes
    const unsigned evflag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    int nl = 0;
    CK(cudaMemsetAsync(wk + b.woff_err, 0, 16, st));
    CK(cudaMemsetAsync(wk + b.woff_queue, 0, b.woff_scratch - b.woff_queue, st));
    PackParams pp;
    pp.gmeta = (const GraphMeta *)(in + b.off_meta);
    pp.n_graphs = b.n_graphs;
    pp.edges = (const int32_t *)(in + b.off_edges);
    pp.elabel = b.labelled ? (const int32_t *)(in + b.off_elab) : nullptr;
    pp.B = b.B;
    pp.adj = (uint64_t *)(wk + b.woff_pool);
    pp.planes = (uint64_t *)(wk + b.woff_pool) + b.adj_words;
    pp.err = (int32_t *)(wk + b.woff_err);
    if (b.n_graphs > 0) {
        CK(launch_pack(pp, b.n_graphs, st));
        ++nl;
    }
    const int nc = (int)b.classes.size();
    if (inject_fire(FASTGED_INJECT_LAUNCH))
        return set_error(FASTGED_ERR_CUDA, "injected launch failure (no K-Best kernel launched)");
    if (t0) CK(cudaEventRecordWithFlags(t0, st, evflag));
    if (b.opt.form == FASTGED_FORM_PLAIN) {
        // one launch per pair, in pair order, single team, on the caller's stream
        std::vector<int> cls(b.n_pairs), pos(b.n_pairs);
        for (int k = 0; k < nc; ++k)
            for (size_t q = 0; q < b.classes[k].order.size(); ++q) {
                cls[b.classes[k].order[q]] = k;
                pos[b.classes[k].order[q]] = (int)q;
            }
        int32_t *qbase = (int32_t *)(wk + b.woff_queue) + kMaxClasses;
        for (int pr = 0; pr < b.n_pairs; ++pr) {
            const int k = cls[pr];
            const ClassPlan &cp = b.classes[k];
            KParams p = make_params(h, b, k, in, wk);
            p.order += pos[pr];
            p.n_order = 1;
            p.queue_head = qbase + pr;
            if (cp.warp)
                CK(launch_kbest_warp(cp.w32, label_instance(b.B), p, 1, 32, (size_t)cp.wl.warp_bytes,
                                     st));
            else if (cp.cluster > 1)
                CK(launch_kbest_cluster(cp.W, cp.wide, label_instance(b.B), p, cp.cluster, cp.block, cp.smem,
                                        cp.cluster, st));
            else
                CK(launch_kbest(cp.W, cp.wide, cp.w32, cp.all_smem, label_instance(b.B), p, 1,
                                cp.block, cp.smem, st));
            ++nl;
        }
    } else if (nc == 1) {
        const ClassPlan &cp = b.classes[0];
        KParams p = make_params(h, b, 0, in, wk);
        if (cp.warp)
            CK(launch_kbest_warp(cp.w32, label_instance(b.B), p, cp.grid, cp.block, cp.smem, st));
        else if (cp.cluster > 1)
            CK(launch_kbest_cluster(cp.W, cp.wide, label_instance(b.B), p, cp.grid, cp.block, cp.smem,
                                    cp.cluster, st));
        else
            CK(launch_kbest(cp.W, cp.wide, cp.w32, cp.all_smem, label_instance(b.B), p, cp.grid,
                            cp.block, cp.smem, st));
        ++nl;
    } else if (nc > 1) {
        for (int k = 0; k < nc; ++k)
            if (!h->class_stream[k]) return set_error(FASTGED_ERR_CUDA, "class stream missing");
        CK(cudaEventRecord(h->ev[kMaxClasses], st));
        for (int k = 0; k < nc; ++k) {
            const ClassPlan &cp = b.classes[k];
            CK(cudaStreamWaitEvent(h->class_stream[k], h->ev[kMaxClasses], 0));
            KParams p = make_params(h, b, k, in, wk);
            if (cp.warp)
                CK(launch_kbest_warp(cp.w32, label_instance(b.B), p, cp.grid, cp.block, cp.smem,
                                     h->class_stream[k]));
            else if (cp.cluster > 1)
                CK(launch_kbest_cluster(cp.W, cp.wide, label_instance(b.B), p, cp.grid, cp.block, cp.smem,
                                        cp.cluster, h->class_stream[k]));
            else
                CK(launch_kbest(cp.W, cp.wide, cp.w32, cp.all_smem, label_instance(b.B), p,
                                cp.grid, cp.block, cp.smem, h->class_stream[k]));
            ++nl;
            CK(cudaEventRecord(h->ev[k], h->class_stream[k]));
            CK(cudaStreamWaitEvent(st, h->ev[k], 0));
        }
    }
    if (t1) CK(cudaEventRecordWithFlags(t1, st, evflag));
    if (launches) *launches = nl;
    return FASTGED_OK;
}

int fastged::finish_outputs(const Batch &b, const uint8_t *host_out, int32_t *out_cost,
                            int32_t *out_mapping, int64_t *out_nevals)
{
    NvtxRange r("fastged results");
    const int32_t err = *(const int32_t *)(host_out + b.woff_err);
    if (err & kErrDuplicateEdge) return set_error(FASTGED_ERR_INVALID_ARG, "duplicate edge in a graph");
    if (err & kErrBounds) {
        const int32_t line = ((const int32_t *)(host_out + b.woff_err))[2];
        return set_error(FASTGED_ERR_CUDA, "device bounds check failed (first at source line " +
                                               std::to_string(line) + ")");
    }
    if (err) return set_error(FASTGED_ERR_CUDA, "device error flag " + std::to_string(err));
    if (out_cost) memcpy(out_cost, host_out + b.woff_cost, 4 * (size_t)b.n_pairs);
    if (out_nevals) memcpy(out_nevals, host_out + b.woff_nev, 8 * (size_t)b.n_pairs);
    if (out_mapping) {
        const int32_t *res = (const int32_t *)(host_out + b.woff_map);
        if (b.perm.empty()) {
            memcpy(out_mapping, res, 4 * (size_t)b.map_total);
        } else {
            // level k branched source vertex perm[k]: return the map in source index order
            for (int p = 0; p < b.n_pairs; ++p) {
                const int64_t o = b.map_off[p];
                const int64_t e = p + 1 < b.n_pairs ? b.map_off[p + 1] : b.map_total;
                for (int64_t k = o; k < e; ++k) out_mapping[o + b.perm[k]] = res[k];
            }
        }
    }
    return FASTGED_OK;
}

// ------------------------------------------------------------------------------------
// one-shot batch
// ------------------------------------------------------------------------------------
// A batch that timed out may still be running on the handle's stream and writing into its
// buffers: wait for it before they are reused.
static void drain(fastged_handle *h)
{
    if (!h->inflight) return;
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    h->inflight = false;
}

int fastged::batch_enqueue(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                           const fastged_options &o)
{
    drain(h);
    Batch &b = h->batch;
    int rc;
    {
        NvtxRange r("fastged flatten");
        rc = flatten(h, pairs, K, o, b);
    }
    if (rc) return rc;
    if (b.n_pairs == 0) return FASTGED_OK;
    if ((rc = ensure_class_streams(h, (int)b.classes.size()))) return rc;
    NvtxRange r("fastged upload + launch");
    cudaStream_t st = h->stream;
    if ((rc = h->dev_in.ensure(b.in_bytes, st, true))) return rc;
    if ((rc = h->dev_work.ensure(b.work_bytes, st, true))) return rc;
    CK(cudaMemcpyAsync(h->dev_in.p, h->pin.p, b.in_bytes, cudaMemcpyHostToDevice, st));
    rc = enqueue(h, b, (uint8_t *)h->dev_in.p, (uint8_t *)h->dev_work.p, st, nullptr);
    if (rc) return rc;
    // results come back through the (already consumed) staging buffer
    CK(cudaMemcpyAsync(h->pin.p, h->dev_work.p, b.out_bytes, cudaMemcpyDeviceToHost, st));
    return FASTGED_OK;
}

int fastged::batch_results(fastged_handle *h, int32_t *out_cost, int32_t *out_mapping,
                           int64_t *out_nevals)
{
    if (h->batch.n_pairs == 0) return FASTGED_OK;
    return finish_outputs(h->batch, (const uint8_t *)h->pin.p, out_cost, out_mapping, out_nevals);
}

extern "C" int fastged_batch_ex(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                                const fastged_options *opt, int32_t *out_cost,
                                int32_t *out_mapping, int64_t *out_nevals)
{
    clear_error();
    if (!h) return set_error(FASTGED_ERR_INVALID_ARG, "null handle");
    const fastged_options o = opt ? *opt : default_options();
    int rc = batch_enqueue(h, pairs, K, o);
    if (rc) {
        // work enqueued before the failure must finish before the buffers are reused
        cudaStreamSynchronize(h->stream);
        cudaGetLastError();
        return rc;
    }
    if (h->timeout_ms > 0) {
        CK(cudaEventRecord(h->done, h->stream));
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            const cudaError_t q = cudaEventQuery(h->done);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return cuda_fail(q, "batch");
            if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(h->timeout_ms)) {
                h->inflight = true;
                return set_error(FASTGED_ERR_TIMEOUT,
                                 "batch exceeded the handle's timeout; it finishes in the background");
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    } else {
        CK(cudaStreamSynchronize(h->stream));
    }
    return batch_results(h, out_cost, out_mapping, out_nevals);
}

extern "C" int fastged_batch(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                             int32_t *out_cost, int32_t *out_mapping)
{
    return fastged_batch_ex(h, pairs, K, nullptr, out_cost, out_mapping, nullptr);
}

// ------------------------------------------------------------------------------------
// device-resident plans
// ------------------------------------------------------------------------------------
// Times every team shape of every size class the table does not know yet, on a sample of
// that class's pairs (each shape run twice, the faster run counts), and records the best.
static int autotune_batch(fastged_handle *h, const fastged_pair_list *pl, int32_t K,
                          const fastged_options &o)
{
    Batch probe;
    int rc = flatten(h, pl, K, o, probe);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(FASTGED_ERR_CUDA, "event creation");
    for (const ClassPlan &cp : probe.classes) {
        const int npairs = (int)cp.order.size();
        const std::string key = class_key(cp, probe.B, npairs, h->sm_count);
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            tune_load_locked();
            auto it = g_tune.find(key);
            if (it != g_tune.end()) continue;
        }
        std::vector<TuneChoice> cands;
        if (cp.warp) {
            // two or four warps per CTA (one-warp CTAs run into the SM's CTA limit when
            // several classes share the GPU)
            for (int gm : {0, 1})
                for (int bt : {64, 128}) {
                    TuneChoice c;
                    c.block = bt;
                    c.gmap = gm;
                    cands.push_back(c);
                }
        } else if (cluster_eligible(cp, npairs, h->sm_count)) {
            for (int cl : {1, 2, 4, 8, 16}) {
                TuneChoice c;
                c.block = cl == 1 ? 256 : 512;
                c.cluster = cl;
                cands.push_back(c);
            }
        } else {
            for (int bt : {128, 256, 512}) {
                TuneChoice c;
                c.block = bt;
                cands.push_back(c);
            }
        }
        // the class's pairs, strided down to a sample that fills every candidate's teams
        // several times over (a sample near one wave of teams is decided by its tail)
        const int cap = std::max(1, 32 * h->sm_count);
        const int step = std::max(1, npairs / cap);
        std::vector<int32_t> sub_pairs, sub_kpp;
        for (int q = 0; q < npairs; q += step) {
            const int pidx = cp.order[q];
            sub_pairs.push_back(pl->pairs[2 * pidx]);
            sub_pairs.push_back(pl->pairs[2 * pidx + 1]);
            if (o.k_per_pair) sub_kpp.push_back(o.k_per_pair[pidx]);
        }
        fastged_pair_list sub = *pl;
        sub.n_pairs = (int32_t)(sub_pairs.size() / 2);
        sub.pairs = sub_pairs.data();
        fastged_options so = o;
        so.k_per_pair = o.k_per_pair ? sub_kpp.data() : nullptr;
        so.form = FASTGED_FORM_BATCHED;
        TuneChoice best;
        double best_ms = 1e30;
        for (const TuneChoice &c : cands) {
            double ms_c = 1e30;
            for (int rep = 0; rep < 2; ++rep) {
                {
                    std::lock_guard<std::mutex> g(g_tune_mu);
                    g_tune_force = c;
                    g_tune_forcing = true;
                }
                cudaEventRecord(e0, h->stream);
                rc = batch_enqueue(h, &sub, K, so);
                cudaEventRecord(e1, h->stream);
                const cudaError_t se = cudaStreamSynchronize(h->stream);
                {
                    std::lock_guard<std::mutex> g(g_tune_mu);
                    g_tune_forcing = false;
                }
                if (rc || se != cudaSuccess) break;   // a shape that cannot run is skipped
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_c = std::min(ms_c, (double)ms);
            }
            if (rc) {
                rc = FASTGED_OK;
                clear_error();
                continue;
            }
            if (ms_c < best_ms) {
                best_ms = ms_c;
                best = c;
            }
        }
        if (best_ms < 1e30) tune_store(key, best, best_ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return FASTGED_OK;
}

extern "C" int fastged_plan_create(fastged_handle *h, const fastged_pair_list *pairs,
                                   int32_t K, const fastged_options *opt, fastged_plan **out)
{
    clear_error();
    if (!h || !out) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    drain(h);
    const fastged_options o = opt ? *opt : default_options();
    if (o.autotune && o.block_threads == 0) {
        const int rc = autotune_batch(h, pairs, K, o);
        if (rc) return rc;
    }
    fastged_plan *p = new fastged_plan();
    p->h = h;
    int rc = flatten(h, pairs, K, o, p->b);
    if (rc) { delete p; return rc; }
    p->b.opt.k_per_pair = nullptr;   // copied into the staging buffer; never dereferenced
    if ((rc = ensure_class_streams(h, (int)p->b.classes.size()))) {
        delete p;
        return rc;
    }
    // exact sizes, allocated on the handle's stream, which is idle: the upload below starts
    // once that stream has caught up
    if ((rc = p->dev_in.ensure(std::max<size_t>(p->b.in_bytes, 256), h->stream, false)) ||
        (rc = p->dev_work.ensure(p->b.work_bytes, h->stream, false)) ||
        (rc = p->pin_out.ensure(std::max<size_t>(p->b.out_bytes, 256), false))) {
        fastged_plan_destroy(p);
        return rc;
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->dev_in.p, h->pin.p, p->b.in_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&p->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->t1);
    if (e != cudaSuccess) {
        fastged_plan_destroy(p);
        return cuda_fail(e, "plan upload");
    }
    p->use_graph = o.use_cuda_graph != 0 && o.form != FASTGED_FORM_PLAIN;
    *out = p;
    return FASTGED_OK;
}

extern "C" int fastged_plan_run(fastged_plan *p, void *stream)
{
    clear_error();
    if (!p) return set_error(FASTGED_ERR_INVALID_ARG, "null plan");
    const Batch &b = p->b;
    NvtxRange r("fastged plan run");
    cudaStream_t st = stream ? (cudaStream_t)stream : p->stream;
    p->last_stream = st;
    if (b.n_pairs == 0) return FASTGED_OK;
    uint8_t *in = (uint8_t *)p->dev_in.p, *wk = (uint8_t *)p->dev_work.p;
    if (!p->use_graph) {
        int nl = 0;
        int rc = enqueue(p->h, b, in, wk, st, &nl, p->t0, p->t1);
        p->launches = nl;
        return rc;
    }
    if (!p->exec) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
        int nl = 0;
        int rc = enqueue(p->h, b, in, wk, p->stream, &nl, p->t0, p->t1, true);
        cudaError_t e = cudaStreamEndCapture(p->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&p->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { p->exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
        p->launches = nl;
    }
    CK(cudaGraphLaunch(p->exec, st));
    return FASTGED_OK;
}

extern "C" int fastged_plan_read(fastged_plan *p, int32_t *out_cost, int32_t *out_mapping,
                                 int64_t *out_nevals)
{
    clear_error();
    if (!p) return set_error(FASTGED_ERR_INVALID_ARG, "null plan");
    const Batch &b = p->b;
    if (b.n_pairs == 0) return FASTGED_OK;
    cudaStream_t st = p->last_stream ? p->last_stream : p->stream;
    CK(cudaMemcpyAsync(p->pin_out.p, p->dev_work.p, b.out_bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return finish_outputs(b, (const uint8_t *)p->pin_out.p, out_cost, out_mapping, out_nevals);
}

extern "C" int fastged_plan_info(const fastged_plan *p, fastged_plan_stats *out)
{
    clear_error();
    if (!p || !out) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    memset(out, 0, sizeof(*out));
    const Batch &b = p->b;
    out->n_pairs = b.n_pairs;
    out->n_classes = (int32_t)b.classes.size();
    out->launches_per_run = p->launches;
    out->graph_replay = p->use_graph ? 1 : 0;
    out->input_bytes = (int64_t)b.in_bytes;
    out->device_bytes = (int64_t)(b.in_bytes + b.work_bytes);
    out->output_bytes = (int64_t)b.out_bytes;
    for (size_t k = 0; k < b.classes.size() && k < 8; ++k) {
        out->block_threads[k] = b.classes[k].block;
        out->grid[k] = b.classes[k].grid;
        out->words[k] = b.classes[k].W;
        out->smem_bytes[k] = (int32_t)b.classes[k].smem;
    }
    return FASTGED_OK;
}

extern "C" int fastged_plan_kernel_ms(fastged_plan *p, float *ms)
{
    clear_error();
    if (!p || !ms) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    *ms = 0.f;
    if (p->b.n_pairs == 0) return FASTGED_OK;
    CK(cudaEventSynchronize(p->t1));
    CK(cudaEventElapsedTime(ms, p->t0, p->t1));
    return FASTGED_OK;
}

extern "C" void fastged_plan_destroy(fastged_plan *p)
{
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->last_stream && p->last_stream != p->stream) cudaStreamSynchronize(p->last_stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->t0) cudaEventDestroy(p->t0);
    if (p->t1) cudaEventDestroy(p->t1);
    p->dev_in.release();
    p->dev_work.release();
    p->pin_out.release();
    delete p;
}
