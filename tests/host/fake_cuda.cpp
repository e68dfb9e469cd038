// Test infrastructure: host-only fakes of the CUDA runtime calls and of the kernel-side
// entry points that the host runtime (fastged_runtime.cu, serve.cu) references, so that its
// host logic (validation, size classes, pair order, staging layout, memory caps, the serving
// dispatcher, error paths) can be exercised on a machine without a GPU. Nothing here launches
// or imitates a kernel: launches succeed without doing anything, device-to-host copies deliver
// zeros (an all-clear status word and zero results), and host functions enqueued on a stream
// run on one executor thread after a configurable delay, the time a batch would take.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "fastged_internal.h"
#include "fastged_runtime.h"

static size_t g_free_bytes = (size_t)250 << 30;   // reported by cudaMemGetInfo
static int g_fail_pinned = 0;                       // next cudaMallocHost calls that fail

extern "C" void fake_set_free_bytes(unsigned long long b) { g_free_bytes = (size_t)b; }
extern "C" void fake_fail_pinned_alloc(int n) { g_fail_pinned = n; }

namespace {
// Host functions of every fake stream, run in enqueue order by one thread, each no earlier
// than `delay_us` after it was enqueued; a stream is idle when none of its host functions is
// queued or running. Created on first use and never destroyed (its thread is detached).
struct HostFnQueue {
    struct Item {
        cudaStream_t s;
        cudaHostFn_t fn;
        void *arg;
        std::chrono::steady_clock::time_point due;
    };
    std::mutex mu;
    std::condition_variable cv, idle_cv;
    std::deque<Item> q;
    std::map<cudaStream_t, int> busy;   // host functions queued or running, per stream
    std::atomic<int> delay_us{0};

    HostFnQueue() { std::thread([this] { run(); }).detach(); }
    void run()
    {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return !q.empty(); });
            const Item it = q.front();   // only this thread removes items
            lk.unlock();
            std::this_thread::sleep_until(it.due);
            it.fn(it.arg);
            lk.lock();
            q.pop_front();
            if (--busy[it.s] == 0) busy.erase(it.s);
            idle_cv.notify_all();
        }
    }
};
HostFnQueue &host_fns()
{
    static HostFnQueue *h = new HostFnQueue();
    return *h;
}
std::atomic<intptr_t> g_next_stream{1};
}  // namespace

extern "C" void fake_set_host_fn_delay_us(int us) { host_fns().delay_us.store(us); }

// The team shape of the last K-Best launch, the elapsed time an event pair reports for each
// shape (set by the test; 0 ms for shapes not set), and how many K-Best launches were made.
static std::mutex g_shape_mu;
static std::map<std::pair<int, int>, float> g_shape_ms;
static std::pair<int, int> g_last_shape{0, 1};
static std::atomic<long long> g_kbest_launches{0};
static void note_launch(int block, int cluster)
{
    std::lock_guard<std::mutex> g(g_shape_mu);
    g_last_shape = {block, cluster};
    ++g_kbest_launches;
}
extern "C" void fake_set_shape_ms(int block, int cluster, float ms)
{
    std::lock_guard<std::mutex> g(g_shape_mu);
    if (block == 0) g_shape_ms.clear();
    else g_shape_ms[{block, cluster}] = ms;
}
extern "C" long long fake_kbest_launches() { return g_kbest_launches.load(); }

// Events report "not ready" until this time: a batch that takes longer than a handle's
// timeout.
static std::atomic<long long> g_events_ready_at_us{0};
static long long now_us()
{
    return std::chrono::duration_cast<std::chrono::microseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}
extern "C" void fake_events_busy_for_ms(int ms) { g_events_ready_at_us.store(now_us() + 1000LL * ms); }

extern "C" {
cudaError_t cudaMallocHost(void **p, size_t n)
{
    if (g_fail_pinned > 0) {
        --g_fail_pinned;
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    *p = aligned_alloc(4096, (n + 4095) / 4096 * 4096);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFreeHost(void *p)
{
    free(p);
    return cudaSuccess;
}
static int g_fail_device = 0;                      // next cudaMalloc calls that fail
extern "C" void fake_fail_device_alloc(int n) { g_fail_device = n; }
cudaError_t cudaMalloc(void **p, size_t n)
{
    if (g_fail_device > 0) {
        --g_fail_device;
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    *p = malloc(n ? n : 1);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p)
{
    free(p);
    return cudaSuccess;
}
cudaError_t cudaMallocAsync(void **p, size_t n, cudaStream_t) { return cudaMalloc(p, n); }
cudaError_t cudaFreeAsync(void *p, cudaStream_t) { return cudaFree(p); }
cudaError_t cudaMemGetInfo(size_t *f, size_t *t)
{
    *f = g_free_bytes;
    *t = (size_t)280 << 30;
    return cudaSuccess;
}
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr a, int)
{
    // a GB300: 152 SMs, 227 KB of shared memory per block, 228 KB per SM
    *v = a == cudaDevAttrMultiProcessorCount              ? 152
         : a == cudaDevAttrMaxSharedMemoryPerBlockOptin    ? 232448
         : a == cudaDevAttrMaxSharedMemoryPerMultiprocessor ? 233472
                                                            : 0;
    return cudaSuccess;
}
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaLaunchHostFunc(cudaStream_t s, cudaHostFn_t fn, void *arg)
{
    HostFnQueue &h = host_fns();
    {
        std::lock_guard<std::mutex> g(h.mu);
        h.q.push_back({s, fn, arg,
                       std::chrono::steady_clock::now() + std::chrono::microseconds(h.delay_us.load())});
        ++h.busy[s];
    }
    h.cv.notify_all();
    return cudaSuccess;
}
cudaError_t cudaGetDevice(int *d)
{
    *d = 0;
    return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char *cudaGetErrorString(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? "out of memory (fake)" : "error (fake)";
}
cudaError_t cudaEventCreate(cudaEvent_t *e) { *e = nullptr; return cudaSuccess; }
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned int) { *e = nullptr; return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t, cudaEvent_t)
{
    std::lock_guard<std::mutex> g(g_shape_mu);
    auto it = g_shape_ms.find(g_last_shape);
    *ms = it == g_shape_ms.end() ? 0.f : it->second;
    return cudaSuccess;
}
cudaError_t cudaEventQuery(cudaEvent_t)
{
    return now_us() < g_events_ready_at_us.load() ? cudaErrorNotReady : cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventRecordWithFlags(cudaEvent_t, cudaStream_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
static char g_fake_graph[16];   // graph and executable handles: one non-null token
cudaError_t cudaGraphInstantiate(cudaGraphExec_t *g, cudaGraph_t, unsigned long long)
{
    *g = reinterpret_cast<cudaGraphExec_t>(g_fake_graph);
    return cudaSuccess;
}
cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaMemcpy(void *dst, const void *, size_t n, cudaMemcpyKind k)
{
    if (k == cudaMemcpyDeviceToHost) memset(dst, 0, n);
    return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void *dst, const void *, size_t n, cudaMemcpyKind k, cudaStream_t)
{
    if (k == cudaMemcpyDeviceToHost) memset(dst, 0, n);
    return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void *, int, size_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamBeginCapture(cudaStream_t, cudaStreamCaptureMode) { return cudaSuccess; }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned int)
{
    *s = reinterpret_cast<cudaStream_t>(16 * g_next_stream.fetch_add(1));
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t *g)
{
    *g = reinterpret_cast<cudaGraph_t>(g_fake_graph);
    return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t s)
{
    HostFnQueue &h = host_fns();
    std::unique_lock<std::mutex> lk(h.mu);
    h.idle_cv.wait(lk, [&] { return h.busy.find(s) == h.busy.end(); });
    return cudaSuccess;
}
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
}

// kernel-side entry points: every team shape fits twice per SM; cluster variants exist where
// the real library has them (two-word classes with narrow maps, wide-map classes of four or
// more words)
namespace fastged {
static std::atomic<int> g_max_pack_graphs{0};   // most graphs one batch packed
static std::atomic<int> g_fail_launches{0};     // next packing launches that fail
cudaError_t launch_pack(const PackParams &, int n_graphs, cudaStream_t)
{
    int f = g_fail_launches.load();
    while (f > 0 && !g_fail_launches.compare_exchange_weak(f, f - 1)) {
    }
    if (f > 0) return cudaErrorLaunchFailure;
    int m = g_max_pack_graphs.load();
    while (n_graphs > m && !g_max_pack_graphs.compare_exchange_weak(m, n_graphs)) {
    }
    return cudaSuccess;
}
cudaError_t launch_kbest(int, bool, bool, bool, int, const KParams &, int, int block, size_t,
                         cudaStream_t)
{
    note_launch(block, 1);
    return cudaSuccess;
}
cudaError_t launch_kbest_cluster(int, bool, int, const KParams &, int, int block, size_t, int cluster,
                                 cudaStream_t)
{
    note_launch(block, cluster);
    return cudaSuccess;
}
cudaError_t kbest_occupancy(int, bool, bool, bool, int, int, size_t, int *out)
{
    *out = 2;
    return cudaSuccess;
}
cudaError_t kbest_cluster_occupancy(int, bool, int, int, size_t, int cluster, int *out)
{
    *out = 152 / cluster;
    return cudaSuccess;
}
// one-warp launches report their vertex-map placement as cluster 100 + gmap
cudaError_t launch_kbest_warp(bool, int, const KParams &p, int, int block, size_t, cudaStream_t)
{
    note_launch(block, 100 + p.wl.gmap);
    return cudaSuccess;
}
cudaError_t kbest_warp_occupancy(bool, int, int block, size_t smem, int *out)
{
    // as many CTAs as fit the SM's 228 KB of shared memory and 64 warps
    const size_t by_smem = smem ? (233472 - 1024) / (smem + 1024) : 64;
    *out = (int)std::min<size_t>(by_smem, (size_t)(2048 / block));
    return cudaSuccess;
}
bool kbest_has_smem_variant(int, bool, bool) { return true; }
bool kbest_has_cluster_variant(int W, bool wide, bool w32)
{
    return !w32 && ((wide && W >= 4) || ((W == 2 || W == 4) && !wide));
}
size_t team_shared_static_bytes() { return 2048; }
size_t team_shared_cluster_bytes() { return 4096; }
}  // namespace fastged

// the most graphs one batch has packed since the last reset
extern "C" int fake_max_pack_graphs(int reset)
{
    return reset ? fastged::g_max_pack_graphs.exchange(0) : fastged::g_max_pack_graphs.load();
}

// the next n packing launches fail (a batch's launch error)
extern "C" void fake_fail_launches(int n) { fastged::g_fail_launches.store(n); }
