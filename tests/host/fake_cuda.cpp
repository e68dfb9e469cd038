// Test infrastructure: host-only fakes of the CUDA runtime calls and of the kernel-side
// entry points that the host runtime (fastged_runtime.cu) references, so that its host logic
// (validation, size classes, pair order, staging layout, memory caps, error paths) can be
// exercised on a machine without a GPU. Nothing here launches or imitates a kernel: launches
// succeed without doing anything, and the tests only read what the host side produced.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "fastged_internal.h"
#include "fastged_runtime.h"

static size_t g_free_bytes = (size_t)250 << 30;   // reported by cudaMemGetInfo
static int g_fail_pinned = 0;                       // next cudaMallocHost calls that fail

extern "C" void fake_set_free_bytes(unsigned long long b) { g_free_bytes = (size_t)b; }
extern "C" void fake_fail_pinned_alloc(int n) { g_fail_pinned = n; }

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
cudaError_t cudaMalloc(void **p, size_t n)
{
    *p = malloc(n ? n : 1);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p)
{
    free(p);
    return cudaSuccess;
}
cudaError_t cudaMemGetInfo(size_t *f, size_t *t)
{
    *f = g_free_bytes;
    *t = (size_t)280 << 30;
    return cudaSuccess;
}
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr, int)
{
    *v = 0;
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
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t, cudaEvent_t) { *ms = 0.f; return cudaSuccess; }
cudaError_t cudaEventQuery(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventRecordWithFlags(cudaEvent_t, cudaStream_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
cudaError_t cudaGraphInstantiate(cudaGraphExec_t *g, cudaGraph_t, unsigned long long) { *g = nullptr; return cudaSuccess; }
cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaMemcpy(void *, const void *, size_t, cudaMemcpyKind) { return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void *, const void *, size_t, cudaMemcpyKind, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaMemsetAsync(void *, int, size_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamBeginCapture(cudaStream_t, cudaStreamCaptureMode) { return cudaSuccess; }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned int) { *s = nullptr; return cudaSuccess; }
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t *g) { *g = nullptr; return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
}

// kernel-side entry points: every team shape fits twice per SM; cluster variants exist where
// the real library has them (two-word classes with narrow maps, wide-map classes of four or
// more words)
namespace fastged {
cudaError_t launch_pack(const PackParams &, int, cudaStream_t) { return cudaSuccess; }
cudaError_t launch_kbest(int, bool, bool, bool, int, const KParams &, int, int, size_t, cudaStream_t)
{
    return cudaSuccess;
}
cudaError_t launch_kbest_cluster(int, int, const KParams &, int, int, size_t, int, cudaStream_t)
{
    return cudaSuccess;
}
cudaError_t kbest_occupancy(int, bool, bool, bool, int, int, size_t, int *out)
{
    *out = 2;
    return cudaSuccess;
}
cudaError_t kbest_cluster_occupancy(int, int, int, size_t, int cluster, int *out)
{
    *out = 152 / cluster;
    return cudaSuccess;
}
bool kbest_has_smem_variant(int, bool, bool) { return true; }
bool kbest_has_cluster_variant(int W, bool wide, bool w32)
{
    return !w32 && ((wide && W >= 4) || (W == 2 && !wide));
}
size_t team_shared_static_bytes() { return 2048; }
size_t team_shared_cluster_bytes() { return 4096; }
}  // namespace fastged
