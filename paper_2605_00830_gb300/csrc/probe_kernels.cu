// probe_kernels.cu -- integer-pipe throughput probes (the ALU roofline of the GED path).
//
// The successor evaluation is pure 32-bit integer work: logic ops (LOP3), adds (IADD3) and
// population counts (POPC). These kernels issue long independent chains of exactly those
// instructions from every SM (inline PTX so that nothing is folded away) and report the
// device-wide rate, which serves as the measured peak for the roofline fraction.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fastged.h"
#include "fastged_runtime.h"

namespace fastged {

template <int KIND>
__global__ void __launch_bounds__(256) int_probe(uint32_t *out, int iters, uint32_t seed)
{
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed ^ (threadIdx.x * 2654435761u + k * 40503u + blockIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (KIND == 0) {        // logic: a_k = a_k ^ (a_{k+1} & ~a_{k+2})
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0xD2;"
                                 : "+r"(a[k]) : "r"(a[(k + 1) & 7]), "r"(a[(k + 2) & 7]));
                } else if (KIND == 1) { // add
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(a[(k + 3) & 7]));
                } else {                // population count
                    asm volatile("popc.b32 %0, %0;" : "+r"(a[k]));
                }
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) x ^= a[k];
    if (x == 0x9E3779B9u) out[blockIdx.x] = x;   // practically never; keeps the chains live
}

}  // namespace fastged

using namespace fastged;

// Measures device-wide 32-bit LOP3, IADD and POPC rates (instructions x lanes per second).
extern "C" int fastged_measure_int_peak(double *lop3_per_s, double *iadd_per_s,
                                        double *popc_per_s)
{
    clear_error();
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(FASTGED_ERR_CUDA, "no device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * 4096) != cudaSuccess)
        return set_error(FASTGED_ERR_OOM, "probe buffer");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int block = 256, grid = sms * 8, iters = 4096;
    double rate[3] = {0, 0, 0};
    for (int kind = 0; kind < 3; ++kind) {
        for (int rep = 0; rep < 3; ++rep) {   // first launch warms up clocks
            cudaEventRecord(e0);
            if (kind == 0) int_probe<0><<<grid, block>>>(out, iters, 12345u);
            else if (kind == 1) int_probe<1><<<grid, block>>>(out, iters, 12345u);
            else int_probe<2><<<grid, block>>>(out, iters, 12345u);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double ops = (double)grid * block * iters * 16.0 * 8.0;
            const double r = ops / (ms * 1e-3);
            if (r > rate[kind]) rate[kind] = r;
        }
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return set_error(FASTGED_ERR_CUDA, cudaGetErrorString(e));
    if (lop3_per_s) *lop3_per_s = rate[0];
    if (iadd_per_s) *iadd_per_s = rate[1];
    if (popc_per_s) *popc_per_s = rate[2];
    return FASTGED_OK;
}
