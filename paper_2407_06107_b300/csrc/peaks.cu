// Measured denominator of the gather roofline: the rate at which the SMs can read random,
// independent 32-byte sectors at L2 (ld.global.cg bypasses L1).  Every thread walks its own
// linear congruential sequence of sector indices; each load touches a different sector, so
// one warp-wide load requests 32 sectors.
#include <cuda_runtime.h>

#include "stf_ctx.h"

namespace {

__global__ void __launch_bounds__(256) k_sector_reads(const uint2* __restrict__ buf, uint32_t sector_mask,
                                                      uint32_t iters, uint32_t* __restrict__ sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a = t * 2654435761u + 12345u;
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t i = 0; i < iters; ++i) {
        a = a * 1664525u + 1013904223u;
        const uint2 v = __ldcg(buf + (size_t)((a >> 7) & sector_mask) * 4);   // 4 x 8 B = one sector
        acc += v.x ^ v.y;
    }
    sink[t] = acc;   // keeps the loads live
}

}  // namespace

extern "C" stf_status stf_measure_sector_rate(stf_ctx c, uint64_t buffer_bytes, double* sectors_per_s) {
    using namespace stfi;
    if (!c || !sectors_per_s) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    if (buffer_bytes < (1ull << 20) || buffer_bytes > (1ull << 30) || (buffer_bytes & (buffer_bytes - 1)))
        return fail(c, STF_ERR_INVALID_ARG, "buffer_bytes must be a power of two in 1 MiB .. 1 GiB");
    CurrentDevice cd(c->device);
    const int threads = 256, blocks = c->num_sms * 8;
    const uint32_t iters = 2048;
    void* buf = nullptr;
    uint32_t* sink = nullptr;
    stf_status s = dev_alloc(c, &buf, buffer_bytes);
    if (s != STF_OK) return s;
    s = dev_alloc(c, (void**)&sink, (size_t)threads * blocks * sizeof(uint32_t));
    if (s != STF_OK) { cudaFree(buf); return s; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(buf, 0x5A, buffer_bytes, c->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const uint32_t mask = (uint32_t)(buffer_bytes / 32 - 1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms the buffer into L2
        e = cudaEventRecord(e0, c->stream);
        k_sector_reads<<<blocks, threads, 0, c->stream>>>((const uint2*)buf, mask, iters, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "sector-rate measurement");
    *sectors_per_s = (double)threads * blocks * iters / (best * 1e-3);
    return STF_OK;
}
