// Pick binning: spatial counting sort of queries, so that neighbouring threads of the
// filter kernels gather from nearby texels (sector and cache-line reuse).  The sort key is
// (texture id, tile of the wrapped uv); the order within a bin is the arrival order of the
// scatter's atomics, which only affects performance: every query writes its own slot.
#include "stf_kernels.h"

namespace stf {

__device__ __forceinline__ uint32_t bin_key(float u, float v, uint32_t tid, uint32_t tile_log2) {
    const uint32_t R = 1u << tile_log2;
    float fu = u - floorf(u), fv = v - floorf(v);           // wrap to [0, 1)
    uint32_t tx = min((uint32_t)(fu * (float)R), R - 1u), ty = min((uint32_t)(fv * (float)R), R - 1u);
    if (!(fu == fu)) tx = 0;                                  // NaN coordinates go to tile 0
    if (!(fv == fv)) ty = 0;
    return (tid << (2 * tile_log2)) | (ty << tile_log2) | tx;
}

__global__ void k_bin_hist(uint64_t n, const float* u, const float* v, const uint32_t* tex_id, uint32_t ntex,
                           uint32_t tile_log2, uint32_t* hist) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t t = tex_id ? __ldg(tex_id + i) : 0u;
        t = t < ntex ? t : 0u;                                // out-of-range ids are binned with 0
        atomicAdd(hist + bin_key(__ldg(u + i), __ldg(v + i), t, tile_log2), 1u);
    }
}

// exclusive scan of 1024 bins per block; block totals to sums[]
__global__ void k_scan_blocks(uint32_t* data, uint64_t nbins, uint32_t* sums) {
    __shared__ uint32_t s[1024];
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    const uint32_t x = i < nbins ? data[i] : 0u;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t y = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    if (i < nbins) data[i] = s[threadIdx.x] - x;
    if (threadIdx.x == 1023) sums[blockIdx.x] = s[1023];
}
// exclusive scan of up to 1024 * 64 block sums in one block (sequential over chunks)
__global__ void k_scan_sums(uint32_t* sums, uint32_t nblocks) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nblocks; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < nblocks ? sums[i] : 0u;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const uint32_t y = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
            __syncthreads();
            s[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < nblocks) sums[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}
__global__ void k_add_sums(uint32_t* data, uint64_t nbins, const uint32_t* sums) {
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < nbins) data[i] += sums[blockIdx.x];
}
__global__ void k_bin_scatter(uint64_t n, const float* u, const float* v, const uint32_t* tex_id, uint32_t ntex,
                              uint32_t tile_log2, uint32_t* cursor, uint32_t* order) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t t = tex_id ? __ldg(tex_id + i) : 0u;
        t = t < ntex ? t : 0u;
        const uint32_t pos = atomicAdd(cursor + bin_key(__ldg(u + i), __ldg(v + i), t, tile_log2), 1u);
        order[pos] = (uint32_t)i;
    }
}

// scratch: nbins counters followed by ceil(nbins / 1024) block sums
cudaError_t launch_bin_queries(uint64_t n, const float* u, const float* v, const uint32_t* tex_id, uint32_t ntex,
                               uint32_t tile_log2, uint32_t* order, uint32_t* scratch, uint64_t nbins,
                               cudaStream_t st) {
    const uint64_t nblk = (nbins + 1023) / 1024;
    uint32_t* hist = scratch;
    uint32_t* sums = scratch + nblk * 1024;
    cudaError_t e = cudaMemsetAsync(hist, 0, nbins * 4, st);
    if (e != cudaSuccess) return e;
    const int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    k_bin_hist<<<grid, 256, 0, st>>>(n, u, v, tex_id, ntex, tile_log2, hist);
    k_scan_blocks<<<(int)nblk, 1024, 0, st>>>(hist, nbins, sums);
    k_scan_sums<<<1, 1024, 0, st>>>(sums, (uint32_t)nblk);
    k_add_sums<<<(int)nblk, 1024, 0, st>>>(hist, nbins, sums);
    k_bin_scatter<<<grid, 256, 0, st>>>(n, u, v, tex_id, ntex, tile_log2, hist, order);
    return cudaGetLastError();
}

}  // namespace stf
