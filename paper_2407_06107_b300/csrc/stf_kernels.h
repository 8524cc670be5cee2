// Internal launch interface between the C-ABI layer (stf_api.cu) and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

namespace stf {

struct TexView {
    const void* base;     // one device allocation holding every level
    int fmt;              // 0 RGBA32F (float4 texels), 1 RGBA8 material (uint2 texels)
    int levels;
    int has_normal;
    int address;          // 0 wrap (2-D textures are always wrap here)
    uint64_t off[16];     // byte offset of each level
    int w[16], h[16];
};

struct FilterShadeArgs {
    uint64_t n, id_base;
    const float *u, *v, *dudx, *dvdx, *dudy, *dvdy;
    int has_derivs;
    int filter, mode, shade;
    uint32_t spp, flags;
    int kside;            // sqrt(spp) for stratified jitter
    uint64_t seed;
    float *r, *g, *b;
    uint32_t* picks;
    uint32_t* status;
};

struct MarchArgs {
    const __half* vox;    // nz*ny*nx FP16
    int nx, ny, nz;
    float sigma_scale;
    float cam[12];
    uint32_t width, height, steps, spp, flags;
    int kside;
    int filter, mode;
    uint64_t seed, pix_begin, pix_count;
    float* T;
    uint32_t* picks;
    uint32_t* status;
};

cudaError_t launch_filter_shade(const FilterShadeArgs& a, const TexView& tv, int num_sms, cudaStream_t st);
cudaError_t launch_march(const MarchArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_pack_rgba8(const void* rgba, const void* rg, void* out, uint64_t n, cudaStream_t st);

}  // namespace stf
