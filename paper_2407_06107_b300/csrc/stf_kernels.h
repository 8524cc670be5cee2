// Internal launch interface between the C-ABI layer (stf_api.cu) and the kernels.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace stf {

// 2-D texture storage formats
enum { FMT_RGBA32F = 0, FMT_RGBA8 = 1, FMT_DCT = 2 };

// Filters.  0-5 are the API's; F_GAUSS_BOX and F_FIS_* are internal ids: the Gaussian convolved
// with the unit box (the N-tap form of FIS), and the FIS picks of the tent, the cubic B-spline
// and the Gaussian.
enum { F_LINEAR = 0, F_BSPLINE = 1, F_CATMULL_ROM = 2, F_MITCHELL = 3, F_EWA = 4,
       F_GAUSS = 5, F_GAUSS_BOX = 6, F_FIS_LINEAR = 7, F_FIS_BSPLINE = 8, F_FIS_GAUSS = 9 };

struct TexView {
    const void* base;     // one device allocation holding every level
    int fmt;              // FMT_RGBA32F (float4 texels), FMT_RGBA8 (uint2 material texels) or
                          // FMT_DCT (32-byte blocks of 8 x 8 texels)
    int levels;
    int has_normal;
    int address;          // 0 wrap (2-D textures are always wrap here)
    uint64_t off[16];     // byte offset of each level
    int w[16], h[16];
};

// texture as the kernels read it (kernel parameter, or one entry of a bindless table)
struct FetchCtx {
    const unsigned char* base;
    int fmt, levels, has_normal;
    uint64_t off[16];
    int w[16], h[16];
};

struct FilterShadeArgs {
    uint64_t n, id_base;
    const uint32_t* order;    // nullable execution order
    const float *u, *v, *dudx, *dvdx, *dudy, *dvdy;
    int has_derivs;
    int filter, mode, shade;
    uint32_t spp, flags;
    int kside;            // sqrt(spp) for stratified jitter
    uint64_t seed;
    float *r, *g, *b;
    uint32_t* picks;
    uint32_t* status;
    const float* ewa_lut;     // EWA: the 128 Gaussian weights (context-owned device array)
    float sigma, inv_s2;      // Gaussian filters: standard deviation in texels, 1 / sigma^2
};

constexpr int EWA_LUT_N = 128;

// Triplanar lookups: plane i projects the surface point along axis i (plane 0 reads (y, z),
// plane 1 (x, z), plane 2 (x, y)), each plane with its own texture.
enum { BLEND_FULL = 0, BLEND_STOCHASTIC = 1 };

struct TriplanarArgs {
    uint64_t n, id_base;
    const uint32_t* order;      // nullable execution order
    const float *px, *py, *pz, *nx, *ny, *nz;
    const float *dxx, *dxy, *dxz, *dyx, *dyy, *dyz;   // dP/dx and dP/dy components
    int has_derivs;
    float scale;                // texture coordinates per world unit
    int filter, mode, blend, shade;
    uint32_t spp, flags;
    int kside;
    uint64_t seed;
    float *r, *g, *b;
    uint32_t* picks;            // nullable: [n][spp][3][2]
    uint32_t* status;
};

struct MarchArgs {
    const __half* vox;    // nz*ny*nx FP16
    int nx, ny, nz;
    // the same voxels with a border of two replicated (clamped) voxels on every face: voxel
    // (x, y, z), each coordinate in [-2, n + 1], at vpad[z * pxy + y * px + x]
    const __half* vpad;
    int px, pxy;
    int fixed32;          // steps x (largest density) < 256: the 1-tap sum fits 32 bits
    float sigma_scale;
    float cam[12];
    uint32_t width, height, steps, spp, flags;
    int kside;
    int filter, mode;
    uint64_t seed, pix_begin, pix_count;
    int tiled;            // threads walk 8 x 4 pixel tiles (width % 8 == 0, range in whole 4-row bands)
    float* T;
    uint32_t* picks;
    uint32_t* status;
};

// learned texture: device view
struct NeuralView {
    int tex_res;
    int res[4];
    float gscale[4];            // res[g] / tex_res, FP32-rounded on the host (IEEE division)
    uint64_t lat_off[4];        // element offset of each grid (same in every latent format)
    int latent_fmt;             // inference latents: 0 FP16, 1 FP8 E4M3 x scale
    const __half* lat16;
    const uint8_t* lat8;
    float* lat32;               // FP32 master latents (training)
    float* dlat;                // latent gradients
    float scale[4];             // FP8 per-grid scales (host copy)
    float* scale_dev;
    float* mlp32;               // FP32 master MLP: W1[64x32] b1[64] W2[64x64] b2[64] W3[8x64] b3[8]
    float* grad32;              // gradients, same layout
    __nv_bfloat16* wbf;         // inference weights: W1 | W2 | W3 padded to 16 rows
    float* bias;                // inference biases: b1 | b2 | b3 padded to 16
    // inference weights with the biases as extra columns, each FP32 bias split exactly into
    // three BF16 parts (row-major): W1 | b1 [64][48], W2 | b2 [64][80], W3 | b3 [16][80]
    __nv_bfloat16* wext;
    const uint8_t* targets;     // explicit 8-channel texture [tex_res][tex_res][8]
};

struct NeuralDecodeArgs {
    uint64_t n, id_base;
    const float *u, *v, *dudx, *dvdx, *dudy, *dvdy;
    int has_derivs;
    int filter, mode, shade;    // mode < 0: decode the explicit texel list ex_ix/ex_iy
    uint32_t spp;
    uint64_t seed;
    int tex_res;
    uint64_t nrows;             // rows (texel decodes) of the launch
    const int32_t *ex_ix, *ex_iy;
    float* y_out;               // decode-only: [n][8]
    float *r, *g, *b;           // filter modes: accumulated, must be zero on entry
    uint32_t* status;
    int inject_timeout;         // fault injection: issue no MMA and wait with a short limit
};

cudaError_t launch_ntc_train(const NeuralView& N, uint32_t step, uint32_t batch, uint32_t first, uint32_t count,
                             uint64_t seed, float* loss_sum, const int32_t* ex_ix, const int32_t* ex_iy, int num_sms,
                             uint32_t* status, cudaStream_t st);
cudaError_t launch_adam(float* p, float* g, float* m, float* v, uint64_t n, float lr, float b1, float b2, float eps,
                        int t, int num_sms, cudaStream_t st);
cudaError_t launch_ntc_quantize(const NeuralView& N, uint64_t lat_total, int fmt, unsigned int* amax_scratch,
                                cudaStream_t st);
cudaError_t launch_ntc_decode(const NeuralView& N, const NeuralDecodeArgs& a, int num_sms, cudaStream_t st);

struct ShadeConst;
ShadeConst make_shade_const();

cudaError_t launch_filter_shade(const FilterShadeArgs& a, const TexView& tv, int num_sms, cudaStream_t st);
FetchCtx make_fetch_ctx(const TexView& tv);
cudaError_t launch_filter_shade_table(const FilterShadeArgs& a, const FetchCtx* table, uint32_t ntex,
                                      const uint32_t* tex_id, unsigned long long* counter, int num_sms,
                                      cudaStream_t st);
cudaError_t launch_triplanar(const TriplanarArgs& a, const TexView tv[3], cudaStream_t st);
// tmap: the volume as a 3-D FP16 tensor map with a 24 x 8 x 8 box (encode_volume_tmap), or
// null; with it, the tricubic N-tap marches stage each warp's voxels in shared memory by TMA.
cudaError_t launch_march(const MarchArgs& a, const CUtensorMap* tmap, int num_sms, cudaStream_t st);
bool encode_volume_tmap(CUtensorMap* out, const void* vox, int nx, int ny, int nz);
// the clamped border copy: dst holds (nx + 4 rounded up to 8) x (ny + 4) x (nz + 4) voxels
constexpr int VOL_PAD = 2;
inline uint32_t vol_pad_pitch(uint32_t nx) { return (nx + 2 * VOL_PAD + 7u) & ~7u; }
cudaError_t launch_pad_volume(const void* src, int nx, int ny, int nz, void* dst, cudaStream_t st);
// the largest non-negative density of n FP16 voxels, as FP16 bits, into *out (device)
cudaError_t launch_vol_max_bits(const void* vox, uint64_t n, unsigned int* out, cudaStream_t st);
cudaError_t launch_bin_queries(uint64_t n, const float* u, const float* v, const uint32_t* tex_id, uint32_t ntex,
                               uint32_t tile_log2, uint32_t* order, uint32_t* scratch, uint64_t nbins,
                               cudaStream_t st);
cudaError_t launch_pack_rgba8(const void* rgba, const void* rg, void* out, uint64_t n, cudaStream_t st);

}  // namespace stf
