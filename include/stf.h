/* stf.h -- C ABI of libstf: stochastic texture filtering (filter-after-shading) on B300.
 *
 * Method: Pharr, Wronski, Salvi, Fajardo, "Filtering After Shading With Stochastic
 * Texture Filtering" (2024).  For every query the library either
 *   - importance-samples ONE texel from a separable filter and shades it (the
 *     stochastic estimator of Eq. stochastic-sum applied to Eq. filtering-after-shading,
 *     Sec. 4 "Stochastic Texture Filtering", Sec. 4.1 FRS), or
 *   - evaluates the conventional N-tap filter-before-shading sum
 *     (Eq. filter-before-shading), or
 *   - evaluates the exact N-tap filter-after-shading sum (Eq. filtering-after-shading).
 *
 * Conventions for every entry point
 *   - No exception crosses the ABI; every call returns an stf_status.  Host-side argument
 *     validation is synchronous: on error nothing is enqueued and outputs are untouched.
 *   - Work is enqueued asynchronously on the context's CUDA stream.  Device-detected
 *     problems (NaN inputs, out-of-range table ids) set bits of a device status word,
 *     read and cleared by stf_get_device_status().
 *   - Ownership: the caller owns query, derivative and output buffers (device pointers,
 *     e.g. torch tensors, 4-byte aligned; 16-byte alignment enables vector loads).  The
 *     library owns textures and volumes: it COPIES the data in at creation and frees it at
 *     destruction.
 *   - A context is not thread-safe; use one per host thread.
 *   - Fault injection for tests (environment variable STF_FAULT, read by stf_create):
 *     "alloc" makes every device allocation of the context fail (STF_ERR_OOM), "launch"
 *     makes every kernel launch fail (STF_ERR_CUDA) without launching, "mma_timeout"
 *     makes the tensor-core decode issue no MMA so its bounded wait runs out (the kernel
 *     frees its tensor memory and sets STF_DEV_TIMEOUT).
 *   - Query ids are 64-bit (they key the Philox counter): the id of query i of a call is
 *     queries->id_base + i, so that shards of one batch draw the same numbers as the whole.
 */
#ifndef STF_H
#define STF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stf_ctx_s* stf_ctx;
typedef uint64_t stf_tex;   /* texture handle, 0 is never valid */
typedef uint64_t stf_vol;   /* volume handle, 0 is never valid */

typedef enum {
    STF_OK = 0,
    STF_ERR_INVALID_ARG = 1,    /* null pointer, size/enum out of range, misalignment    */
    STF_ERR_BAD_HANDLE = 2,     /* unknown or destroyed texture / volume handle          */
    STF_ERR_OOM = 3,            /* device allocation failed                              */
    STF_ERR_CUDA = 4,           /* a CUDA runtime call failed (see stf_last_error)       */
    STF_ERR_UNSUPPORTED = 5,    /* valid but unsupported combination (e.g. positivized
                                   with a non-negative filter)                          */
    STF_ERR_DEVICE_STATUS = 6,  /* the device status word had bits set                  */
    STF_ERR_TIMEOUT = 7         /* a bounded device wait gave up                         */
} stf_status;

typedef enum {
    STF_FMT_RGBA32F = 0,  /* RGB albedo, A = roughness (GGX alpha), 16 B/texel            */
    STF_FMT_RGBA8 = 1,    /* UNORM albedo RGB, A byte -> roughness 0.05 + 0.95 a/255       */
    STF_FMT_RG8 = 2,      /* tangent-space normal XY (UNORM, z reconstructed)              */
    STF_FMT_R16F = 3,     /* FP16 density (volumes)                                       */
    STF_FMT_DCT6 = 4      /* DCT-compressed material (supplement "Texture compression"): per
                             level, ceil(H/8) x ceil(W/8) blocks of 32 bytes, row-major, each 6
                             little-endian uint32 channel words (albedo R, G, B, roughness,
                             normal X, Y, each in [0,1]) and 8 padding bytes.  A word holds the
                             orthonormal 2-D DCT-II coefficients u + v <= 2 of one 8 x 8 block:
                             bits 0-6 the DC term (q * 8/127), then 5-bit fields for (u,v) =
                             (1,0), (0,1), (2,0), (1,1), (0,2) ((q - 15) * 2/15).  Levels narrower
                             than 8 repeat periodically inside their block.  A texel decodes to
                             the inverse DCT of those six terms at its position; roughness maps
                             to 0.05 + 0.95 r, the normal to (2x-1, 2y-1, z) normalised.
                             stf_filter_shade only (not texture tables); no normal_data. */
} stf_format;

/* 1-D reconstruction kernels, applied separably (supplement "Filter Kernels").
 * With MIP levels and derivatives, every filter also blends the two nearest levels
 * linearly (trilinear for STF_FILTER_LINEAR). */
typedef enum {
    STF_FILTER_LINEAR = 0,       /* tent K1: bilinear / trilinear, 2 taps per axis        */
    STF_FILTER_BSPLINE = 1,      /* cubic B-spline K_bs, 4 taps per axis                  */
    STF_FILTER_CATMULL_ROM = 2,  /* Keys cubic K3 with a = -1/2, 4 taps, negative lobes   */
    STF_FILTER_MITCHELL = 3,     /* Mitchell-Netravali BC(1/3,1/3), 4 taps, neg. lobes    */
    STF_FILTER_EWA = 4,          /* elliptically weighted average over a Gaussian (supplement
                                    "Stochastic EWA", as pbrt evaluates it): the ellipse of the
                                    derivative footprint plus a one-texel reconstruction term,
                                    eccentricity capped at 64, weights exp(-2r^2)-exp(-2) from a
                                    128-entry table.  Modes NTAP_BEFORE,
                                    NTAP_AFTER (each level normalised by its weight sum) and
                                    STOCHASTIC (one texel by weighted reservoir sampling over the
                                    ellipse's box, raster order, uniform remapped per decision);
                                    no screen-space jitter; flags: LOD0 only */
    STF_FILTER_GAUSSIAN = 5      /* Gaussian exp(-d^2/(2 sigma^2)) at texel centres, normalised
                                    (Sec. 4.2 FIS, supplement Gaussian listings); needs
                                    stf_filter_shade_ex for sigma and the sampler */
} stf_filter;

/* How a stochastic lookup draws its texel (stf_filter_shade_ex):
 *   FRS: filter reservoir sampling, i.e. CDF picks over the discrete weights.  For the Gaussian
 *        the window is the 4 x 4 texels at offsets -1..2 from floor(p), as in the listing.
 *   FIS: filter importance sampling.  A continuous offset o (texels) is drawn from a density
 *        whose convolution with the unit box is the filter, then the nearest texel
 *        floor(x W + o) is taken:
 *          LINEAR   o = u - 1/2, which gives the tent;
 *          BSPLINE  o = u1 + u2 + u3 - 3/2, the quadratic B-spline, which gives the cubic one;
 *          GAUSSIAN o = sigma * Box-Muller(1 - u_a, u_b), which gives the Gaussian convolved
 *                   with the box.
 *        The N-tap modes with FIS evaluate the filter that FIS converges to: the tent, the
 *        cubic B-spline, or the box-convolved Gaussian.
 * Gaussian N-tap windows cover |i - p| <= ceil(5 sigma) + 1 per axis. */
typedef enum { STF_SAMPLER_FRS = 0, STF_SAMPLER_FIS = 1 } stf_sampler;

typedef struct {
    stf_filter filter;
    stf_sampler sampler;
    float sigma;         /* Gaussian standard deviation in texels, (0, 8]; ignored otherwise */
} stf_filter_desc;

typedef enum {
    STF_MODE_NTAP_BEFORE = 0,           /* shade(sum_i w_i t_i)             Eq. filter-before-shading */
    STF_MODE_NTAP_AFTER = 1,            /* sum_i w_i shade(t_i) (exact)     Eq. filtering-after-shading */
    STF_MODE_STOCHASTIC = 2,            /* one texel drawn ~|w|, times sign * sum|w|  Eq. stochastic-sum */
    STF_MODE_STOCHASTIC_POSITIVIZED = 3 /* one texel from each sign set (Sec. 2.2 positivization) */
} stf_mode;

typedef enum {
    STF_SHADE_GGX_LAMBERT = 0,  /* f_hat = [rho/pi + D G F/(4 nl nv)] nl, fixed l, v      */
    STF_SHADE_LINEAR = 1        /* identity on albedo (affine shade, Sec. 3)               */
} stf_shade;

typedef enum { STF_ADDRESS_WRAP = 0, STF_ADDRESS_CLAMP = 1 } stf_address;

/* flags */
#define STF_FLAG_STRATIFIED 1u  /* jitter on a sqrt(spp) x sqrt(spp) grid (spp must be a square) */
#define STF_FLAG_LATTICE 2u     /* stochastic modes: the pick uniforms of the spp samples of a query
                                   (pixel) form a randomly shifted lattice, frac(s/spp + phi), so they
                                   are stratified across samples; each stays uniform (unbiased) */
#define STF_FLAG_REUSE 4u       /* 1-tap stochastic mode: one uniform per sample (per step in a volume)
                                   drives the level and every axis, remapped after each decision
                                   (Eq. uniform-sample-reuse; the listings' sample reuse) */
#define STF_FLAG_LOD0 8u        /* 2-D: sample the finest MIP level only (no MIP prefiltering, Sec.
                                   4.2.1's "no MIP mapping" variant and its point-sampled reference) */

/* device status bits */
#define STF_DEV_NAN_INPUT 1u
#define STF_DEV_BAD_INDEX 2u
#define STF_DEV_TIMEOUT 4u      /* a bounded device wait gave up (tensor-core decode) */

#define STF_MAX_LEVELS 16

typedef struct {
    uint32_t width, height;        /* level 0 size, 1 .. 16384                              */
    uint32_t num_levels;           /* 1 .. 16; level l is max(1, w >> l) x max(1, h >> l)   */
    stf_format format;             /* STF_FMT_RGBA32F or STF_FMT_RGBA8                       */
    stf_address address;
    const void* const* level_data; /* num_levels pointers, row-major (y then x), tightly packed */
    const void* const* normal_data;/* nullable; num_levels RG8 pointers (RGBA8 only)        */
    int data_on_device;            /* 0: host pointers; 1: device pointers                  */
} stf_texture_desc;

typedef struct {
    uint64_t n;          /* number of queries (0 is a valid no-op)                          */
    uint64_t id_base;    /* Philox id of query 0                                            */
    const float* u;      /* [n] texture coordinates, any real value (wrapped / clamped)     */
    const float* v;      /* [n]                                                             */
    const uint32_t* order;  /* nullable: [n] permutation; thread i evaluates query order[i]
                            (e.g. from stf_bin_queries, for gather locality).  Results land in
                            each query's own slot and are identical with or without it.    */
} stf_queries;

typedef struct {         /* screen-space derivatives of (u, v), [n] each                    */
    const float* dudx;
    const float* dvdx;
    const float* dudy;
    const float* dvdy;
} stf_derivs;

typedef struct {
    float* r;            /* [n] mean shaded value over spp, SoA                             */
    float* g;
    float* b;
    uint32_t* picks;     /* nullable: [n][spp][2] selected texels (lvl<<28 | iy<<14 | ix),
                            slot 1 = negative sample of positivization, 0xFFFFFFFF = none   */
} stf_output;

/* ---- context --------------------------------------------------------------------------- */
/* device: CUDA ordinal; cuda_stream: cudaStream_t or NULL for the legacy default stream. */
stf_status stf_create(int device, void* cuda_stream, stf_ctx* out);
stf_status stf_destroy(stf_ctx ctx);
/* Later calls queue on cuda_stream.  Synchronises the previous stream first: the context's
 * scratch (binning histogram, device status word) is then never in use on two streams. */
stf_status stf_set_stream(stf_ctx ctx, void* cuda_stream);
stf_status stf_synchronize(stf_ctx ctx);
/* Reads and clears the device status word (synchronises the stream and the host-buffer
 * pipeline).  Returns STF_ERR_DEVICE_STATUS if any bit was set. */
stf_status stf_get_device_status(stf_ctx ctx, uint32_t* flags);
const char* stf_status_string(stf_status s);
const char* stf_last_error(stf_ctx ctx);

/* ---- textures (Eq. texture-definition: texels on a uniform grid, Sec. 2.1) ------------ */
stf_status stf_create_texture(stf_ctx ctx, const stf_texture_desc* desc, stf_tex* out);
stf_status stf_destroy_texture(stf_ctx ctx, stf_tex tex);

/* ---- 2-D filter + shade ---------------------------------------------------------------- */
/* For every query: spp samples, each = screen-space jitter inside the derivative
 * footprint (Sec. 4.2.1), stochastic MIP level (or linear blend for N-tap modes), the
 * filter in `mode`, shade; out = mean over samples.  derivs == NULL: no jitter, level 0.
 * spp >= 1; positivized mode needs a signed filter (else STF_ERR_UNSUPPORTED). */
stf_status stf_filter_shade(stf_ctx ctx, stf_tex tex, const stf_queries* q, const stf_derivs* d,
                            stf_filter filter, stf_mode mode, stf_shade shade, uint32_t spp,
                            uint64_t seed, uint32_t flags, const stf_output* out);

/* stf_filter_shade with a filter descriptor (filter, sampler, sigma).  FRS with filters 0-4
 * is stf_filter_shade.  GAUSSIAN and FIS: no positivization (STF_ERR_UNSUPPORTED); flags
 * STRATIFIED and LOD0 only; FIS for LINEAR, BSPLINE and GAUSSIAN (else STF_ERR_UNSUPPORTED);
 * sigma outside (0, 8] for GAUSSIAN is STF_ERR_INVALID_ARG. */
stf_status stf_filter_shade_ex(stf_ctx ctx, stf_tex tex, const stf_queries* q, const stf_derivs* d,
                               const stf_filter_desc* filter, stf_mode mode, stf_shade shade, uint32_t spp,
                               uint64_t seed, uint32_t flags, const stf_output* out);

/* Same computation from HOST buffers (u, v, derivs, r, g, b, picks all host memory):
 * copies the inputs to library-owned device staging memory, runs, copies the results back
 * and synchronises.  Pinned host memory gives full PCIe bandwidth. */
stf_status stf_filter_shade_host(stf_ctx ctx, stf_tex tex, const stf_queries* q, const stf_derivs* d,
                                 stf_filter filter, stf_mode mode, stf_shade shade, uint32_t spp,
                                 uint64_t seed, uint32_t flags, const stf_output* out);
/* stf_filter_shade_host without the final wait: the copies and launches are queued on the
 * library's copy-pipeline streams and the call returns.  Consecutive calls keep the pipeline
 * full (the next call's first copies overlap the previous call's last ones).  The host query
 * buffers must stay unchanged, and the results are valid, only after stf_synchronize (which
 * waits for these streams as well as the context's stream).  stf_get_device_status,
 * stf_destroy_texture and stf_destroy also wait for them.  Calls of any sizes may follow
 * one another: a call whose staging layout differs from the previous call's waits, on the
 * GPU and not on the host, for all earlier pipeline work before it reuses the staging.  The
 * call still validates its arguments synchronously; a failure while queueing waits for the
 * pipeline and is returned. */
stf_status stf_filter_shade_host_async(stf_ctx ctx, stf_tex tex, const stf_queries* q, const stf_derivs* d,
                                       stf_filter filter, stf_mode mode, stf_shade shade, uint32_t spp,
                                       uint64_t seed, uint32_t flags, const stf_output* out);

/* ---- bindless texture table: many textures in one persistent launch ------------------ */
typedef uint64_t stf_table;
/* A table of n existing textures (any sizes, formats and MIP counts); the textures must
 * outlive the table (stf_destroy_texture refuses a texture a table still references). */
stf_status stf_create_texture_table(stf_ctx ctx, uint32_t n, const stf_tex* textures, stf_table* out);
stf_status stf_destroy_texture_table(stf_ctx ctx, stf_table table);
/* stf_filter_shade over mixed textures: query i uses table entry tex_id[i] (device uint32
 * [n]); one persistent launch whose blocks claim query chunks from an atomic work counter
 * (table-owned, reset by each call; one call per table at a time).  An out-of-range id
 * sets STF_DEV_BAD_INDEX and yields 0 for that query. */
stf_status stf_filter_shade_table(stf_ctx ctx, stf_table table, const stf_queries* q, const uint32_t* tex_id,
                                  const stf_derivs* d, stf_filter filter, stf_mode mode, stf_shade shade,
                                  uint32_t spp, uint64_t seed, uint32_t flags, const stf_output* out);

/* ---- triplanar mapping (Sec. 5 "Triplanar mapping"; Sec. 4.4 material graphs) --------- */
/* A surface point P with normal N is looked up on three planes: plane 0 at
 * (u, v) = scale * (P.y, P.z), plane 1 at scale * (P.x, P.z), plane 2 at scale * (P.x, P.y),
 * each in its own texture, with the derivatives of P projected the same way.  The blend
 * weights are b_i = |N_i|^4 / sum_j |N_j|^4 (FP32, fixed order); a normal whose weights all
 * vanish uses plane 2 alone.  Each plane's lookup is the 2-D lookup of stf_filter_shade
 * (jitter in the plane's footprint, level from its derivatives and its texture's level-0
 * size, the filter in `mode`), all planes of a sample from the same uniforms. */
typedef enum {
    STF_BLEND_FULL = 0,        /* every plane with b_i > 0, weighted: sum_i b_i L_i.  With
                                  NTAP_BEFORE the planes' filtered materials are blended and the
                                  result is shaded once.                                      */
    STF_BLEND_STOCHASTIC = 1   /* one plane per sample, drawn with probability b_i (Eq.
                                  stochastic-sum over the blend), from the fifth uniform of the
                                  sample's second Philox stream; weight b_i / p_i = 1          */
} stf_blend;

typedef struct {
    uint64_t n;          /* number of queries (0 is a valid no-op)                          */
    uint64_t id_base;    /* Philox id of query 0                                            */
    const float* px;     /* [n] surface position, world units                               */
    const float* py;
    const float* pz;
    const float* nx;     /* [n] surface normal, any length                                  */
    const float* ny;
    const float* nz;
    const uint32_t* order;  /* nullable: [n] execution order, as in stf_queries              */
} stf_tri_queries;

typedef struct {         /* screen-space derivatives of P, [n] each                         */
    const float* dpdx_x;
    const float* dpdx_y;
    const float* dpdx_z;
    const float* dpdy_x;
    const float* dpdy_y;
    const float* dpdy_z;
} stf_tri_derivs;

/* Triplanar filter + shade.  tex: three texture handles (planes 0, 1, 2; they may repeat),
 * either all DCT6 or none; filters LINEAR, BSPLINE, CATMULL_ROM, MITCHELL; flags STRATIFIED,
 * LATTICE and LOD0 (REUSE: STF_ERR_UNSUPPORTED); scale finite and non-zero.  derivs NULL: no
 * jitter, level 0.  out->picks (nullable) is [n][spp][3][2]: per plane the stf_output pick
 * pair, 0xFFFFFFFF for a plane the sample did not look up (and for N-tap modes).
 * Device memory throughout; asynchronous on the context's stream. */
stf_status stf_triplanar_shade(stf_ctx ctx, const stf_tex tex[3], float scale, const stf_tri_queries* q,
                               const stf_tri_derivs* d, stf_filter filter, stf_mode mode, stf_blend blend,
                               stf_shade shade, uint32_t spp, uint64_t seed, uint32_t flags,
                               const stf_output* out);

/* ---- pick binning: spatial ordering of queries for gather locality -------------------- */
/* Counting sort of the n queries by bin = (tex_id[i], tile of (frac(u), frac(v)) on a
 * 2^tile_log2 x 2^tile_log2 grid): order_out[n] (device uint32) lists the queries bin by
 * bin.  tex_id nullable (one texture); ntex = number of texture ids (1 if tex_id is NULL);
 * ntex * 4^tile_log2 <= 2^26, n < 2^32.  Uses context-owned scratch for the histogram
 * (grown on demand, which synchronises the context stream; separate from the host-buffer
 * pipeline's staging, so it may overlap asynchronous host-buffer calls).  The order within
 * a bin is not deterministic. */
stf_status stf_bin_queries(stf_ctx ctx, uint64_t n, const float* u, const float* v, const uint32_t* tex_id,
                           uint32_t ntex, uint32_t tile_log2, uint32_t* order_out);

/* Same computation as stf_filter_shade_host, for callers that must not allocate device
 * memory while they look up textures (a frame loop with a fixed memory budget, or a
 * plug-in inside an application that owns all device allocations).  The paper has no
 * counterpart: this is a deployment variant.  Queries, results and the device status word
 * are staged in one fixed device array of the library (a little over 9 MiB, held by every
 * GPU that loads the library until the process exits) instead of context-owned buffers
 * grown with cudaMalloc, so the call allocates nothing.
 *   - Takes every filter (EWA included), mode, shade and flag (LOD0 included) that
 *     stf_filter_shade_host takes, with the same checks.
 *   - At most 262144 queries per call (STF_ERR_INVALID_ARG beyond); picks must be NULL
 *     (STF_ERR_UNSUPPORTED otherwise); no execution order (q->order must be NULL).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (other streams, other
 *     host threads, other contexts on the same device) race and corrupt each other.
 *   - Synchronises the context stream; returns STF_ERR_DEVICE_STATUS if the kernel
 *     flagged its inputs (the results are still written).  The call's device status bits
 *     live in the shared array and are reported by this return value only: they are not
 *     merged into the context's status word, so stf_get_device_status does not see them. */
stf_status stf_filter_shade_host_noalloc(stf_ctx ctx, stf_tex tex, const stf_queries* q, const stf_derivs* d,
                                         stf_filter filter, stf_mode mode, stf_shade shade, uint32_t spp,
                                         uint64_t seed, uint32_t flags, const stf_output* out);

/* ---- 3-D volume march (Sec. 5 "Offline rendering", transmittance exp(-sigma dt)) ------- */
/* data: nz*ny*nx FP16 densities (x fastest); sigma = sigma_scale * density.  The library keeps
 * two device copies: the grid itself (read by the N-tap marches and the TMA-staged comparator)
 * and a copy with a clamped two-voxel border on every face, rows padded to a multiple of 8
 * voxels, which the 1-tap march reads without clamping its picks (about 2.1x the grid's bytes in
 * all).  It also records the grid's largest density: where steps x that maximum is below 256,
 * the 1-tap march sums its fixed-point densities in 32 bits.  Synchronises the context stream. */
stf_status stf_create_volume(stf_ctx ctx, uint32_t nx, uint32_t ny, uint32_t nz, stf_format format,
                             float sigma_scale, const void* data, int data_on_device, stf_vol* out);
stf_status stf_destroy_volume(stf_ctx ctx, stf_vol vol);

/* cam: 12 floats = eye[3], forward[3], right[3] (scaled by tan(fov/2)*aspect), up[3]
 * (scaled by tan(fov/2)).  Pixels pix_begin .. pix_begin+pix_count-1 of a width x height
 * image (row-major); out_T[pix_count] = mean transmittance over spp.  filter: LINEAR
 * (trilinear, 8 taps) or BSPLINE (tricubic, 64 taps); mode: NTAP_BEFORE, NTAP_AFTER or
 * STOCHASTIC.  out_picks nullable: [pix_count][spp][steps] voxels (z<<20 | y<<10 | x). */
stf_status stf_march_volume(stf_ctx ctx, stf_vol vol, const float* cam, uint32_t width,
                            uint32_t height, uint32_t steps, stf_filter filter, stf_mode mode,
                            uint32_t spp, uint64_t seed, uint32_t flags, uint64_t pix_begin,
                            uint64_t pix_count, float* out_T, uint32_t* out_picks);

/* ---- learned form: neural texture ----------------------------------------------------
 * A tex_res x tex_res texture of 8 channels (albedo RGB, roughness, normal XY, metalness,
 * height; each byte/255) represented by 4 latent grids (8 channels each, grid_res[g]^2
 * texels, sampled bilinearly with wrap at the texel centre) and an MLP 32 -> 64 (ReLU)
 * -> 64 (ReLU) -> 8 with BF16 weights and FP32 accumulation.  The paper cites learned
 * texture compression as an expensive-to-decode representation that stochastic filtering
 * decodes once per lookup (Sec. 1, Sec. 5); the network itself is this library's.
 * Training: MSE on texels drawn by Philox (ctr = (sample, step, 0, 0x4E54), key = seed),
 * analytic backward, Adam (Kingma & Ba 2015). */
typedef uint64_t stf_neural;

typedef struct {
    uint32_t tex_res;               /* decoded texture size, 1 .. 16384                     */
    uint32_t grid_res[4];           /* latent grid sizes, 1 .. 4096                          */
    const float* const* latent_init;/* 4 host arrays [grid_res^2][8] FP32                   */
    const float* mlp_init;          /* host FP32 [6792] = W1[64x32] b1[64] W2[64x64] b2[64]
                                       W3[8x64] b3[8], row-major [out][in]                  */
    const uint8_t* targets;         /* host [tex_res^2][8] bytes, nullable (no training)     */
} stf_neural_desc;

/* Adam (Kingma & Ba 2015) with bias correction.  lr_min_frac < 1 decays both learning rates
 * over the `steps` of one stf_neural_train call on a half cosine, from lr at the first step
 * to lr * lr_min_frac at the last: lr_k = lr (f + (1 - f)(1 + cos(pi k / steps)) / 2),
 * k = 0 .. steps-1.  lr_min_frac = 1 keeps them constant. */
typedef struct { float lr_latent, lr_mlp, beta1, beta2, eps, lr_min_frac; } stf_adam_params;

typedef enum {
    STF_LATENT_KEEP = -1,           /* stf_neural_quantize: rebuild in the current format    */
    STF_LATENT_FP16 = 0,            /* inference latents FP16 (round to nearest even)        */
    STF_LATENT_FP8_E4M3 = 1         /* FP8 E4M3 with a per-grid FP32 scale = max|l| / 448   */
} stf_latent_format;

typedef enum {                      /* stf_neural_get / stf_neural_set blocks                */
    STF_NEURAL_LATENTS = 0,         /* FP32 master latents, all grids concatenated           */
    STF_NEURAL_MLP = 1,             /* FP32 master MLP [6792]                                */
    STF_NEURAL_GRAD_LATENTS = 2,    /* FP32 latent gradients                                 */
    STF_NEURAL_GRAD_MLP = 3,        /* FP32 MLP gradients                                    */
    STF_NEURAL_ADAM = 4,            /* FP32 Adam moments: m_lat, v_lat, m_mlp, v_mlp         */
    STF_NEURAL_SCALES = 5,          /* FP32 [4] FP8 per-grid scales                          */
    STF_NEURAL_STEP = 6             /* uint32 optimiser step counter                         */
} stf_neural_block;

stf_status stf_neural_create(stf_ctx ctx, const stf_neural_desc* desc, stf_neural* out);
stf_status stf_neural_destroy(stf_ctx ctx, stf_neural net);
/* `steps` optimiser steps of `batch` samples each (batch <= 2^24); losses: nullable host
 * array [steps] receiving each step's mean squared error.  Re-quantises the inference
 * form with the current latent format afterwards.  Synchronises the stream. */
stf_status stf_neural_train(stf_ctx ctx, stf_neural net, uint32_t steps, uint32_t batch,
                            const stf_adam_params* adam, uint64_t seed, float* losses);
/* Gradients of one batch without an update (they replace the gradient blocks): the step
 * index selects the Philox samples, or ex_ix/ex_iy (device int32 [batch], nullable)
 * give the texels.  loss: host float. */
stf_status stf_neural_grad(stf_ctx ctx, stf_neural net, uint32_t step, uint32_t batch, uint64_t seed,
                           const int32_t* ex_ix, const int32_t* ex_iy, float* loss);
/* Data-parallel training: one process per GPU, one replica of the network each (created
 * from the same initial parameters).  Every optimiser step k of a run of `steps`:
 *   1. each rank calls stf_neural_grad_range for its share [first, first + count) of the
 *      step's `batch` Philox samples (sample ids are global and the loss is normalised by
 *      the whole batch, so the ranks' gradients SUM to the batch gradient);
 *   2. the caller sums the two gradient arrays of stf_neural_grad_buffers over the ranks in
 *      place (an all-reduce on the context stream), the one exchange step of training;
 *   3. each rank calls stf_neural_adam_step(k, steps): identical updates keep the replicas
 *      identical.
 * Then stf_neural_quantize rebuilds the inference form.  With one rank this is
 * stf_neural_train.  Both calls are asynchronous on the context stream. */
/* Replaces the gradient arrays with the gradients of samples [first, first + count) of
 * the batch of optimiser step `step` (first + count <= batch <= 2^24; count may be 0).
 * loss: nullable device float to which this part's share of the batch's mean squared
 * error is added. */
stf_status stf_neural_grad_range(stf_ctx ctx, stf_neural net, uint32_t step, uint32_t batch, uint32_t first,
                                 uint32_t count, uint64_t seed, float* loss);
/* Device addresses and lengths (FP32 elements) of the latent and MLP gradient arrays,
 * owned by the network and valid until it is destroyed.  The MLP array follows the latent
 * array at the next 256-byte boundary, and the gap between them is zero: one all-reduce
 * (sum) over the FP32 span [grad_latents, grad_mlp + n_mlp) sums both arrays. */
stf_status stf_neural_grad_buffers(stf_ctx ctx, stf_neural net, float** grad_latents, uint64_t* n_latents,
                                   float** grad_mlp, uint64_t* n_mlp);
/* Optimiser step k (0 <= k < steps) of a run of `steps` with the current gradients, which
 * it consumes (zeroes); the learning-rate schedule is stf_neural_train's. */
stf_status stf_neural_adam_step(stf_ctx ctx, stf_neural net, const stf_adam_params* adam, uint32_t k, uint32_t steps);
/* Build the inference form (BF16 weights, FP16 or FP8 latents) from the FP32 masters. */
stf_status stf_neural_quantize(stf_ctx ctx, stf_neural net, stf_latent_format fmt);
/* Copy a block to / from host memory; bytes must equal the block size. Synchronous. */
stf_status stf_neural_get(stf_ctx ctx, stf_neural net, stf_neural_block what, void* host, size_t bytes);
stf_status stf_neural_set(stf_ctx ctx, stf_neural net, stf_neural_block what, const void* host, size_t bytes);
/* Checkpoint: latents, MLP, Adam moments and step counter to / from a file. */
stf_status stf_neural_save(stf_ctx ctx, stf_neural net, const char* path);
stf_status stf_neural_load(stf_ctx ctx, stf_neural net, const char* path);
/* Decode explicit texels on the tensor cores: ix, iy device int32 [n]; y device FP32 [n][8]. */
stf_status stf_neural_decode(stf_ctx ctx, stf_neural net, uint64_t n, const int32_t* ix, const int32_t* iy,
                             float* y);
/* Filter + shade on the decoded texture (level 0, wrap): STOCHASTIC = one decode per
 * sample (POSITIVIZED: two), NTAP_BEFORE = decode every tap, filter, shade once
 * (decode-then-filter), NTAP_AFTER = decode and shade every tap.  Same queries, jitter,
 * RNG and estimators as stf_filter_shade; flags must be 0; picks are not reported. */
stf_status stf_neural_filter_shade(stf_ctx ctx, stf_neural net, const stf_queries* q, const stf_derivs* d,
                                   stf_filter filter, stf_mode mode, stf_shade shade, uint32_t spp,
                                   uint64_t seed, uint32_t flags, const stf_output* out);

/* ---- measurement: the gather roofline's denominator ----------------------------------
 * The paper has no counterpart: this is the measured peak against which the 1-tap kernels'
 * gather rate is reported.  Reads random, independent 32-byte sectors of a device buffer of
 * buffer_bytes (a power of two, 1 MiB .. 1 GiB; a buffer well inside the 126 MB L2 measures
 * the L2 hit rate, one larger than L2 the DRAM sector rate) at L2 (bypassing L1), and writes
 * the best of 3 timed runs as sectors per second to *sectors_per_s (host).  Allocates and
 * frees the buffer; synchronises the context stream.  STF_ERR_INVALID_ARG for a bad size or
 * a null output. */
stf_status stf_measure_sector_rate(stf_ctx ctx, uint64_t buffer_bytes, double* sectors_per_s);

#ifdef __cplusplus
}
#endif
#endif /* STF_H */
