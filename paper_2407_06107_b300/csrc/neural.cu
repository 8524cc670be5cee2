// Learned form: neural texture (4 FP16 / FP8 latent grids + MLP 32->64->64->8) trained by
// hand-written forward/backward/Adam kernels and decoded on the 5th-generation tensor
// cores (tcgen05.mma kind::f16, BF16 operands in shared memory, FP32 accumulators in
// TMEM).  Stochastic filtering decodes the MLP once per lookup instead of once per filter
// tap (Sec. 4: one texel per lookup inside the filter integral).
//
// Decode tile: 128 rows (one row = one texel decode).  Per tile:
//   rows -> latent features (bilinear, FP32, fixed order) -> BF16 A tile (smem)
//   MMA1 128x64x32 -> TMEM -> +b1, ReLU, BF16 -> A tile
//   MMA2 128x64x64 -> TMEM -> +b2, ReLU, BF16 -> A tile
//   MMA3 128x16x64 (8 outputs padded to N=16) -> TMEM -> +b3 -> shade / store.
// Shared-memory operands use the no-swizzle K-major canonical layout: 8-row x 16-byte core
// matrices; core matrices adjacent along K are 128 B apart (LBO), 8-row groups are
// (K/8)*128 B apart (SBO).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "stf_device.cuh"
#include "stf_kernels.h"

namespace stf {

// ------------------------------------------------------------------ PTX helpers

// Packed FP32 pairs (pk2, upk2, mul2, add2, fma2: .f32x2, one rounding per lane) come from
// stf_device.cuh.
// BF16 pair (lo in the low half) of a packed FP32 pair, round to nearest; with RELU,
// negative values become 0 (ReLU then rounding equals rounding then ReLU)
template <bool RELU>
__device__ __forceinline__ uint32_t bf16x2_of(uint64_t v) {
    const float2 f = upk2(v);
    uint32_t r;
    if (RELU) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(f.y), "f"(f.x));
    else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(f.y), "f"(f.x));
    return r;
}

// Bounded wait on an mbarrier phase: gives up after ~max_cycles SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long max_cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > max_cycles) return false;
    return true;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, relative LBO, layout SWIZZLE_NONE
}
// instruction descriptor, kind::f16: D = FP32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// The same two, executed by a whole warp: elect.sync picks one lane (the lowest, the same on
// every call with the full mask) to issue, so the warp's control flow and operands stay uniform.
__device__ __forceinline__ void mma_bf16_warp(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit_warp(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
        ::"r"(smem_u32(bar))
        : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element (row, k) in a K-major no-swizzle tile with K columns
__host__ __device__ constexpr uint32_t kmaj_off(uint32_t row, uint32_t k, uint32_t K) {
    return (row >> 3) * (K / 8) * 128u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

// ------------------------------------------------------------------ latent features
// bilinear taps of grid g at the centre of texel (ix, iy): FP32 in the oracle's order
struct LTap { int x0, y0, x1, y1; float w00, w10, w01, w11; };
__device__ __forceinline__ LTap latent_taps(const NeuralView& N, int g, int ix, int iy) {
    const float s = N.gscale[g];
    const float px = __fmaf_rn(__fadd_rn((float)ix, 0.5f), s, -0.5f);
    const float py = __fmaf_rn(__fadd_rn((float)iy, 0.5f), s, -0.5f);
    const float fx = floorf(px), fy = floorf(py);
    const float tx = __fsub_rn(px, fx), ty = __fsub_rn(py, fy);
    const float ux = __fsub_rn(1.0f, tx), uy = __fsub_rn(1.0f, ty);
    LTap t;
    const int R = N.res[g];
    // ix, iy lie in [0, tex_res), so p lies in [-1/2, R - 1/2) and floor(p) in [-1, R - 1]: the
    // wrap is -1 -> R - 1 alone, a select
    const int ix0 = (int)fx, iy0 = (int)fy;
    t.x0 = ix0 < 0 ? R - 1 : ix0; t.y0 = iy0 < 0 ? R - 1 : iy0;
    t.x1 = t.x0 + 1 == R ? 0 : t.x0 + 1;     // the next texel, wrapped
    t.y1 = t.y0 + 1 == R ? 0 : t.y0 + 1;
    t.w00 = __fmul_rn(ux, uy); t.w10 = __fmul_rn(tx, uy); t.w01 = __fmul_rn(ux, ty); t.w11 = __fmul_rn(tx, ty);
    return t;
}

// 8 FP32 master latent channels of one grid texel (32 bytes, one sector) as 4 packed pairs:
// one 256-bit load, read-only during the kernel and not kept in L1 (random texels have no
// reuse within an SM; L1 stays for the registers a thread spills)
__device__ __forceinline__ void load_master8(const NeuralView& N, int g, int x, int y, uint64_t v[4]) {
    const float* p = N.lat32 + N.lat_off[g] + ((size_t)y * N.res[g] + x) * 8;
    float a[8];
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
                 : "l"(p));
    v[0] = pk2(a[0], a[1]); v[1] = pk2(a[2], a[3]); v[2] = pk2(a[4], a[5]); v[3] = pk2(a[6], a[7]);
}

// Inference form (FP16 or FP8 latents): the four taps of a grid as raw 16-byte (FP16) or
// 8-byte (FP8, in .x .y) texels, and their conversion to packed FP32 pairs.
template <int LF>
__device__ __forceinline__ void load_taps_raw(const NeuralView& N, int g, const LTap& t, uint4 q[4]) {
    const int xs[4] = {t.x0, t.x1, t.x0, t.x1}, ys[4] = {t.y0, t.y0, t.y1, t.y1};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const size_t o = ((size_t)ys[i] * N.res[g] + xs[i]) * 8;
        if constexpr (LF == 0) {
            q[i] = __ldg(reinterpret_cast<const uint4*>(N.lat16 + N.lat_off[g] + o));
        } else {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(N.lat8 + N.lat_off[g] + o));
            q[i] = make_uint4(v.x, v.y, 0u, 0u);
        }
    }
}
template <int LF>
__device__ __forceinline__ void raw_to_pairs(const NeuralView& N, int g, uint4 q, uint64_t v[4]) {
    if constexpr (LF == 0) {
        const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) { const float2 f = __half22float2(h[i]); v[i] = pk2(f.x, f.y); }
    } else {
        const uint8_t* b = reinterpret_cast<const uint8_t*>(&q);
        const uint64_t sc = pk2(N.scale[g], N.scale[g]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_fp8_e4m3 e0, e1;
            e0.__x = b[2 * i];
            e1.__x = b[2 * i + 1];
            v[i] = mul2(pk2((float)e0, (float)e1), sc);
        }
    }
}
// The 32 features of one decode row, rounded to BF16 and stored grid by grid into row
// `row` of the K-major A tile (same order and rounding as master_features).  The four taps of
// grid g+1 are loaded before grid g is interpolated, so two grids' gathers are in flight.
// LF: the latent format (0 FP16, 1 FP8 x scale), fixed per kernel instantiation.
template <int LF, int KA = 32>
__device__ __forceinline__ void features_to_tile(const NeuralView& N, int ix, int iy, uint8_t* A, int row) {
    LTap tc = latent_taps(N, 0, ix, iy);
    uint4 cur[4];
    load_taps_raw<LF>(N, 0, tc, cur);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint4 nxt[4];
        LTap tn = tc;
        if (g < 3) {
            tn = latent_taps(N, g + 1, ix, iy);
            load_taps_raw<LF>(N, g + 1, tn, nxt);
        }
        uint64_t a[4], b[4], c[4], d[4];
        raw_to_pairs<LF>(N, g, cur[0], a);
        raw_to_pairs<LF>(N, g, cur[1], b);
        raw_to_pairs<LF>(N, g, cur[2], c);
        raw_to_pairs<LF>(N, g, cur[3], d);
        const uint64_t w00 = pk2(tc.w00, tc.w00), w10 = pk2(tc.w10, tc.w10);
        const uint64_t w01 = pk2(tc.w01, tc.w01), w11 = pk2(tc.w11, tc.w11);
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint64_t v = mul2(w00, a[k]);
            v = fma2(w10, b[k], v);
            v = fma2(w01, c[k], v);
            o[k] = bf16x2_of<false>(fma2(w11, d[k], v));
        }
        *reinterpret_cast<uint4*>(A + kmaj_off(row, 8 * g, KA)) = make_uint4(o[0], o[1], o[2], o[3]);
        if (g < 3) {
#pragma unroll
            for (int i = 0; i < 4; ++i) cur[i] = nxt[i];
            tc = tn;
        }
    }
}

// ------------------------------------------------------------------ optimiser
// Adam with bias correction; consumes and zeroes the gradient
struct AdamConst { float lr, b1, b2, eps, c1, c2; };
__device__ __forceinline__ void adam1(float& p, float& g, float& m, float& v, const AdamConst& A) {
    const float gi = g;
    m = fmaf(A.b1, m, (1.0f - A.b1) * gi);
    v = fmaf(A.b2, v, (1.0f - A.b2) * gi * gi);
    g = 0.0f;
    p -= A.lr * (m / A.c1) / (sqrtf(v / A.c2) + A.eps);
}
// The arrays are 16-byte aligned: four parameters per thread and iteration with 16-byte
// loads and stores (the step is HBM-bound: 32 bytes per parameter), then the scalar tail.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       uint64_t n, AdamConst A) {
    const uint64_t n4 = n / 4, stride = (uint64_t)gridDim.x * blockDim.x;
    float4 *p4 = reinterpret_cast<float4*>(p), *g4 = reinterpret_cast<float4*>(g);
    float4 *m4 = reinterpret_cast<float4*>(m), *v4 = reinterpret_cast<float4*>(v);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 pp = p4[i], gg = g4[i], mm = m4[i], vv = v4[i];
        adam1(pp.x, gg.x, mm.x, vv.x, A);
        adam1(pp.y, gg.y, mm.y, vv.y, A);
        adam1(pp.z, gg.z, mm.z, vv.z, A);
        adam1(pp.w, gg.w, mm.w, vv.w, A);
        p4[i] = pp; g4[i] = gg; m4[i] = mm; v4[i] = vv;
    }
    for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        adam1(p[i], g[i], m[i], v[i], A);
}

// ------------------------------------------------------------------ quantisation
__global__ void k_to_fp16(const float* __restrict__ src, __half* __restrict__ dst, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}
// per-grid max |latent| (non-negative floats order like their bit patterns)
__global__ void k_absmax(const float* __restrict__ src, uint64_t n, unsigned int* out) {
    float m = 0.0f;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(src[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}
// FP8 E4M3 (round to nearest even, saturating to +-448) of latent / scale
__global__ void k_to_e4m3(const float* __restrict__ src, uint8_t* __restrict__ dst, uint64_t n, const unsigned int* amax) {
    const float scale = fmaxf(__uint_as_float(*amax), 1e-30f) / 448.0f;
    const float inv = 1.0f / scale;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (uint8_t)__nv_cvt_float_to_fp8(src[i] * inv, __NV_SATFINITE, __NV_E4M3);
}
__global__ void k_scale_from_amax(const unsigned int* amax, float* scale, int n) {
    if (threadIdx.x < n) scale[threadIdx.x] = fmaxf(__uint_as_float(amax[threadIdx.x]), 1e-30f) / 448.0f;
}
// MLP master -> BF16 weights [W1 64x32 | W2 64x64 | W3 padded 16x64] and FP32 biases [b1|b2|b3 pad 16]
__global__ void k_pack_mlp(const float* __restrict__ P, __nv_bfloat16* __restrict__ wb, float* __restrict__ bias) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2048 + 4096 + 1024; i += gridDim.x * blockDim.x) {
        float w;
        if (i < 2048) w = P[i];
        else if (i < 6144) w = P[2048 + 64 + (i - 2048)];
        else { const int j = i - 6144; w = j < 512 ? P[2048 + 64 + 4096 + 64 + j] : 0.0f; }
        wb[i] = __float2bfloat16_rn(w);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 64 + 64 + 16; i += gridDim.x * blockDim.x) {
        float b;
        if (i < 64) b = P[2048 + i];
        else if (i < 128) b = P[2048 + 64 + 4096 + (i - 64)];
        else { const int j = i - 128; b = j < 8 ? P[2048 + 64 + 4096 + 64 + 512 + j] : 0.0f; }
        bias[i] = b;
    }
}

// Part p (0, 1, 2) of an FP32 value split into three BF16 values whose sum is exact: the
// rounding h of b, the rounding m of b - h (exact in FP32), and b - h - m (at most 8
// significant bits, so exactly a BF16 value).
__device__ __forceinline__ __nv_bfloat16 bf16_part(float b, int p) {
    const __nv_bfloat16 h = __float2bfloat16_rn(b);
    const float r1 = __fsub_rn(b, __bfloat162float(h));
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(m));
    return p == 0 ? h : (p == 1 ? m : __float2bfloat16_rn(r2));
}
// MLP master -> BF16 weights with the biases folded in as three extra K columns each (see
// NeuralView::wext): a GEMM over [x | 1 1 1 | 0..] then adds the FP32 bias exactly, as
// three exact products inside the FP32 accumulation.
__global__ void k_pack_mlp_ext(const float* __restrict__ P, __nv_bfloat16* __restrict__ w) {
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 64 * 48 + 64 * 80 + 16 * 80; i += gridDim.x * blockDim.x) {
        __nv_bfloat16 v = zero;
        if (i < 64 * 48) {
            const int o = i / 48, k = i % 48;
            if (k < 32) v = __float2bfloat16_rn(P[o * 32 + k]);
            else if (k < 35) v = bf16_part(P[2048 + o], k - 32);
        } else if (i < 64 * 48 + 64 * 80) {
            const int j = i - 64 * 48, o = j / 80, k = j % 80;
            if (k < 64) v = __float2bfloat16_rn(P[2112 + o * 64 + k]);
            else if (k < 67) v = bf16_part(P[6208 + o], k - 64);
        } else {
            const int j = i - 64 * 48 - 64 * 80, o = j / 80, k = j % 80;
            if (o < 8) {
                if (k < 64) v = __float2bfloat16_rn(P[6272 + o * 64 + k]);
                else if (k < 67) v = bf16_part(P[6784 + o], k - 64);
            }
        }
        w[i] = v;
    }
}

// ------------------------------------------------------------------ tensor-core decode
constexpr int NT_ROWS = 128;
constexpr uint32_t TMEM_COLS = 64;     // the three layers reuse columns 0..63 in turn
constexpr int DEC_CTAS_PER_SM = 6;     // 6 x 64 TMEM columns <= 512, 6 x ~37 KB smem <= 228 KB
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

struct __align__(128) DecodeSmem {
    // 16 KB operand tile: the features (K = 32, first 8 KB) for layer 1, then the hidden
    // activations (K = 64) for layers 2 and 3; each write happens after the MMA that read
    // the previous contents has completed
    uint8_t A[NT_ROWS * 64 * 2];
    uint8_t W1[64 * 32 * 2];          // 4 KB
    uint8_t W2[64 * 64 * 2];          // 8 KB
    uint8_t W3[16 * 64 * 2];          // 2 KB (rows 8..15 zero)
    float bias[64 + 64 + 16];
    float ch[NT_ROWS][9];             // decoded channels per row
    float wt[NT_ROWS];                // row weight
    long long pair[NT_ROWS];          // query of the row's (query, sample) pair, -1 = idle
    uint64_t bar;
    uint32_t tmem;
    int abort_flag;
};

// copy a row-major [N][K] BF16 matrix into the K-major no-swizzle core-matrix layout
__device__ __forceinline__ void stage_weights(uint8_t* dst, const __nv_bfloat16* src, int Nr, int K) {
    const int chunks = Nr * K / 8;          // 16-byte chunks
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        const int row = c / (K / 8), kc = c % (K / 8);
        const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)row * K + kc * 8);
        *reinterpret_cast<uint4*>(dst + kmaj_off(row, kc * 8, K)) = v;
    }
}

// Rows per (query, sample) pair: 1 (stochastic), 2 (positivized), NT x NT (N-tap).  They
// divide the 128-row tile, so a pair's rows form an aligned group inside one tile.
template <int FILTER, int MODE>
__host__ __device__ constexpr int rows_per_pair() {
    return (MODE == M_STOCHASTIC) ? 1 : (MODE == M_POSITIVIZED ? 2 : ntaps(FILTER) * ntaps(FILTER));
}

// Row generation for the filter modes: row -> (query, texel, weight); query -1 = idle.
struct RowOut { long long query; int ix, iy; float w; };

template <int FILTER, int MODE>
__device__ __forceinline__ RowOut make_row(const NeuralDecodeArgs& a, const RoundKeys& K, uint64_t row) {
    constexpr int NT = ntaps(FILTER), T0 = tap0(FILTER);
    constexpr int NR = rows_per_pair<FILTER, MODE>();
    RowOut o{-1, 0, 0, 0.0f};
    const uint64_t pair = row / NR;
    const int j = (int)(row % NR);
    const uint64_t npairs = a.n * (uint64_t)a.spp;
    if (pair >= npairs) return o;
    uint64_t q;
    uint32_t s;
    if ((a.spp & (a.spp - 1)) == 0u) {    // a power of two: a shift and a mask
        const int sh = __popc(a.spp - 1);
        q = pair >> sh;
        s = (uint32_t)pair & (a.spp - 1);
    } else if (npairs <= 0xFFFFFFFFull) {   // 32-bit division (the 64-bit one is a long sequence)
        const uint32_t p32 = (uint32_t)pair;
        q = p32 / a.spp;
        s = p32 - (uint32_t)q * a.spp;
    } else {
        q = pair / a.spp;
        s = (uint32_t)(pair - q * a.spp);
    }
    const uint64_t id = a.id_base + q;
    const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
    const U5 A = uniforms5(philox(id_lo, id_hi, s, 0u, K));
    float x = a.u[q], y = a.v[q];
    if (a.has_derivs) {
        const float jx = __fsub_rn(A.u[0], 0.5f), jy = __fsub_rn(A.u[1], 0.5f);
        x = __fmaf_rn(jy, a.dudy[q], __fmaf_rn(jx, a.dudx[q], x));
        y = __fmaf_rn(jy, a.dvdy[q], __fmaf_rn(jx, a.dvdx[q], y));
    }
    const int R = a.tex_res;
    const AxisPos ax = axis_pos(x, (float)R), ay = axis_pos(y, (float)R);
    float wx[4], wy[4];
    if constexpr (MODE == M_STOCHASTIC) {
        if constexpr (is_signed(FILTER)) {
            axis_pick_weights<FILTER>(ax.t, wx);
            axis_pick_weights<FILTER>(ay.t, wy);
        }
    } else {
        axis_weights<FILTER>(ax.t, wx);
        axis_weights<FILTER>(ay.t, wy);
    }
    o.query = (long long)q;
    if (MODE == M_STOCHASTIC) {
        if constexpr (is_signed(FILTER)) {
            float Sx, Sy;
            bool nx = false, ny = false;
            const int kx = cdf_pick_sign<NT, true>(wx, A.u[3], &Sx, &nx);
            const int ky = cdf_pick_sign<NT, true>(wy, A.u[4], &Sy, &ny);
            o.ix = wrap_index(ax.i0 + T0 + kx, R); o.iy = wrap_index(ay.i0 + T0 + ky, R);
            float W = Sx * Sy;
            if constexpr (pick_weight_scale<FILTER>() != 1.0f) W = __fmul_rn(W, pick_weight_scale<FILTER>());
            o.w = (nx != ny) ? -W : W;
        } else {   // a positive filter: the CDF in closed form, weight 1
            o.ix = wrap_index(ax.i0 + T0 + pick_positive<FILTER>(ax.t, A.u[3]), R);
            o.iy = wrap_index(ay.i0 + T0 + pick_positive<FILTER>(ay.t, A.u[4]), R);
            o.w = 1.0f;
        }
    } else if (MODE == M_POSITIVIZED) {
        float Px, Nx, Py, Ny;
        cdf_pick<NT>(wx, 0.0f, +1, &Px); cdf_pick<NT>(wx, 0.0f, -1, &Nx);
        cdf_pick<NT>(wy, 0.0f, +1, &Py); cdf_pick<NT>(wy, 0.0f, -1, &Ny);
        const float Wp = __fmaf_rn(Nx, Ny, __fmul_rn(Px, Py));
        const float Wn = __fmaf_rn(Nx, Py, __fmul_rn(Px, Ny));
        const U5 B = uniforms5(philox(id_lo, id_hi, s, 1u, K));
        if (j == 0) {
            const int cp = (__fmul_rn(B.u[0], Wp) < __fmul_rn(Px, Py)) ? +1 : -1;
            const int kx = cdf_pick<NT>(wx, A.u[3], cp, nullptr), ky = cdf_pick<NT>(wy, A.u[4], cp, nullptr);
            o.ix = wrap_index(ax.i0 + T0 + kx, R); o.iy = wrap_index(ay.i0 + T0 + ky, R); o.w = Wp;
        } else if (Wn > 0.0f) {
            const int cn = (__fmul_rn(B.u[3], Wn) < __fmul_rn(Px, Ny)) ? +1 : -1;
            const int qx = cdf_pick<NT>(wx, B.u[1], cn, nullptr), qy = cdf_pick<NT>(wy, B.u[2], -cn, nullptr);
            o.ix = wrap_index(ax.i0 + T0 + qx, R); o.iy = wrap_index(ay.i0 + T0 + qy, R); o.w = -Wn;
        } else {
            o.ix = 0; o.iy = 0; o.w = 0.0f;
        }
    } else {
        const int kx = j % NT, ky = j / NT;
        float wsx = wx[0], wsy = wy[0];
#pragma unroll
        for (int k = 1; k < NT; ++k) { wsx = (k == kx) ? wx[k] : wsx; wsy = (k == ky) ? wy[k] : wsy; }
        o.ix = wrap_index(ax.i0 + T0 + kx, R); o.iy = wrap_index(ay.i0 + T0 + ky, R); o.w = wsx * wsy;
    }
    return o;
}

template <int FILTER, int MODE, int LF>
__global__ void __launch_bounds__(NT_ROWS, DEC_CTAS_PER_SM) k_ntc_decode_tc(NeuralView N, NeuralDecodeArgs a, RoundKeys K, ShadeConst SC) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    DecodeSmem& S = *reinterpret_cast<DecodeSmem*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;

    stage_weights(S.W1, N.wbf, 64, 32);
    stage_weights(S.W2, N.wbf + 2048, 64, 64);
    stage_weights(S.W3, N.wbf + 6144, 16, 64);
    for (int i = t; i < 144; i += NT_ROWS) S.bias[i] = N.bias[i];
    if (t == 0) { mbar_init(&S.bar, 1); S.abort_flag = 0; }
    if (warp == 0) tmem_alloc(&S.tmem, TMEM_COLS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t a1 = smem_u32(S.A), a2 = a1;
    const uint32_t w1 = smem_u32(S.W1), w2 = smem_u32(S.W2), w3 = smem_u32(S.W3);
    uint32_t phase = 0;
    bool ok = true;

    const uint64_t nrows = a.nrows;
    const uint64_t ntiles = (nrows + NT_ROWS - 1) / NT_ROWS;
    for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        // ---- rows -> features -> A1
        const uint64_t row = tile * NT_ROWS + t;
        int ix = 0, iy = 0;
        long long pr = -1;
        float w = 0.0f;
        if (row < nrows) {
            if constexpr (MODE < 0) {
                // explicit texels wrap into [0, tex_res) (latent_taps relies on that range)
                ix = wrap_index(a.ex_ix[row], a.tex_res); iy = wrap_index(a.ex_iy[row], a.tex_res);
                pr = (long long)row; w = 1.0f;
            } else {
                const RowOut r = make_row<FILTER, MODE>(a, K, row);
                ix = r.ix; iy = r.iy; pr = r.query; w = r.w;
            }
        }
        S.pair[t] = pr;
        S.wt[t] = w;
        features_to_tile<LF>(N, ix, iy, S.A, t);
        // ---- three GEMM layers
#pragma unroll 1
        for (int layer = 0; layer < 3; ++layer) {
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (t == 0 && !a.inject_timeout) {
                tc_fence_after();
                if (layer == 0) {
                    for (int s = 0; s < 2; ++s)
                        mma_bf16(tmem, smem_desc(a1 + 256 * s, 128, 512), smem_desc(w1 + 256 * s, 128, 512),
                                 idesc_bf16(128, 64), s > 0);
                } else if (layer == 1) {
                    for (int s = 0; s < 4; ++s)
                        mma_bf16(tmem, smem_desc(a2 + 256 * s, 128, 1024), smem_desc(w2 + 256 * s, 128, 1024),
                                 idesc_bf16(128, 64), s > 0);
                } else {
                    for (int s = 0; s < 4; ++s)
                        mma_bf16(tmem, smem_desc(a2 + 256 * s, 128, 1024), smem_desc(w3 + 256 * s, 128, 1024),
                                 idesc_bf16(128, 16), s > 0);
                }
                mma_commit(&S.bar);
            }
            // one thread polls the MMA-completion barrier; the others wait at the block
            // barrier, which costs no issue slots
            if (t == 0 && !mbar_wait_bounded(&S.bar, phase, a.inject_timeout ? 2000000LL : WAIT_CYCLES))
                S.abort_flag = 1;
            phase ^= 1u;
            __syncthreads();
            tc_fence_after();
            if (S.abort_flag) { ok = false; break; }
            if (layer < 2) {
                uint32_t r[4][16];
                const uint32_t col = 0u;
#pragma unroll
                for (int c = 0; c < 4; ++c) tmem_ld16(tmem + lane_base + col + 16 * c, r[c]);
                tmem_wait_ld();
                // bias (FP32 pairs), ReLU and BF16 rounding of 8 columns at a time
                const ulonglong2* bias2 = reinterpret_cast<const ulonglong2*>(S.bias + (layer == 0 ? 0 : 64));
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const ulonglong2 ba = bias2[2 * c], bb = bias2[2 * c + 1];
                    const uint64_t bv[4] = {ba.x, ba.y, bb.x, bb.y};
                    uint32_t p[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k0 = 8 * c + 2 * i;
                        const uint64_t z = add2(pk2(__uint_as_float(r[k0 >> 4][k0 & 15]),
                                                    __uint_as_float(r[(k0 + 1) >> 4][(k0 + 1) & 15])), bv[i]);
                        p[i] = bf16x2_of<true>(z);
                    }
                    *reinterpret_cast<uint4*>(S.A + kmaj_off(t, 8 * c, 64)) = make_uint4(p[0], p[1], p[2], p[3]);
                }
            } else {
                uint32_t r[16];
                tmem_ld16(tmem + lane_base, r);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 8; ++i) S.ch[t][i] = __uint_as_float(r[i]) + S.bias[128 + i];
            }
        }
        if (!ok) break;
        __syncthreads();
        // ---- epilogue
        if constexpr (MODE < 0) {
            if (row < nrows) {
#pragma unroll
                for (int i = 0; i < 8; ++i) a.y_out[row * 8 + i] = S.ch[t][i];
            }
        } else {
            // one thread per (query, sample) pair: the first row of its aligned group
            constexpr int NR = rows_per_pair<FILTER, MODE>();
            const long long qq = S.pair[t];
            if (qq >= 0 && t % NR == 0) {
                float est[3] = {0.f, 0.f, 0.f};
                if constexpr (MODE == M_NTAP_BEFORE) {
                    float c[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    for (int r = t; r < t + NR; ++r)
                        for (int i = 0; i < 8; ++i) c[i] = fmaf(S.wt[r], S.ch[r][i], c[i]);
                    const float3 f3 = shade<false>(a.shade, material_from_channels(c), SC);
                    est[0] = f3.x; est[1] = f3.y; est[2] = f3.z;
                } else {
                    for (int r = t; r < t + NR; ++r) {
                        if (S.wt[r] == 0.0f) continue;
                        const float3 f3 = shade<false>(a.shade, material_from_channels(S.ch[r]), SC);
                        est[0] = fmaf(S.wt[r], f3.x, est[0]);
                        est[1] = fmaf(S.wt[r], f3.y, est[1]);
                        est[2] = fmaf(S.wt[r], f3.z, est[2]);
                    }
                }
                const uint64_t q = (uint64_t)qq;
                const float inv = 1.0f / (float)a.spp;
                atomicAdd(a.r + q, est[0] * inv);
                atomicAdd(a.g + q, est[1] * inv);
                atomicAdd(a.b + q, est[2] * inv);
            }
        }
        __syncthreads();
    }
    if (!ok && t == 0) atomicOr(a.status, DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------ warp-specialised 1-tap decode
// The stochastic (one decode per sample) filter + shade of the learned texture as a pipeline
// per CTA whose stages hand 128-row tiles over through mbarriers instead of block barriers:
//   warps 0-3, producers: row r of a tile = (query, sample) r -> Philox pick, 16 latent
//     gathers and FP32 bilinear features -> the BF16 A tile (two buffers, so the next tile is
//     gathered while this one is in the GEMMs);
//   warp 8, one lane: the three tcgen05.mma layers of each tile;
//   warps 4-7, epilogue (TMEM lanes 0-127, one per row): each hidden layer's ReLU and BF16
//     rounding from TMEM into the H tile, then the 8 channels -> material -> GGX, and each
//     query's mean over its samples.
// The biases ride in the GEMMs as three extra K columns (NeuralView::wext, ones in A and H),
// so an epilogue is a TMEM load, a fused ReLU-and-round and a shared store.  TMEM: layers 1 and
// 2 accumulate in columns 0-63, layer 3 in 64-79.  Every wait is bounded; a timeout makes every
// role leave its loop, and the kernel reports DEV_TIMEOUT.
constexpr int WS_THREADS = 288;
constexpr int WS_CTAS_PER_SM = 3;
constexpr uint32_t WS_TMEM_COLS = 128;
constexpr int WS_K1 = 48, WS_K2 = 80;

struct __align__(128) DecWsSmem {
    uint8_t A[2][NT_ROWS * WS_K1 * 2];   // features | 1 1 1 | 0 (K-major, no swizzle)
    uint8_t H[NT_ROWS * WS_K2 * 2];      // hidden activations | 1 1 1 | 0
    uint8_t W1[64 * WS_K1 * 2];
    uint8_t W2[64 * WS_K2 * 2];
    uint8_t W3[16 * WS_K2 * 2];          // rows 8..15 zero
    long long q[2][NT_ROWS];             // query of each row of an A buffer (-1: idle)
    float w[2][NT_ROWS];                 // the row's weight (sign * S_x * S_y for a signed filter)
    uint64_t full_a[2], a_free[2], mma1, mma2, mma3, h1, h2, fin;
    uint32_t tmem;
    volatile int abort_flag;
};
static_assert(sizeof(DecWsSmem) * WS_CTAS_PER_SM + 3 * 1024 <= 228 * 1024, "three CTAs per SM");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once any role has given up.  The abort flag and the clock
// are read on every 8th poll only, so a waiting warp spends fewer issue slots polling.
__device__ __forceinline__ bool ws_wait1(volatile int* abort_flag, uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 7u) == 0u && (*abort_flag || clock64() - t0 > limit)) {
            *abort_flag = 1;
            return false;
        }
    }
}
// The same for a whole warp: every lane waits, and the decision is the warp's (__all_sync), so
// a warp whose lanes then run collective instructions (TMEM loads, shuffles) never leaves a
// loop with some lanes only.
__device__ __forceinline__ bool ws_wait(volatile int* abort_flag, uint64_t* bar, uint32_t parity, long long limit) {
    return __all_sync(0xFFFFFFFFu, ws_wait1(abort_flag, bar, parity, limit));
}
// ReLU, then BF16 round-to-nearest, of two FP32 values (lo in the low half)
__device__ __forceinline__ uint32_t relu_bf16x2(uint32_t lo, uint32_t hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
    return r;
}
// one row of a hidden layer: TMEM columns 0..63 of this lane -> ReLU -> BF16 -> row `row` of H
__device__ __forceinline__ void ws_hidden(uint32_t taddr, uint8_t* H, int row) {
    uint32_t r[4][16];
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_ld16(taddr + 16 * c, r[c]);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 8 * c + 2 * i;
            p[i] = relu_bf16x2(r[k >> 4][k & 15], r[(k + 1) >> 4][(k + 1) & 15]);
        }
        *reinterpret_cast<uint4*>(H + kmaj_off(row, 8 * c, WS_K2)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
}
// the constant columns K0 .. K0+15 of a tile row: 1 1 1 then zeros (bias columns)
__device__ __forceinline__ void ws_ones(uint8_t* tile, int row, int K0, int K) {
    *reinterpret_cast<uint4*>(tile + kmaj_off(row, K0, K)) = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
    *reinterpret_cast<uint4*>(tile + kmaj_off(row, K0 + 8, K)) = make_uint4(0u, 0u, 0u, 0u);
}

template <int FILTER, int LF>
__global__ void __launch_bounds__(WS_THREADS, WS_CTAS_PER_SM)
k_ntc_decode_ws(NeuralView N, NeuralDecodeArgs a, RoundKeys K) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    DecWsSmem& S = *reinterpret_cast<DecWsSmem*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const long long limit = a.inject_timeout ? 2000000LL : WAIT_CYCLES;

    stage_weights(S.W1, N.wext, 64, WS_K1);
    stage_weights(S.W2, N.wext + 64 * WS_K1, 64, WS_K2);
    stage_weights(S.W3, N.wext + 64 * WS_K1 + 64 * WS_K2, 16, WS_K2);
    for (int r = t; r < NT_ROWS; r += WS_THREADS) {
        ws_ones(S.A[0], r, 32, WS_K1);
        ws_ones(S.A[1], r, 32, WS_K1);
        ws_ones(S.H, r, 64, WS_K2);
    }
    if (t == 0) {
        mbar_init(&S.full_a[0], NT_ROWS); mbar_init(&S.full_a[1], NT_ROWS);
        mbar_init(&S.a_free[0], 4); mbar_init(&S.a_free[1], 4);
        mbar_init(&S.mma1, 1); mbar_init(&S.mma2, 1); mbar_init(&S.mma3, 1); mbar_init(&S.fin, 1);
        mbar_init(&S.h1, NT_ROWS); mbar_init(&S.h2, NT_ROWS);
        S.abort_flag = 0;
    }
    if (warp == 4) tmem_alloc(&S.tmem, WS_TMEM_COLS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint64_t nrows = a.nrows;
    const uint64_t ntiles = (nrows + NT_ROWS - 1) / NT_ROWS;

    if (warp < 4) {
        // ---------------------------------------------------------------- producers
        for (uint64_t i = 0;; ++i) {
            const uint64_t tile = blockIdx.x + i * gridDim.x;
            if (tile >= ntiles) break;
            const int b = (int)(i & 1);
            if (i >= 2 && !ws_wait(&S.abort_flag, &S.a_free[b], (uint32_t)(((i >> 1) - 1) & 1), limit)) break;
            const uint64_t row = tile * NT_ROWS + t;
            RowOut r{-1, 0, 0, 0.0f};
            if (row < nrows) r = make_row<FILTER, M_STOCHASTIC>(a, K, row);
            S.q[b][t] = r.query;
            S.w[b][t] = r.w;
            features_to_tile<LF, WS_K1>(N, r.ix, r.iy, S.A[b], t);
            fence_async_smem();
            mbar_arrive(&S.full_a[b]);
        }
    } else if (warp == 8) {
        // ---------------------------------------------------------------- MMA issue
        // The whole warp runs the loop and the waits, with warp-uniform control flow and
        // operands; one elected lane (the same every time) issues the MMAs and their commits.
        const uint32_t w1 = smem_u32(S.W1), w2 = smem_u32(S.W2), w3 = smem_u32(S.W3), h = smem_u32(S.H);
        constexpr uint32_t SB1 = (WS_K1 / 8) * 128, SB2 = (WS_K2 / 8) * 128;
        for (uint64_t i = 0;; ++i) {
            const uint64_t tile = blockIdx.x + i * gridDim.x;
            if (tile >= ntiles) break;
            const int b = (int)(i & 1);
            if (!ws_wait(&S.abort_flag, &S.full_a[b], (uint32_t)((i >> 1) & 1), limit)) break;
            tc_fence_after();
            if (!a.inject_timeout) {
                const uint32_t aa = smem_u32(S.A[b]);
#pragma unroll
                for (int s = 0; s < WS_K1 / 16; ++s)
                    mma_bf16_warp(tmem, smem_desc(aa + 256 * s, 128, SB1), smem_desc(w1 + 256 * s, 128, SB1),
                                  idesc_bf16(128, 64), s > 0);
                mma_commit_warp(&S.mma1);
            }
            if (!ws_wait(&S.abort_flag, &S.h1, (uint32_t)(i & 1), limit)) break;
            tc_fence_after();
            if (!a.inject_timeout) {
#pragma unroll
                for (int s = 0; s < WS_K2 / 16; ++s)
                    mma_bf16_warp(tmem, smem_desc(h + 256 * s, 128, SB2), smem_desc(w2 + 256 * s, 128, SB2),
                                  idesc_bf16(128, 64), s > 0);
                mma_commit_warp(&S.mma2);
            }
            if (!ws_wait(&S.abort_flag, &S.h2, (uint32_t)(i & 1), limit)) break;
            tc_fence_after();
            if (!a.inject_timeout) {
#pragma unroll
                for (int s = 0; s < WS_K2 / 16; ++s)
                    mma_bf16_warp(tmem + 64, smem_desc(h + 256 * s, 128, SB2), smem_desc(w3 + 256 * s, 128, SB2),
                                  idesc_bf16(128, 16), s > 0);
                mma_commit_warp(&S.mma3);
            }
        }
        // every MMA the elected lane issued has completed before the TMEM is released
        mma_commit_warp(&S.fin);
        const long long t0 = clock64();
        while (!mbar_try_wait(&S.fin, 0u) && clock64() - t0 < limit) {}
    } else {
        // ---------------------------------------------------------------- epilogue
        const int e = t - 128;                                  // TMEM lane = tile row
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const float inv_spp = 1.0f / (float)a.spp;
        const bool grouped = (32u % a.spp) == 0u;               // a query's samples share a warp
        for (uint64_t i = 0;; ++i) {
            const uint64_t tile = blockIdx.x + i * gridDim.x;
            if (tile >= ntiles) break;
            const int b = (int)(i & 1);
            const uint32_t par = (uint32_t)(i & 1);
            if (!ws_wait(&S.abort_flag, &S.mma1, par, limit)) break;
            // the producers' row data: acquired from their own barrier (its phase for this tile
            // has completed, and it cannot move on before this warp frees the buffer below)
            if (!ws_wait(&S.abort_flag, &S.full_a[b], (uint32_t)((i >> 1) & 1), limit)) break;
            tc_fence_after();
            const long long q = S.q[b][e];
            const float w = S.w[b][e];
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.a_free[b]);
            ws_hidden(taddr, S.H, e);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(&S.h1);
            if (!ws_wait(&S.abort_flag, &S.mma2, par, limit)) break;
            tc_fence_after();
            ws_hidden(taddr, S.H, e);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(&S.h2);
            if (!ws_wait(&S.abort_flag, &S.mma3, par, limit)) break;
            tc_fence_after();
            uint32_t r[16];
            tmem_ld16(taddr + 64, r);
            tmem_wait_ld();
            tc_fence_before();
            float y[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) y[c] = __uint_as_float(r[c]);
            float3 est = make_float3(0.f, 0.f, 0.f);
            if (q >= 0) {
                const Material m = material_from_channels(y);
                float3 f;
                if (a.shade == SH_LINEAR) {
                    f = m.rho;
                } else {
                    float rr, gg, bb;
                    shade_ggx_t<float, false>(mat_t(m), rr, gg, bb);
                    f = make_float3(rr, gg, bb);
                }
                est = make_float3(w * f.x, w * f.y, w * f.z);
            }
            if (grouped) {
                // butterfly sum over the query's spp consecutive lanes, then one store
                for (uint32_t o = 1; o < a.spp; o <<= 1) {
                    est.x += __shfl_xor_sync(0xFFFFFFFFu, est.x, o);
                    est.y += __shfl_xor_sync(0xFFFFFFFFu, est.y, o);
                    est.z += __shfl_xor_sync(0xFFFFFFFFu, est.z, o);
                }
                if (q >= 0 && (uint32_t)e % a.spp == 0u) {
                    a.r[q] = est.x * inv_spp;
                    a.g[q] = est.y * inv_spp;
                    a.b[q] = est.z * inv_spp;
                }
            } else if (q >= 0) {
                atomicAdd(a.r + q, est.x * inv_spp);
                atomicAdd(a.g + q, est.y * inv_spp);
                atomicAdd(a.b + q, est.z * inv_spp);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (t == 0 && S.abort_flag) atomicOr(a.status, DEV_TIMEOUT);
    tc_fence_after();
    if (warp == 4) tmem_dealloc(tmem, WS_TMEM_COLS);
}

// ------------------------------------------------------------------ training (tcgen05)
// One training sample (one row) per thread of a 128-sample tile.  Forward: the decode's three
// GEMMs on BF16 operands, the biases folded in.  Backward, per tile:
//   dH2 = dY W3            (A dY, K-major;  B W3 read MN-major)          -> TMEM scratch
//   dW3 | db3 += dY^T [H2 | 1]  (A the dY tile read MN-major; B the H2 tile MN-major)
//   dH1 = dZ2 W2,  dW2 | db2 += dZ2^T [H1 | 1]
//   dX  = dZ1 W1,  dW1 | db1 += dZ1^T [X | 1]
// with dZ = dH (.) [Z > 0] and dY = 2 (y - target) / (8 batch), each rounded to BF16 as a
// GEMM operand.  The activation tiles are written once, row = sample, in the K-major layout
// of the forward GEMMs.  A K-major core matrix (8 samples x 8 features) is also an MN-major
// core matrix of the transposed tile (8 features contiguous, 8 samples), so the
// weight-gradient GEMMs read the same bytes with features along M or N and samples along K;
// the weights, stored K-major for the forward, are read MN-major as the backward's B.
// A block of ones after the features of X, H1 and H2 adds the bias in the forward GEMMs and
// makes each bias gradient one more column of a weight-gradient accumulator.  dZ2 is written
// over H2 once the layer-3 GEMMs have read H2, and dZ1 over H1 once the layer-2 GEMMs have
// read H1; both keep the ones block of the tile they replace.
//
// The weight-gradient GEMMs run at M = 64 (the 64 output features of a layer; dY's 8 and
// padding), K = the tile's 128 samples; their accumulators (80 + 48 + 80 columns) sum over
// every tile of the CTA.  An M = 64 accumulator keeps row r in TMEM lane 32 (r / 16) + r % 16:
// lanes 0..15 of each 32-lane quarter.  Rather than one tile per CTA, waiting on every GEMM
// round, a CTA (one per SM, all 512 TMEM columns) keeps TRW_GROUPS tiles in flight: each
// group of four warps owns one tile at a time (gathers, epilogues, loss, latent-gradient
// scatter) with its own 64 scratch columns, and one MMA thread serves the groups in whatever
// order their stages become ready.  Only that thread issues MMAs, so the weight-gradient
// GEMMs of all groups accumulate into one set of accumulators in issue order.  Hand-over per
// stage: the group's 128 threads arrive on ready[g] after writing their rows (generic-proxy
// writes fenced to the async proxy); the MMA thread issues the stage and commits to done[g];
// the group waits on done[g].  Every wait is bounded; a role that gives up sets abort_flag,
// which ends every other wait.
constexpr int TR_ROWS = 128;
constexpr int TRW_GROUPS = 3;
constexpr int TRW_THREADS = TRW_GROUPS * TR_ROWS + 32;
constexpr uint32_t TRW_TMEM_COLS = 512;
constexpr uint32_t TW_DW2 = 0, TW_DW1 = 80, TW_DW3 = 128;   // accumulator columns (80, 48, 80)
constexpr uint32_t TW_SCRATCH = 256;                          // group g: columns 256 + 64 g ..
constexpr int FX = 48, FH = 80, FY = 16;                      // row lengths of the tiles (elements)
constexpr uint32_t IDESC_A_MN = 1u << 15, IDESC_B_MN = 1u << 16;

struct TrwGroup {
    uint8_t X[TR_ROWS * FX * 2];      // 32 latent features | 16 ones
    uint8_t H1[TR_ROWS * FH * 2];     // 64 activations | 16 ones; later dZ1 | 16 ones
    uint8_t H2[TR_ROWS * FH * 2];     // 64 activations | 16 ones; later dZ2 | 16 ones
    uint8_t dY[TR_ROWS * FY * 2];     // 8 output gradients | 8 zeros
};
struct __align__(128) TrainWsSmem {
    TrwGroup grp[TRW_GROUPS];
    // BF16 weights with the biases folded in (K-major): W1 | b1 [64][48], W2 | b2 [64][80],
    // W3 | b3 [16][80] (rows 8..15 zero); the bias columns meet the ones blocks of X, H1, H2
    uint8_t W1[64 * FX * 2], W2[64 * FH * 2], W3[16 * FH * 2];
    uint64_t ready[TRW_GROUPS], done[TRW_GROUPS], fin;
    uint32_t tmem;
    volatile int abort_flag;
    int acc_valid;
    float red[TRW_GROUPS * 4];
};
static_assert(TW_SCRATCH + 64 * TRW_GROUPS <= TRW_TMEM_COLS, "scratch columns of every group");
static_assert(TW_DW3 + 80 <= TW_SCRATCH, "accumulators below the scratch columns");
// The M = 64 read of dY (16 columns) as 64 features runs past the dY tile by at most
// 15 x 256 + 8 x 128 - 4,096 = 768 B, into the next group's X tile or, after the last
// group, into W1 (rows >= 8 of that accumulator are never read)
static_assert(15 * FY * 16 + 8 * 128 - TR_ROWS * FY * 2 <= 64 * FX * 2, "dY over-read stays in the struct");
static_assert(2 * sizeof(TrainWsSmem) > 228 * 1024, "one CTA per SM: it allocates all 512 TMEM columns");
static_assert(sizeof(TrainWsSmem) + 1024 <= 227 * 1024, "shared memory of one CTA");

// FP32 master weights W [rows][Kw] and bias b [rows] (rows >= present are zero) -> BF16
// K-major tile [rows][Kt]: W, then the bias as three exact BF16 parts, then zeros.  Against
// a ones block in the activation tile the three parts add the FP32 bias inside the GEMM.
__device__ __forceinline__ void stage_weights_ext(uint8_t* dst, const float* W, const float* b, int rows, int Kw,
                                                  int Kt, int present) {
    const int chunks = rows * Kt / 8;
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        const int row = c / (Kt / 8), kc = c % (Kt / 8);
        uint32_t p[4] = {0u, 0u, 0u, 0u};
        if (row < present) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = 8 * kc + i;
                __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
                if (k < Kw) v = __float2bfloat16_rn(W[(size_t)row * Kw + k]);
                else if (k < Kw + 3) v = bf16_part(b[row], k - Kw);
                p[i >> 1] |= (uint32_t)__bfloat16_as_ushort(v) << (16 * (i & 1));
            }
        }
        *reinterpret_cast<uint4*>(dst + kmaj_off(row, kc * 8, Kt)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
}

// Descriptor of an MN-major no-swizzle operand: core matrices (8 K rows x 16 B along MN)
// mn_stride apart along MN and k_stride apart along K.  As for K-major operands, the
// leading byte offset is the stride along K and the stride byte offset the one along M or
// N (the gradient tests fail with the two exchanged).
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t mn_stride, uint32_t k_stride) {
    return smem_desc(saddr, k_stride, mn_stride);
}

// The 32 features of a training sample from the FP32 master latents -> BF16 row `row` of the
// X tile: per grid and channel, w00 a + w10 b + w01 c + w11 d in this order, each step one
// rounding (the oracle's order).  Two grids' gathers (16 loads, 64 registers) are in flight
// at a time, so a 128-register thread does not spill.
__device__ __forceinline__ void master_features_to_tile(const NeuralView& N, int ix, int iy, uint8_t* X, int row) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        LTap t[2];
        uint64_t a[2][4], b[2][4], c[2][4], d[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            t[q] = latent_taps(N, 2 * h + q, ix, iy);
            load_master8(N, 2 * h + q, t[q].x0, t[q].y0, a[q]);
            load_master8(N, 2 * h + q, t[q].x1, t[q].y0, b[q]);
            load_master8(N, 2 * h + q, t[q].x0, t[q].y1, c[q]);
            load_master8(N, 2 * h + q, t[q].x1, t[q].y1, d[q]);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint64_t w00 = pk2(t[q].w00, t[q].w00), w10 = pk2(t[q].w10, t[q].w10);
            const uint64_t w01 = pk2(t[q].w01, t[q].w01), w11 = pk2(t[q].w11, t[q].w11);
            uint32_t p[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint64_t v = mul2(w00, a[q][k]);
                v = fma2(w10, b[q][k], v);
                v = fma2(w01, c[q][k], v);
                p[k] = bf16x2_of<false>(fma2(w11, d[q][k], v));
            }
            *reinterpret_cast<uint4*>(X + kmaj_off(row, 8 * (2 * h + q), FX)) = make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// Non-blocking test of an mbarrier phase (the MMA thread polls several barriers in turn).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Hidden layer epilogue: 64 pre-activations z (bias included) from TMEM -> ReLU -> BF16 row
// of a tile with F columns, 32 columns at a time
template <int F>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, uint8_t* dst, int row) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t r[2][16];
        tmem_ld16(taddr + 32 * h, r[0]);
        tmem_ld16(taddr + 32 * h + 16, r[1]);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = 8 * c + 2 * i;         // column within this half
                p[i] = relu_bf16x2(r[j >> 4][j & 15], r[(j + 1) >> 4][(j + 1) & 15]);
            }
            *reinterpret_cast<uint4*>(dst + kmaj_off(row, 32 * h + 8 * c, F)) = make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// 0xFFFF in each half of a BF16 pair that is > 0
__device__ __forceinline__ uint32_t positive_mask(uint32_t h) {
    __nv_bfloat162 v;
    memcpy(&v, &h, 4);
    return __hgt2_mask(v, __float2bfloat162_rn(0.0f));
}

// Gradient epilogue: 64 values dH from TMEM -> dZ = dH (.) [z > 0], BF16, written over the
// same row of `tile` (F columns), which holds the layer's ReLU outputs: a ReLU output is
// nonzero exactly where z > 0 (BF16 keeps FP32's exponent range, so a positive FP32 z rounds
// to zero only below 2^-133).  dZ in BF16 is the rounded dH, or 0.
template <int F>
__device__ __forceinline__ void grad_epilogue(uint32_t taddr, uint8_t* tile, int row) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t r[2][16];
        tmem_ld16(taddr + 32 * h, r[0]);
        tmem_ld16(taddr + 32 * h + 16, r[1]);
        uint4 hv[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) hv[c] = *reinterpret_cast<const uint4*>(tile + kmaj_off(row, 32 * h + 8 * c, F));
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t hw[4] = {hv[c].x, hv[c].y, hv[c].z, hv[c].w};
            uint32_t p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = 8 * c + 2 * i;
                const uint32_t d = bf16x2_of<false>(pk2(__uint_as_float(r[j >> 4][j & 15]),
                                                        __uint_as_float(r[(j + 1) >> 4][(j + 1) & 15])));
                p[i] = d & positive_mask(hw[i]);
            }
            *reinterpret_cast<uint4*>(tile + kmaj_off(row, 32 * h + 8 * c, F)) = make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// The GEMMs of one stage of a group's tile (issued by the MMA warp's elected lane).  fresh_*: the first
// accumulation into that weight-gradient accumulator in this CTA overwrites it.
__device__ __forceinline__ void train_stage(TrainWsSmem& S, int g, int stage, uint32_t tmem, bool& fresh3,
                                            bool& fresh2, bool& fresh1) {
    const TrwGroup& G = S.grp[g];
    const uint32_t scr = tmem + TW_SCRATCH + 64u * (uint32_t)g;
    const uint32_t sX = smem_u32(G.X), sH1 = smem_u32(G.H1), sH2 = smem_u32(G.H2), sY = smem_u32(G.dY);
    const uint32_t sW1 = smem_u32(S.W1), sW2 = smem_u32(S.W2), sW3 = smem_u32(S.W3);
    switch (stage) {
    case 0:     // Z1 = [X | 1] [W1 | b1]^T
        for (int s = 0; s < FX / 16; ++s)
            mma_bf16_warp(scr, smem_desc(sX + 256 * s, 128, FX * 16), smem_desc(sW1 + 256 * s, 128, FX * 16),
                     idesc_bf16(128, 64), s > 0);
        break;
    case 1:     // Z2 = [H1 | 1] [W2 | b2]^T
        for (int s = 0; s < FH / 16; ++s)
            mma_bf16_warp(scr, smem_desc(sH1 + 256 * s, 128, FH * 16), smem_desc(sW2 + 256 * s, 128, FH * 16),
                     idesc_bf16(128, 64), s > 0);
        break;
    case 2:     // Y = [H2 | 1] [W3 | b3]^T (8 outputs and 8 zero rows)
        for (int s = 0; s < FH / 16; ++s)
            mma_bf16_warp(scr, smem_desc(sH2 + 256 * s, 128, FH * 16), smem_desc(sW3 + 256 * s, 128, FH * 16),
                     idesc_bf16(128, 16), s > 0);
        break;
    case 3:     // dH2 = dY W3;  dW3 | db3 += dY^T [H2 | 1]
        mma_bf16_warp(scr, smem_desc(sY, 128, FY * 16), mn_desc(sW3, 128, FH * 16), idesc_bf16(128, 64) | IDESC_B_MN, 0);
        for (int s = 0; s < 8; ++s)
            mma_bf16_warp(tmem + TW_DW3, mn_desc(sY + 2 * FY * 16 * s, 128, FY * 16),
                     mn_desc(sH2 + 2 * FH * 16 * s, 128, FH * 16), idesc_bf16(64, 80) | IDESC_A_MN | IDESC_B_MN,
                     (fresh3 && s == 0) ? 0u : 1u);
        fresh3 = false;
        break;
    case 4:     // dH1 = dZ2 W2;  dW2 | db2 += dZ2^T [H1 | 1]   (dZ2 in the H2 tile)
        for (int s = 0; s < 4; ++s)
            mma_bf16_warp(scr, smem_desc(sH2 + 256 * s, 128, FH * 16), mn_desc(sW2 + 2 * FH * 16 * s, 128, FH * 16),
                     idesc_bf16(128, 64) | IDESC_B_MN, s > 0);
        for (int s = 0; s < 8; ++s)
            mma_bf16_warp(tmem + TW_DW2, mn_desc(sH2 + 2 * FH * 16 * s, 128, FH * 16),
                     mn_desc(sH1 + 2 * FH * 16 * s, 128, FH * 16), idesc_bf16(64, 80) | IDESC_A_MN | IDESC_B_MN,
                     (fresh2 && s == 0) ? 0u : 1u);
        fresh2 = false;
        break;
    default:    // dX = dZ1 W1;  dW1 | db1 += dZ1^T [X | 1]   (dZ1 in the H1 tile)
        for (int s = 0; s < 4; ++s)
            mma_bf16_warp(scr, smem_desc(sH1 + 256 * s, 128, FH * 16), mn_desc(sW1 + 2 * FX * 16 * s, 128, FX * 16),
                     idesc_bf16(128, 32) | IDESC_B_MN, s > 0);
        for (int s = 0; s < 8; ++s)
            mma_bf16_warp(tmem + TW_DW1, mn_desc(sH1 + 2 * FH * 16 * s, 128, FH * 16),
                     mn_desc(sX + 2 * FX * 16 * s, 128, FX * 16), idesc_bf16(64, 48) | IDESC_A_MN | IDESC_B_MN,
                     (fresh1 && s == 0) ? 0u : 1u);
        fresh1 = false;
        break;
    }
}

constexpr int TRAIN_STAGES = 6;

__global__ void __launch_bounds__(TRW_THREADS, 1)
k_ntc_train_ws(NeuralView N, uint32_t step, uint32_t batch, uint32_t first, uint32_t count, RoundKeys K,
               float* loss_sum, uint32_t use_explicit, const int32_t* ex_ix, const int32_t* ex_iy, uint32_t* status) {
    extern __shared__ __align__(1024) uint8_t train_raw[];
    TrainWsSmem& S = *reinterpret_cast<TrainWsSmem*>(train_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int grp = warp >> 2;                  // tile group; grp == TRW_GROUPS: the MMA warp
    const int e = t - TR_ROWS * grp;            // row of the group's tile = its TMEM lane
    const float* P = N.mlp32;       // W1 [64][32], b1, W2 [64][64], b2, W3 [8][64], b3
    stage_weights_ext(S.W1, P, P + 2048, 64, 32, FX, 64);
    stage_weights_ext(S.W2, P + 2112, P + 6208, 64, 64, FH, 64);
    stage_weights_ext(S.W3, P + 6272, P + 6784, 16, 64, FH, 8);
    if (grp < TRW_GROUPS) {   // constant blocks of this thread's rows: ones after the features, zeros after dY
        TrwGroup& G = S.grp[grp];
        const uint4 one = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            *reinterpret_cast<uint4*>(G.X + kmaj_off(e, 32 + 8 * h, FX)) = one;
            *reinterpret_cast<uint4*>(G.H1 + kmaj_off(e, 64 + 8 * h, FH)) = one;
            *reinterpret_cast<uint4*>(G.H2 + kmaj_off(e, 64 + 8 * h, FH)) = one;
        }
        *reinterpret_cast<uint4*>(G.dY + kmaj_off(e, 8, FY)) = zero;
    }
    if (t == 0) {
        for (int g = 0; g < TRW_GROUPS; ++g) { mbar_init(&S.ready[g], TR_ROWS); mbar_init(&S.done[g], 1); }
        mbar_init(&S.fin, 1);
        S.abort_flag = 0;
        S.acc_valid = 0;
    }
    if (warp == 0) tmem_alloc(&S.tmem, TRW_TMEM_COLS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t ntiles = (count + TR_ROWS - 1) / TR_ROWS;
    const uint32_t tstride = gridDim.x * TRW_GROUPS;
    float loss = 0.0f;

    if (grp < TRW_GROUPS) {
        // ---------------------------------------------------------------- tile groups
        TrwGroup& G = S.grp[grp];
        const uint32_t scr = tmem + TW_SCRATCH + 64u * (uint32_t)grp + ((uint32_t)((warp & 3) * 32) << 16);
        const float inv = 1.0f / (8.0f * (float)batch);
        uint32_t handed = 0;     // stages handed over so far (the parity of ready and done)
        // publish this stage's rows to the MMA thread, then wait for its GEMMs
        auto hand_over = [&]() -> bool {
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(&S.ready[grp]);
            const bool ok = ws_wait(&S.abort_flag, &S.done[grp], handed & 1u, WAIT_CYCLES);
            ++handed;
            tc_fence_after();
            return ok;
        };
        // samples first .. first + count - 1 of the step's batch (global ids: the ranks of a
        // data-parallel step draw disjoint parts of the same batch); the loss and gradients are
        // normalised by the whole batch, so the parts' gradients sum to the batch gradient
        for (uint32_t tile = grp * gridDim.x + blockIdx.x; tile < ntiles; tile += tstride) {
            const uint32_t j = tile * TR_ROWS + e;
            const bool live = j < count;
            const uint32_t k = first + j;
            int ix = 0, iy = 0;
            uint2 tgt = make_uint2(0u, 0u);     // the sample's 8 target channels (bytes)
            if (live) {
                if (use_explicit) {   // wrapped into [0, tex_res), the range latent_taps relies on
                    ix = wrap_index(ex_ix[k], (int)N.tex_res); iy = wrap_index(ex_iy[k], (int)N.tex_res);
                }
                else {
                    const uint4 w = philox(k, step, 0u, 0x4E54u, K);
                    ix = (int)__umulhi(w.x, (uint32_t)N.tex_res);
                    iy = (int)__umulhi(w.y, (uint32_t)N.tex_res);
                }
                asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
                             : "=r"(tgt.x), "=r"(tgt.y)
                             : "l"(N.targets + ((size_t)iy * N.tex_res + ix) * 8));
            }
            master_features_to_tile(N, ix, iy, G.X, e);     // FP32 master latents -> BF16 row of X
            if (!hand_over()) break;                                          // Z1
            hidden_epilogue<FH>(scr, G.H1, e);
            if (!hand_over()) break;                                          // Z2
            hidden_epilogue<FH>(scr, G.H2, e);
            if (!hand_over()) break;                                          // Y
            {   // outputs -> MSE loss and dY (BF16 row of the dY tile)
                uint32_t r[16];
                tmem_ld16(scr, r);
                tmem_wait_ld();
                float dy[8];
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const float y = __uint_as_float(r[o]);
                    const uint32_t byte = ((o < 4 ? tgt.x : tgt.y) >> (8 * (o & 3))) & 0xFFu;
                    const float d = live ? y - (float)byte * (1.0f / 255.0f) : 0.0f;
                    loss = fmaf(d * d, inv, loss);
                    dy[o] = 2.0f * d * inv;
                }
                *reinterpret_cast<uint4*>(G.dY + kmaj_off(e, 0, FY)) =
                    make_uint4(bf16x2_of<false>(pk2(dy[0], dy[1])), bf16x2_of<false>(pk2(dy[2], dy[3])),
                               bf16x2_of<false>(pk2(dy[4], dy[5])), bf16x2_of<false>(pk2(dy[6], dy[7])));
            }
            if (!hand_over()) break;                                          // dH2, dW3
            grad_epilogue<FH>(scr, G.H2, e);                                  // dZ2 replaces H2
            if (!hand_over()) break;                                          // dH1, dW2
            grad_epilogue<FH>(scr, G.H1, e);                                  // dZ1 replaces H1
            if (!hand_over()) break;                                          // dX, dW1
            {   // dX -> latent gradients, spread over each grid's 4 taps with the bilinear weights
                uint32_t r0[16], r1[16];
                tmem_ld16(scr, r0);
                tmem_ld16(scr + 16, r1);
                tmem_wait_ld();
                tc_fence_before();
                if (live) {
#pragma unroll
                    for (int gi = 0; gi < 4; ++gi) {
                        const LTap tp = latent_taps(N, gi, ix, iy);
                        float dx[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            dx[c] = __uint_as_float(gi < 2 ? r0[8 * gi + c] : r1[8 * (gi - 2) + c]);
                        float* dl = N.dlat + N.lat_off[gi];
                        const int R = N.res[gi];
                        const int xs[4] = {tp.x0, tp.x1, tp.x0, tp.x1}, ys[4] = {tp.y0, tp.y0, tp.y1, tp.y1};
                        const float ws[4] = {tp.w00, tp.w10, tp.w01, tp.w11};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float4* p = reinterpret_cast<float4*>(dl + ((size_t)ys[q] * R + xs[q]) * 8);
                            atomicAdd(p, make_float4(ws[q] * dx[0], ws[q] * dx[1], ws[q] * dx[2], ws[q] * dx[3]));
                            atomicAdd(p + 1, make_float4(ws[q] * dx[4], ws[q] * dx[5], ws[q] * dx[6], ws[q] * dx[7]));
                        }
                    }
                }
            }
        }
    } else {
        // ---------------------------------------------------------------- MMA warp
        // The whole warp runs the scheduler with warp-uniform decisions and operands; one lane
        // elected inside the issue instructions (elect.sync) issues the MMAs and commits.
        uint32_t left[TRW_GROUPS], stage[TRW_GROUPS], par[TRW_GROUPS];
        uint32_t remaining = 0;
#pragma unroll
        for (int g = 0; g < TRW_GROUPS; ++g) {
            const uint32_t t0 = g * gridDim.x + blockIdx.x;      // the group's first tile
            left[g] = t0 < ntiles ? ((ntiles - 1 - t0) / tstride + 1) * TRAIN_STAGES : 0u;
            stage[g] = 0u;
            par[g] = 0u;
            remaining += left[g];
        }
        bool fresh3 = true, fresh2 = true, fresh1 = true;
        long long since = clock64();
        while (remaining) {
            bool progress = false;
#pragma unroll
            for (int g = 0; g < TRW_GROUPS; ++g) {
                if (left[g] == 0u || !__all_sync(0xFFFFFFFFu, mbar_test_wait(&S.ready[g], par[g]))) continue;
                tc_fence_after();
                train_stage(S, g, (int)stage[g], tmem, fresh3, fresh2, fresh1);
                mma_commit_warp(&S.done[g]);
                stage[g] = stage[g] + 1u == (uint32_t)TRAIN_STAGES ? 0u : stage[g] + 1u;
                par[g] ^= 1u;
                --left[g];
                --remaining;
                progress = true;
            }
            if (progress) since = clock64();
            else if (__any_sync(0xFFFFFFFFu, S.abort_flag || clock64() - since > WAIT_CYCLES)) { S.abort_flag = 1; break; }
        }
        // every MMA the elected lane issued has completed before the accumulators are read
        mma_commit_warp(&S.fin);
        const long long t1 = clock64();
        bool fin = false;
        while (!(fin = mbar_try_wait(&S.fin, 0u)) && clock64() - t1 < WAIT_CYCLES) {}
        if (!__all_sync(0xFFFFFFFFu, fin)) S.abort_flag = 1;
        S.acc_valid = (!fresh1 && remaining == 0u) ? 1 : 0;
        tc_fence_before();
    }
    // loss of this CTA's samples
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
    if (lane == 0 && grp < TRW_GROUPS) S.red[warp] = loss;
    __syncthreads();
    tc_fence_after();
    const bool ok = S.abort_flag == 0;
    if (t == 0) {
        float s = 0.0f;
        for (int w = 0; w < TRW_GROUPS * 4; ++w) s += S.red[w];
        atomicAdd(loss_sum, s);
    }
    // accumulators -> global gradients, read by the first group's warps: lanes 0..15 of warp
    // w hold rows 16 w .. 16 w + 15 (the output features; dW3's rows 0..7)
    if (ok && S.acc_valid && warp < 4) {
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const int row = 16 * warp + lane;
        const bool has = lane < 16;
        float* Gg = N.grad32;
        uint32_t r[16];
#pragma unroll 1
        for (int c = 0; c < 5; ++c) {            // dW2 [64][64] | db2
            tmem_ld16(tmem + lane_base + TW_DW2 + 16 * c, r);
            tmem_wait_ld();
            if (has)
                for (int j = 0; j < 16; ++j) {
                    const int col = 16 * c + j;
                    if (col < 64) atomicAdd(Gg + 2112 + row * 64 + col, __uint_as_float(r[j]));
                    else if (col == 64) atomicAdd(Gg + 6208 + row, __uint_as_float(r[j]));
                }
        }
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {            // dW1 [64][32] | db1
            tmem_ld16(tmem + lane_base + TW_DW1 + 16 * c, r);
            tmem_wait_ld();
            if (has)
                for (int j = 0; j < 16; ++j) {
                    const int col = 16 * c + j;
                    if (col < 32) atomicAdd(Gg + row * 32 + col, __uint_as_float(r[j]));
                    else if (col == 32) atomicAdd(Gg + 2048 + row, __uint_as_float(r[j]));
                }
        }
#pragma unroll 1
        for (int c = 0; c < 5; ++c) {            // dW3 [8][64] | db3
            tmem_ld16(tmem + lane_base + TW_DW3 + 16 * c, r);
            tmem_wait_ld();
            if (has && row < 8)
                for (int j = 0; j < 16; ++j) {
                    const int col = 16 * c + j;
                    if (col < 64) atomicAdd(Gg + 6272 + row * 64 + col, __uint_as_float(r[j]));
                    else if (col == 64) atomicAdd(Gg + 6784 + row, __uint_as_float(r[j]));
                }
        }
    }
    if (!ok && t == 0) atomicOr(status, DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TRW_TMEM_COLS);
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_ntc_train(const NeuralView& N, uint32_t step, uint32_t batch, uint32_t first, uint32_t count,
                             uint64_t seed, float* loss_sum, const int32_t* ex_ix, const int32_t* ex_iy, int num_sms,
                             uint32_t* status, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    // tile i goes to group i / grid of CTA i % grid (cyclically beyond grid x groups): a small
    // batch spreads over one tile per SM before a CTA's second group takes one
    const uint32_t tiles = (count + TR_ROWS - 1) / TR_ROWS;
    const uint32_t cap = (uint32_t)num_sms;
    const int grid = (int)(tiles < cap ? tiles : cap);
    cudaFuncSetAttribute(k_ntc_train_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainWsSmem));
    k_ntc_train_ws<<<grid, TRW_THREADS, sizeof(TrainWsSmem), st>>>(N, step, batch, first, count, expand_key(seed),
                                                                   loss_sum, ex_ix != nullptr, ex_ix, ex_iy, status);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* g, float* m, float* v, uint64_t n, float lr, float b1, float b2, float eps,
                        int t, int num_sms, cudaStream_t st) {
    const AdamConst A{lr, b1, b2, eps, 1.0f - powf(b1, (float)t), 1.0f - powf(b2, (float)t)};
    const uint64_t blocks = (n / 4 + 255) / 256, cap = (uint64_t)num_sms * 16;
    k_adam<<<(int)(blocks < cap ? (blocks ? blocks : 1) : cap), 256, 0, st>>>(p, g, m, v, n, A);
    return cudaGetLastError();
}

cudaError_t launch_ntc_quantize(const NeuralView& N, uint64_t lat_total, int fmt, unsigned int* amax_scratch,
                                cudaStream_t st) {
    k_pack_mlp<<<8, 256, 0, st>>>(N.mlp32, N.wbf, N.bias);
    k_pack_mlp_ext<<<16, 256, 0, st>>>(N.mlp32, N.wext);
    if (fmt == 0) {
        k_to_fp16<<<1024, 256, 0, st>>>(N.lat32, const_cast<__half*>(N.lat16), lat_total);
    } else {
        cudaMemsetAsync(amax_scratch, 0, 4 * sizeof(unsigned int), st);
        for (int g = 0; g < 4; ++g) {
            const uint64_t n = (uint64_t)N.res[g] * N.res[g] * 8;
            k_absmax<<<256, 256, 0, st>>>(N.lat32 + N.lat_off[g], n, amax_scratch + g);
            k_to_e4m3<<<512, 256, 0, st>>>(N.lat32 + N.lat_off[g], const_cast<uint8_t*>(N.lat8) + N.lat_off[g], n,
                                           amax_scratch + g);
        }
        k_scale_from_amax<<<1, 32, 0, st>>>(amax_scratch, N.scale_dev, 4);
    }
    return cudaGetLastError();
}

size_t ntc_decode_smem_bytes() { return sizeof(DecodeSmem) + 1024; }

template <int FILTER, int MODE, int LF>
static cudaError_t launch_dec_lf(const NeuralView& N, const NeuralDecodeArgs& a, int grid, cudaStream_t st) {
    const size_t smem = sizeof(DecodeSmem);
    cudaFuncSetAttribute(k_ntc_decode_tc<FILTER, MODE, LF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ntc_decode_tc<FILTER, MODE, LF><<<grid, NT_ROWS, smem, st>>>(N, a, expand_key(a.seed), make_shade_const());
    return cudaGetLastError();
}
template <int FILTER, int LF>
static cudaError_t launch_dec_ws_lf(const NeuralView& N, const NeuralDecodeArgs& a, int num_sms, cudaStream_t st) {
    const uint64_t tiles = (a.nrows + NT_ROWS - 1) / NT_ROWS;
    const uint64_t cap = (uint64_t)num_sms * WS_CTAS_PER_SM;
    const int grid = (int)(tiles < cap ? (tiles ? tiles : 1) : cap);
    const size_t smem = sizeof(DecWsSmem);
    cudaFuncSetAttribute(k_ntc_decode_ws<FILTER, LF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ntc_decode_ws<FILTER, LF><<<grid, WS_THREADS, smem, st>>>(N, a, expand_key(a.seed));
    return cudaGetLastError();
}
template <int FILTER, int MODE>
static cudaError_t launch_dec(const NeuralView& N, const NeuralDecodeArgs& a, int grid, cudaStream_t st) {
    return N.latent_fmt == 0 ? launch_dec_lf<FILTER, MODE, 0>(N, a, grid, st) : launch_dec_lf<FILTER, MODE, 1>(N, a, grid, st);
}

cudaError_t launch_ntc_decode(const NeuralView& N, const NeuralDecodeArgs& a, int num_sms, cudaStream_t st) {
    const uint64_t tiles = (a.nrows + NT_ROWS - 1) / NT_ROWS;
    const uint64_t cap = (uint64_t)num_sms * DEC_CTAS_PER_SM;
    const int grid = (int)(tiles < cap ? (tiles ? tiles : 1) : cap);
    if (a.mode < 0) return launch_dec<F_LINEAR, -1>(N, a, grid, st);
#define STF_DEC_MODES(F)                                                             \
    if (a.filter == F) {                                                             \
        switch (a.mode) {                                                            \
            case M_NTAP_BEFORE: return launch_dec<F, M_NTAP_BEFORE>(N, a, grid, st); \
            case M_NTAP_AFTER: return launch_dec<F, M_NTAP_AFTER>(N, a, grid, st);   \
            case M_STOCHASTIC:                                                       \
                return N.latent_fmt == 0 ? launch_dec_ws_lf<F, 0>(N, a, num_sms, st)  \
                                         : launch_dec_ws_lf<F, 1>(N, a, num_sms, st); \
            default: break;                                                          \
        }                                                                            \
    }
    STF_DEC_MODES(F_LINEAR)
    STF_DEC_MODES(F_BSPLINE)
    STF_DEC_MODES(F_CATMULL_ROM)
    STF_DEC_MODES(F_MITCHELL)
#undef STF_DEC_MODES
    if (a.mode == M_POSITIVIZED) {
        if (a.filter == F_MITCHELL) return launch_dec<F_MITCHELL, M_POSITIVIZED>(N, a, grid, st);
        if (a.filter == F_CATMULL_ROM) return launch_dec<F_CATMULL_ROM, M_POSITIVIZED>(N, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stf
