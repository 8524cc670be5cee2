// Device-side building blocks of stochastic texture filtering (sm_103a).
//
// Decision arithmetic (positions, weights, CDFs) spells every rounding out with
// __fmul_rn / __fadd_rn / __fmaf_rn, so the compiler can neither contract nor reorder it:
// the selected texel is then a deterministic function of the FP32 inputs (the precision
// of the paper's float listings), reproduced by the CPU oracle with fmaf.  Value
// arithmetic (shading, sums) is free to use FMA.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>

#include "stf_kernels.h"

namespace stf {

// ---------------------------------------------------------------- scalar / packed FP32 pairs
// Value arithmetic is written once for T = float (one sample) and T = F2 (two values, one per
// lane of a 64-bit register pair operated on by the .f32x2 instructions).  Every operation
// below rounds once, to nearest, per lane.  Each packed instruction returns what the scalar
// one returns (checked on B300 over 2^25 random operand pairs per operation, with
// cancellation, subnormals and the byte-decode pattern); a whole kernel built on them agreed
// with its scalar twin only to an ulp on ~0.1% of results, so the packed forms serve value
// arithmetic with a tolerance (the learned form's features and epilogues), not the lookup
// kernels whose specialised and general instantiations must agree bit for bit.
struct F2 { uint64_t v; };
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk2(uint64_t r) {
    float2 f;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
    return f;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ F2 f2(float lo, float hi) { return F2{pk2(lo, hi)}; }
__device__ __forceinline__ F2 f2(float x) { return F2{pk2(x, x)}; }
__device__ __forceinline__ float lo(F2 a) { return upk2(a.v).x; }
__device__ __forceinline__ float hi(F2 a) { return upk2(a.v).y; }
__device__ __forceinline__ float lo(float a) { return a; }

__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ F2 vmul(F2 a, F2 b) { return F2{mul2(a.v, b.v)}; }
__device__ __forceinline__ F2 vadd(F2 a, F2 b) { return F2{add2(a.v, b.v)}; }
// a - b = fma(b, -1, a): one rounding, as __fsub_rn
__device__ __forceinline__ F2 vsub(F2 a, F2 b) { return F2{fma2(b.v, pk2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2{fma2(a.v, b.v, c.v)}; }
// a constant of type T
template <class T> __device__ __forceinline__ T vconst(float x);
template <> __device__ __forceinline__ float vconst<float>(float x) { return x; }
template <> __device__ __forceinline__ F2 vconst<F2>(float x) { return f2(x); }
// per-lane maps
template <class Fn> __device__ __forceinline__ float vmap(float a, Fn fn) { return fn(a); }
template <class Fn> __device__ __forceinline__ F2 vmap(F2 a, Fn fn) { const float2 x = upk2(a.v); return f2(fn(x.x), fn(x.y)); }

// ---------------------------------------------------------------- shared memory and mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

enum { M_NTAP_BEFORE = 0, M_NTAP_AFTER = 1, M_STOCHASTIC = 2, M_POSITIVIZED = 3 };
enum { SH_GGX = 0, SH_LINEAR = 1 };
enum { FLAG_STRATIFIED = 1u, FLAG_LATTICE = 2u, FLAG_REUSE = 4u, FLAG_LOD0 = 8u };
enum { DEV_NAN_INPUT = 1u, DEV_BAD_INDEX = 2u, DEV_TIMEOUT = 4u };
constexpr uint32_t NO_PICK = 0xFFFFFFFFu;

__host__ __device__ constexpr int ntaps(int f) { return f == F_LINEAR ? 2 : 4; }
__host__ __device__ constexpr int tap0(int f) { return f == F_LINEAR ? 0 : -1; }
__host__ __device__ constexpr bool is_signed(int f) { return f == F_CATMULL_ROM || f == F_MITCHELL; }

// Kernel variants.  GENERAL handles every flag and the pick output; PLAIN is a call with no
// flags and no picks; LATTICE a call whose only flag is FLAG_LATTICE, without picks (it
// matters to the stochastic modes only).  The specialised variants compile the unused
// branches out and need fewer registers.
enum { KV_GENERAL = 0, KV_PLAIN = 1, KV_LATTICE = 2 };
__host__ __device__ constexpr uint32_t variant_flags(int v) { return v == KV_LATTICE ? (uint32_t)FLAG_LATTICE : 0u; }
inline int kernel_variant(uint32_t flags, const void* picks) {
    if (picks) return KV_GENERAL;
    if (flags == 0) return KV_PLAIN;
    return flags == (uint32_t)FLAG_LATTICE ? KV_LATTICE : KV_GENERAL;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC 2011).  ctr = (id_lo, id_hi, sample, stream), key = seed.
// The ten round keys depend on the seed only: the host expands them once per launch
// (RoundKeys, passed as a kernel parameter), so a round is two wide multiplies and two
// three-input XORs.
struct RoundKeys { uint32_t k[20]; };

inline RoundKeys expand_key(uint64_t seed) {
    RoundKeys r;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) { r.k[2 * i] = k0; r.k[2 * i + 1] = k1; k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    return r;
}

constexpr uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;   // round multipliers

// rounds FIRST..9 on the state (x0, x1, x2, x3)
template <int FIRST>
__host__ __device__ __forceinline__ void philox_rounds(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                                       const RoundKeys& K) {
#pragma unroll
    for (int r = FIRST; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * x0, p1 = (uint64_t)PHILOX_M1 * x2;
        x0 = (uint32_t)(p1 >> 32) ^ x1 ^ K.k[2 * r];
        x1 = (uint32_t)p1;
        x2 = (uint32_t)(p0 >> 32) ^ x3 ^ K.k[2 * r + 1];
        x3 = (uint32_t)p0;
    }
}

__host__ __device__ __forceinline__ uint4 philox(uint32_t id_lo, uint32_t id_hi, uint32_t sample,
                                                 uint32_t stream, const RoundKeys& K) {
    uint32_t x0 = id_lo, x1 = id_hi, x2 = sample, x3 = stream;
    philox_rounds<0>(x0, x1, x2, x3, K);
    return make_uint4(x0, x1, x2, x3);
}

// The same generator with the counter words that stay fixed across a loop hoisted out of it.
// A round multiplies counter words 0 and 2; where a product depends on fixed words only, it
// and the XORs that use it are computed once, before the loop.  Both return exactly
// philox() of the same counter.
//   PhiloxS: counter (id_lo, id_hi, s, stream), only the sample s varying -- the first two
//            rounds cost two multiplies and three XORs instead of four and four;
//   PhiloxT: counter (id_lo, id_hi, s, t), only the last word t varying -- the first three
//            rounds cost two multiplies and four XORs instead of six and six.
struct PhiloxS {
    uint32_t c0, c1, l1, c2;
    __host__ __device__ __forceinline__ PhiloxS(uint32_t id_lo, uint32_t id_hi, uint32_t stream, const RoundKeys& K) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * id_lo;                 // round 0, word 0
        const uint32_t x2 = (uint32_t)(p0 >> 32) ^ stream ^ K.k[1];      // word 2 after round 0
        c0 = id_hi ^ K.k[0];
        const uint64_t q = (uint64_t)PHILOX_M1 * x2;                     // round 1, word 2
        c1 = (uint32_t)(q >> 32) ^ K.k[2];
        l1 = (uint32_t)q;                                                // word 1 after round 1
        c2 = (uint32_t)p0 ^ K.k[3];
    }
    __host__ __device__ __forceinline__ uint4 operator()(uint32_t s, const RoundKeys& K) const {
        const uint64_t p1 = (uint64_t)PHILOX_M1 * s;                     // round 0, word 2
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c0, y1 = (uint32_t)p1;
        const uint64_t p0 = (uint64_t)PHILOX_M0 * y0;                    // round 1, word 0
        uint32_t x0 = y1 ^ c1, x1 = l1, x2 = (uint32_t)(p0 >> 32) ^ c2, x3 = (uint32_t)p0;
        philox_rounds<2>(x0, x1, x2, x3, K);
        return make_uint4(x0, x1, x2, x3);
    }
};
struct PhiloxT {
    uint32_t d0, d1, d2, e1, d3;
    __host__ __device__ __forceinline__ PhiloxT(uint32_t id_lo, uint32_t id_hi, uint32_t s, const RoundKeys& K) {
        const uint64_t p0 = (uint64_t)PHILOX_M0 * id_lo, p1 = (uint64_t)PHILOX_M1 * s;   // round 0
        const uint32_t g0 = (uint32_t)(p1 >> 32) ^ id_hi ^ K.k[0];
        d0 = (uint32_t)(p0 >> 32) ^ K.k[1];                              // word 2 after round 0: d0 ^ t
        d1 = (uint32_t)p1 ^ K.k[2];
        const uint64_t r0 = (uint64_t)PHILOX_M0 * g0;                    // round 1, word 0
        const uint32_t e2 = (uint32_t)(r0 >> 32) ^ (uint32_t)p0 ^ K.k[3];
        const uint64_t r2 = (uint64_t)PHILOX_M1 * e2;                    // round 2, word 2
        d2 = (uint32_t)(r2 >> 32) ^ K.k[4];
        e1 = (uint32_t)r2;                                               // word 1 after round 2
        d3 = (uint32_t)r0 ^ K.k[5];
    }
    __host__ __device__ __forceinline__ uint4 operator()(uint32_t t, const RoundKeys& K) const {
        const uint64_t p1 = (uint64_t)PHILOX_M1 * (d0 ^ t);              // round 1, word 2
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ d1, y1 = (uint32_t)p1;
        const uint64_t p0 = (uint64_t)PHILOX_M0 * y0;                    // round 2, word 0
        uint32_t x0 = y1 ^ d2, x1 = e1, x2 = (uint32_t)(p0 >> 32) ^ d3, x3 = (uint32_t)p0;
        philox_rounds<3>(x0, x1, x2, x3, K);
        return make_uint4(x0, x1, x2, x3);
    }
};
// top 24 bits scaled by 2^-24: exact in FP32
__device__ __forceinline__ float unif(uint32_t x) { return __uint2float_rn(x >> 8) * 5.9604644775390625e-8f; }

// five 24-bit uniforms per Philox output: four high parts, plus the low bytes of words 0-2
struct U5 { float u[5]; };
__device__ __forceinline__ U5 uniforms5(uint4 w) {
    U5 r;
    r.u[0] = unif(w.x); r.u[1] = unif(w.y); r.u[2] = unif(w.z); r.u[3] = unif(w.w);
    const uint32_t f = ((w.x & 0xFFu) << 16) | ((w.y & 0xFFu) << 8) | (w.z & 0xFFu);
    r.u[4] = __uint2float_rn(f) * 5.9604644775390625e-8f;
    return r;
}
// Randomly shifted lattice across the spp samples of one query (FLAG_LATTICE): sample s
// takes frac(s/spp + phi) with a per-query offset phi, in exact integer arithmetic on the
// 2^bits grid.
__device__ __forceinline__ uint32_t lattice_shift(uint32_t s, uint32_t spp, int bits) {
    return (uint32_t)(((uint64_t)s << bits) / spp);          // floor(s 2^bits / spp), once per sample
}
// (times `scale`, a small integer: the product is the one rounding)
__device__ __forceinline__ float lattice(uint32_t phi, uint32_t shift, int bits, float scale = 1.0f) {
    return __uint2float_rn((phi + shift) & ((1u << bits) - 1u)) * (__int_as_float((127 - bits) << 23) * scale);
}
// integer numerators of uniforms5
struct I5 { uint32_t f[5]; };
__device__ __forceinline__ I5 ints5(uint4 w) {
    I5 r;
    r.f[0] = w.x >> 8; r.f[1] = w.y >> 8; r.f[2] = w.z >> 8; r.f[3] = w.w >> 8;
    r.f[4] = ((w.x & 0xFFu) << 16) | ((w.y & 0xFFu) << 8) | (w.z & 0xFFu);
    return r;
}
// integer numerators of the three 21-bit uniforms of step parity `odd`
__device__ __forceinline__ void ints3_of6(uint4 w, int odd, uint32_t f[3]) {
    if (!odd) { f[0] = w.x >> 11; f[1] = w.y >> 11; f[2] = w.z >> 11; }
    else {
        f[0] = w.w >> 11;
        f[1] = (w.x & 0x7FFu) | ((w.y & 0x3FFu) << 11);
        f[2] = (w.z & 0x7FFu) | ((w.w & 0x3FFu) << 11);
    }
}

// six 21-bit uniforms per Philox output: three for each of two volume march steps, each
// times `scale` (a power of two times a small integer: the product is the one rounding)
__device__ __forceinline__ void uniforms3_of6(uint4 w, int odd, float u[3], float scale = 1.0f) {
    const float k = 4.76837158203125e-7f * scale;
    if (!odd) {
        u[0] = __uint2float_rn(w.x >> 11) * k; u[1] = __uint2float_rn(w.y >> 11) * k;
        u[2] = __uint2float_rn(w.z >> 11) * k;
    } else {
        u[0] = __uint2float_rn(w.w >> 11) * k;
        u[1] = __uint2float_rn((w.x & 0x7FFu) | ((w.y & 0x3FFu) << 11)) * k;
        u[2] = __uint2float_rn((w.z & 0x7FFu) | ((w.w & 0x3FFu) << 11)) * k;
    }
}

// ---------------------------------------------------------------- FP32 decision weights
// Per-axis weights for the taps at distances 1+t, t, 1-t, 2-t (cubic) or 1-t, t (linear).
// The B-spline uses the polynomials of the paper's bicubic listing.  The two signed cubics
// (Keys a = -1/2, Mitchell-Netravali BC(1/3,1/3)) are evaluated in forms factored at their
// roots, so a weight near zero keeps its relative precision: the expanded outer polynomial
// cancels near its double root at |x| = 2, and a positivized negative sample chooses its
// sign class from the ratio of such small weights.  With s = 1 - t:
//   Keys: outer a (x-1)(x-2)^2, inner (x-1)(3x^2/2 - x - 1):
//     w0 = -t s^2/2, w1 = s (1 + t (1 - 3t/2)), w2 = t (1 + s (1 - 3s/2)), w3 = -s t^2/2
//   Mitchell: outer (x-2)^2 (8 - 7x)/18, inner 7x^3/6 - 2x^2 + 8/9 (>= 1/18, in Horner form):
//     w0 = s^2 (1 - 7t)/18, w3 = t^2 (7t - 6)/18
// Multiply-add chains are explicit single-rounded FMAs (__fmaf_rn), nothing else fuses.
// Per-axis weights for T = float (one axis of one sample) or T = F2 (the same axis of two
// samples, or two axes), in the same operation sequence.
template <int F, class T>
__device__ __forceinline__ void axis_weights_t(T t, T w[4]) {
    const T one = vconst<T>(1.0f);
    if constexpr (F == F_LINEAR) {
        w[0] = vsub(one, t);
        w[1] = t;
    } else if constexpr (F == F_BSPLINE) {
        // the listing's polynomials in Horner form with fused multiply-adds:
        //   (1-t)^3, t^2 (3t - 6) + 4, t (t (3 - 3t) + 3) + 1, t^3, each times 1/6
        const T k = vconst<T>(1.0f / 6.0f);
        const T t2 = vmul(t, t);
        const T omt = vsub(one, t);
        w[0] = vmul(k, vmul(vmul(omt, omt), omt));
        w[1] = vmul(k, vfma(t2, vfma(vconst<T>(3.0f), t, vconst<T>(-6.0f)), vconst<T>(4.0f)));
        w[2] = vmul(k, vfma(t, vfma(t, vfma(vconst<T>(-3.0f), t, vconst<T>(3.0f)), vconst<T>(3.0f)), one));
        w[3] = vmul(k, vmul(t2, t));
    } else {
        const T s = vsub(one, t), t2 = vmul(t, t), s2 = vmul(s, s);
        if constexpr (F == F_CATMULL_ROM) {
            w[0] = vmul(vmul(vconst<T>(-0.5f), t), s2);
            w[1] = vmul(s, vfma(t, vfma(vconst<T>(-1.5f), t, one), one));
            w[2] = vmul(t, vfma(s, vfma(vconst<T>(-1.5f), s, one), one));
            w[3] = vmul(vmul(vconst<T>(-0.5f), s), t2);
        } else {   // Mitchell B = C = 1/3; inner piece 7x^3/6 - 2x^2 + 8/9 in Horner form
            const T k18 = vconst<T>(1.0f / 18.0f), c3 = vconst<T>(7.0f / 6.0f), c2 = vconst<T>(-2.0f);
            const T c0 = vconst<T>(8.0f / 9.0f);
            w[0] = vmul(vmul(s2, vfma(vconst<T>(-7.0f), t, one)), k18);
            w[1] = vfma(vmul(vfma(c3, t, c2), t), t, c0);
            w[2] = vfma(vmul(vfma(c3, s, c2), s), s, c0);
            w[3] = vmul(vmul(t2, vfma(vconst<T>(7.0f), t, vconst<T>(-6.0f))), k18);
        }
    }
}
// Weights for a pick, where only their ratios matter: the B-spline's polynomials without the
// common factor 1/6 (the CDF pick divides it out; the estimate's weight is 1 for a positive
// filter), Keys' times 2 (the factor 1/2 of its outer pieces cancels; the estimate's weight
// S_x S_y is scaled back by pick_weight_scale), the others' as axis_weights_t gives them
// (Mitchell's scaled by 18 the same way measured no faster).
template <int F> __host__ __device__ constexpr float pick_weight_scale() {
    return F == F_CATMULL_ROM ? 0.25f : 1.0f;
}
template <int F, class T>
__device__ __forceinline__ void axis_pick_weights_t(T t, T w[4]) {
    if constexpr (F == F_CATMULL_ROM && sizeof(T) == sizeof(float)) {
        // 2 x: -t s^2, s (2 + t (2 - 3t)), t (2 + s (2 - 3s)), -s t^2
        const float s = __fsub_rn(1.0f, t), t2 = __fmul_rn(t, t), s2 = __fmul_rn(s, s);
        w[0] = __fmul_rn(-t, s2);
        w[1] = __fmul_rn(s, __fmaf_rn(t, __fmaf_rn(-3.0f, t, 2.0f), 2.0f));
        w[2] = __fmul_rn(t, __fmaf_rn(s, __fmaf_rn(-3.0f, s, 2.0f), 2.0f));
        w[3] = __fmul_rn(-s, t2);
    } else if constexpr (F == F_BSPLINE) {
        const T one = vconst<T>(1.0f);
        const T t2 = vmul(t, t);
        const T omt = vsub(one, t);
        w[0] = vmul(vmul(omt, omt), omt);
        w[1] = vfma(t2, vfma(vconst<T>(3.0f), t, vconst<T>(-6.0f)), vconst<T>(4.0f));
        w[2] = vfma(t, vfma(t, vfma(vconst<T>(-3.0f), t, vconst<T>(3.0f)), vconst<T>(3.0f)), one);
        w[3] = vmul(t2, t);
    } else {
        axis_weights_t<F, T>(t, w);
    }
}
template <int F> __device__ __forceinline__ void axis_weights(float t, float w[4]) { axis_weights_t<F, float>(t, w); }
template <int F> __device__ __forceinline__ void axis_pick_weights(float t, float w[4]) { axis_pick_weights_t<F, float>(t, w); }

// CDF inversion over one axis: first k with xi*S < prefix_k, S = sum of |w| over the
// taps of sign class CLS (0: all, +1: w > 0, -1: w < 0).  Returns the tap index.
template <int N>
__device__ __forceinline__ int cdf_pick(const float w[4], float xi, int cls, float* total) {
    float c[N];
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const bool in = cls == 0 || (cls > 0 ? w[k] > 0.0f : w[k] < 0.0f);
        acc = __fadd_rn(acc, in ? fabsf(w[k]) : 0.0f);
        c[k] = acc;
    }
    if (total) *total = acc;
    const float target = __fmul_rn(xi, acc);
    int k = N - 1;
#pragma unroll
    for (int j = N - 2; j >= 0; --j) k = (target < c[j]) ? j : k;
    return k;
}

// cdf_pick over all taps (class 0) that also reports whether the picked weight is negative,
// selected in the same compare chain as the index.  INNER_POS: the two inner weights of a
// 4-tap filter are known to be positive (Keys and Mitchell-Netravali: at least 1/2 (1-t) and
// 1/18 on [0, 1)), so only the outer taps can carry a minus sign.
template <int N, bool INNER_POS = false>
__device__ __forceinline__ int cdf_pick_sign(const float w[4], float xi, float* total, bool* neg) {
    float c[N];
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) { acc = __fadd_rn(acc, fabsf(w[k])); c[k] = acc; }
    *total = acc;
    const float target = __fmul_rn(xi, acc);
    if constexpr (INNER_POS && N == 4) {
        const bool h0 = target < c[0], h1 = target < c[1], h2 = target < c[2];
        *neg = h0 ? (w[0] < 0.0f) : (!h2 && w[3] < 0.0f);
        return h0 ? 0 : (h1 ? 1 : (h2 ? 2 : 3));
    }
    int k = N - 1;
    bool ng = w[N - 1] < 0.0f;
#pragma unroll
    for (int j = N - 2; j >= 0; --j) {
        const bool hit = target < c[j];
        k = hit ? j : k;
        ng = hit ? (w[j] < 0.0f) : ng;
    }
    *neg = ng;
    return k;
}

// The tap a positive filter picks on one axis for the uniform xi, the first k with xi < C_k,
// from the CDF's closed form (the weights sum to one): tent C_0 = 1 - t; cubic B-spline
// 6 C_0 = (1-t)^3, 6 C_1 = 5 - 3t - 3t^2 + 2t^3, 6 C_2 = 6 - t^3 (prefix sums of the
// polynomials of the bicubic listing).  In FP32 each boundary lies within ~1e-7 of its exact
// value, inside the 1e-6 band around a boundary where a pick may differ from the exact one.
// pick_positive_scaled takes xs = pick_scale<F>() * xi; a caller that forms xi = n * 2^-b
// from an integer n < 2^b can fold the scale into that multiply (n * (6 * 2^-b) rounds to
// the same value as (n * 2^-b) * 6).
template <int F> __host__ __device__ constexpr float pick_scale() { return F == F_BSPLINE ? 6.0f : 1.0f; }
template <int F>
__device__ __forceinline__ int pick_positive_scaled(float t, float xs) {
    static_assert(F == F_LINEAR || F == F_BSPLINE, "positive filters only");
    if constexpr (F == F_LINEAR) {
        return xs < __fsub_rn(1.0f, t) ? 0 : 1;
    } else {
        const float s = __fsub_rn(1.0f, t);
        const float c0 = __fmul_rn(__fmul_rn(s, s), s);
        const float c1 = __fmaf_rn(__fmaf_rn(__fmaf_rn(2.0f, t, -3.0f), t, -3.0f), t, 5.0f);
        const float c2 = __fmaf_rn(-__fmul_rn(t, t), t, 6.0f);
        // binary search: the middle boundary first, then the one on its side
        const bool hi = xs >= c1;
        return (hi ? 2 : 0) + ((xs >= (hi ? c2 : c0)) ? 1 : 0);
    }
}
template <int F>
__device__ __forceinline__ int pick_positive(float t, float xi) {
    return pick_positive_scaled<F>(t, F == F_BSPLINE ? __fmul_rn(xi, 6.0f) : xi);
}
// The same for two axes at once (x, y), the B-spline boundaries in packed FP32 pairs (one
// rounding per lane: the values equal pick_positive's); the _scaled form takes pre-scaled
// uniforms as pick_positive_scaled does
template <int F>
__device__ __forceinline__ void pick_positive2_scaled(F2 t, float xs_x, float xs_y, int* kx, int* ky) {
    if constexpr (F == F_LINEAR) {
        const float2 tt = upk2(t.v);
        *kx = pick_positive_scaled<F>(tt.x, xs_x);
        *ky = pick_positive_scaled<F>(tt.y, xs_y);
    } else {
        const F2 s = vsub(vconst<F2>(1.0f), t);
        const float2 c0 = upk2(vmul(vmul(s, s), s).v);
        const float2 c1 = upk2(vfma(vfma(vfma(vconst<F2>(2.0f), t, vconst<F2>(-3.0f)), t, vconst<F2>(-3.0f)), t,
                                    vconst<F2>(5.0f)).v);
        const float2 c2 = upk2(vfma(vmul(vmul(t, t), vconst<F2>(-1.0f)), t, vconst<F2>(6.0f)).v);
        const bool hx = xs_x >= c1.x, hy = xs_y >= c1.y;
        *kx = (hx ? 2 : 0) + ((xs_x >= (hx ? c2.x : c0.x)) ? 1 : 0);
        *ky = (hy ? 2 : 0) + ((xs_y >= (hy ? c2.y : c0.y)) ? 1 : 0);
    }
}
template <int F>
__device__ __forceinline__ void pick_positive2(float tx, float ty, float xi_x, float xi_y, int* kx, int* ky) {
    if constexpr (F == F_LINEAR) {
        *kx = pick_positive<F>(tx, xi_x);
        *ky = pick_positive<F>(ty, xi_y);
    } else {
        const float2 xs = upk2(vmul(f2(xi_x, xi_y), vconst<F2>(6.0f)).v);
        pick_positive2_scaled<F>(f2(tx, ty), xs.x, xs.y, kx, ky);
    }
}

// Positivization's per-axis sums and picks for a 4-tap filter whose inner taps are positive
// (Keys, Mitchell-Netravali): the positive class is {tap 0 if w0 > 0, 1, 2, tap 3 if w3 > 0},
// the negative class {tap 0 if w0 < 0, tap 3 if w3 < 0}.  The prefix sums are cdf_pick's for
// classes +1 and -1, in the same order (a skipped tap adds an exact zero), so the sums and the
// picks equal cdf_pick's.
struct SignedAxis4 { float c0, c1, c2, P, n0, N; };
__device__ __forceinline__ SignedAxis4 signed_axis4(const float w[4]) {
    SignedAxis4 a;
    a.c0 = w[0] > 0.0f ? w[0] : 0.0f;
    a.c1 = __fadd_rn(a.c0, w[1]);
    a.c2 = __fadd_rn(a.c1, w[2]);
    a.P = __fadd_rn(a.c2, w[3] > 0.0f ? w[3] : 0.0f);
    a.n0 = w[0] < 0.0f ? -w[0] : 0.0f;
    a.N = __fadd_rn(a.n0, w[3] < 0.0f ? -w[3] : 0.0f);
    return a;
}
// the tap of class cls (+1 or -1) for the uniform xi
__device__ __forceinline__ int signed_pick4(const SignedAxis4& a, float xi, int cls) {
    const float tp = __fmul_rn(xi, a.P), tn = __fmul_rn(xi, a.N);
    const int kp = tp < a.c0 ? 0 : (tp < a.c1 ? 1 : (tp < a.c2 ? 2 : 3));
    const int kn = tn < a.n0 ? 0 : 3;
    return cls > 0 ? kp : kn;
}

// Sample reuse: the same pick, and the uniform remapped into the chosen interval,
// u' = (xi S - C_{k-1}) / (C_k - C_{k-1}) (Eq. uniform-sample-reuse on a sampling array).
template <int N>
__device__ __forceinline__ int cdf_pick_reuse(const float w[4], float xi, float* remapped) {
    float c[N];
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) { acc = __fadd_rn(acc, fabsf(w[k])); c[k] = acc; }
    const float target = __fmul_rn(xi, acc);
    int k = N - 1;
    float lo = c[N - 2], hi = c[N - 1];
#pragma unroll
    for (int j = N - 2; j >= 0; --j) {
        if (target < c[j]) { k = j; hi = c[j]; lo = j > 0 ? c[j - 1] : 0.0f; }
    }
    *remapped = __fdiv_rn(__fsub_rn(target, lo), __fsub_rn(hi, lo));
    return k;
}
__device__ __forceinline__ int level_reuse(float xi, float f, float* remapped) {
    if (xi < f) { *remapped = __fdiv_rn(xi, f); return 1; }
    *remapped = __fdiv_rn(__fsub_rn(xi, f), __fsub_rn(1.0f, f));
    return 0;
}

// raster position on one axis: p = x*res - 1/2, i0 = floor(p), t = p - i0 (FP32)
struct AxisPos { int i0; float t; };
__device__ __forceinline__ AxisPos axis_pos(float x, float res) {
    float p = __fmaf_rn(x, res, -0.5f);
    float fl = floorf(p);
    return {(int)fl, __fsub_rn(p, fl)};
}

__device__ __forceinline__ int wrap_index(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;          // common case: no wrap
    int r = i % n;
    return r < 0 ? r + n : r;
}
__device__ __forceinline__ int clamp_index(int i, int n) { return min(max(i, 0), n - 1); }

// ---------------------------------------------------------------- shading (FP32)
struct Material { float3 rho; float rough; float3 n; };

// Fixed light / view directions (unit in exact arithmetic), the derived half vector (FP32-rounded
// normalize(l+v)) and F(v.h) / (2 pi), as the host evaluates them; the shading kernels take
// the same directions as compile-time constants (GgxK).
struct ShadeConst {
    float3 l, v, h;
    float Fk;   // F / (2 pi): Schlick Fresnel at v.h (F0 = 0.04) with the constant factors of D G F / 4
};

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Approximate reciprocal and reciprocal square root: one MUFU instruction each, flushing
// subnormals.  Used only in shading and decoding, whose results carry a tolerance, never in
// a decision.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The light, view and half vectors as compile-time FP32 constants: l = (0.48, 0.36, 0.80),
// v = (-0.28, 0, 0.96) (unit in exact arithmetic) and h = normalize(l + v), stored scaled by
// kappa = Fk^(-1/4), where Fk = F(v.h) / (2 pi) is the Schlick Fresnel at v.h (F0 = 0.04) with
// the constant factors of D G F / 4.  h enters only n.h and |n x h|^2, so the scaled vector
// gives q' = kappa^2 q for the denominator q = a2 (n.h)^2 + |n x h|^2 of D, and a2 / q'^2 is
// Fk a2 / q^2: the constant factor costs no multiply.  Each constant is evaluated in double
// and rounded once to FP32.
struct GgxK {
    static constexpr float lx = 0.48f, ly = 0.36f, lz = 0.80f;
    static constexpr float vx = -0.28f, vz = 0.96f;
    static constexpr float hx = 0x1.91191ap-2f, hy = 0x1.68fcfep-1f, hz = 0x1.b93536p+1f;   // kappa h
};

// A decoded material as scalars (T = float) or as two samples' materials (T = F2).
template <class T> struct MatT { T rx, ry, rz, rough, nx, ny, nz; };

// x where both n.l > 0 and n.v > 0, else 0, per lane
__device__ __forceinline__ float above(float x, float nl, float nv) { return (nl > 0.0f && nv > 0.0f) ? x : 0.0f; }
__device__ __forceinline__ F2 above(F2 x, F2 nl, F2 nv) {
    const float2 X = upk2(x.v), L = upk2(nl.v), V = upk2(nv.v);
    return f2(above(X.x, L.x, V.x), above(X.y, L.y, V.y));
}

// f_hat = [rho/pi + D G2 F / (4 nl nv)] nl  (GGX, height-correlated Smith, Schlick), zero
// where nl <= 0 or nv <= 0.  Every operation is one explicit rounding, so the T = float and
// T = F2 forms agree bit for bit.  CLAMP: clamp the roughness to [0.05, 1] first; a caller
// whose decoded roughness lies in that range already (0.05 + 0.95 x with x in [0, 1]) skips it.
template <class T, bool CLAMP = true>
__device__ __forceinline__ void shade_ggx_t(const MatT<T>& m, T& r, T& g, T& b) {
    using K = GgxK;
    const T nl = vfma(m.nz, vconst<T>(K::lz), vfma(m.ny, vconst<T>(K::ly), vmul(m.nx, vconst<T>(K::lx))));
    const T nv = vfma(m.nz, vconst<T>(K::vz), vmul(m.nx, vconst<T>(K::vx)));
    T a = m.rough;
    if constexpr (CLAMP) a = vmap(m.rough, [](float x) { return fminf(fmaxf(x, 0.05f), 1.0f); });
    const T a2 = vmul(a, a);
    // |n x h|^2 instead of 1 - (n.h)^2: D = a2 / (pi q^2) is relative to q >= a2 (n.h)^2,
    // so the cancellation of 1 - (n.h)^2 near n = h would show in D
    const T cx = vfma(m.ny, vconst<T>(K::hz), vmul(m.nz, vconst<T>(-K::hy)));
    const T cy = vfma(m.nz, vconst<T>(K::hx), vmul(m.nx, vconst<T>(-K::hz)));
    const T cz = vfma(m.nx, vconst<T>(K::hy), vmul(m.ny, vconst<T>(-K::hx)));
    const T nh = vfma(m.nz, vconst<T>(K::hz), vfma(m.ny, vconst<T>(K::hy), vmul(m.nx, vconst<T>(K::hx))));
    const T q = vfma(vmul(a2, nh), nh, vfma(cz, cz, vfma(cy, cy, vmul(cx, cx))));
    auto rcp = [](float x) { return rcp_approx(x); };
    auto rsq = [](float x) { return rsqrt_approx(x); };
    const T rq = vmap(q, rcp), rnl = vmap(nl, rcp), rnv = vmap(nv, rcp);
    // D = a2 / (pi q^2).  Lambda = (sqrt(1 + a2 tan^2) - 1) / 2 with tan^2 = 1/(n.w)^2 - 1
    // (|n| = 1), so G2 = 1 / (1 + Ll + Lv) = 2 / (sqrt(sl) + sqrt(sv)): a sum of two positive
    // roots, one reciprocal, no cancellation.  The constants 1/pi, 2, 1/4 and F ride in kappa.
    const T one = vconst<T>(1.0f), mone = vconst<T>(-1.0f);
    const T sl = vfma(a2, vfma(rnl, rnl, mone), one);
    const T sv = vfma(a2, vfma(rnv, rnv, mone), one);
    const T rg = vmap(vfma(sl, vmap(sl, rsq), vmul(sv, vmap(sv, rsq))), rcp);
    // the lobe exists only above both horizons
    const T spec = above(vmul(vmul(vmul(vmul(a2, rq), rq), rg), rnv), nl, nv);
    const T kd = above(vmul(nl, vconst<T>(0.318309886183790672f)), nl, nv);
    r = vfma(m.rx, kd, spec);
    g = vfma(m.ry, kd, spec);
    b = vfma(m.rz, kd, spec);
}

__device__ __forceinline__ MatT<float> mat_t(const Material& m) {
    return {m.rho.x, m.rho.y, m.rho.z, m.rough, m.n.x, m.n.y, m.n.z};
}
template <bool CLAMP = true>
__device__ __forceinline__ float3 shade_ggx(const Material& m, const ShadeConst&) {
    float r, g, b;
    shade_ggx_t<float, CLAMP>(mat_t(m), r, g, b);
    return make_float3(r, g, b);
}

// CLAMP = false: the caller's roughness is in [0.05, 1] already (a decoded texel of an RGBA8,
// DCT or learned texture); the clamp would return it unchanged.
template <bool CLAMP = true>
__device__ __forceinline__ float3 shade(int sh, const Material& m, const ShadeConst& C) {
    if (sh == SH_LINEAR) return m.rho;
    return shade_ggx<CLAMP>(m, C);
}

// ---------------------------------------------------------------- texel decode
// RGBA8 material texel packed with its RG8 normal into 8 bytes (uint2):
//   x = albedo R | G<<8 | B<<16 | roughness byte<<24, y = normal X | Y<<8, has_normal flag
// Byte j of w as the float 2^23 + byte (one byte permute into the bits of 2^23).
__device__ __forceinline__ float byte_plus_2p23(uint32_t w, uint32_t j) {
    return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7540u | j));
}
// byte j of w times k, rounded once: the fused (2^23 + b) k - 2^23 k is exactly b k
// (2^23 k is exact), so this equals the FP32 product (float)b * k
__device__ __forceinline__ float byte_times(uint32_t w, uint32_t j, float k) {
    return __fmaf_rn(byte_plus_2p23(w, j), k, -8388608.0f * k);
}
// The packed material texel (RGBA8 albedo + roughness in x, RG8 normal in y) of one sample
// (T = float, t1 ignored) or of two (T = F2: t0 in the low lane, t1 in the high lane).
//   albedo = byte/255, roughness = 0.05 + 0.95 byte/255;
//   normal = (X, Y, sqrt R) / 255 with X = 2r - 255, Y = 2g - 255, R = 255^2 - X^2 - Y^2,
//   exactly unit length when R > 0; otherwise z = 0 and (X, Y) is normalised.
template <class T>
__device__ __forceinline__ T bytes_of(uint32_t w0, uint32_t w1, uint32_t j);
template <> __device__ __forceinline__ float bytes_of<float>(uint32_t w0, uint32_t, uint32_t j) { return byte_plus_2p23(w0, j); }
template <> __device__ __forceinline__ F2 bytes_of<F2>(uint32_t w0, uint32_t w1, uint32_t j) {
    return f2(byte_plus_2p23(w0, j), byte_plus_2p23(w1, j));
}
template <class T>
__device__ __forceinline__ MatT<T> decode_rgba8n_t(uint2 t0, uint2 t1 = make_uint2(0u, 0u)) {
    const float k = 1.0f / 255.0f;
    MatT<T> m;
    // byte times k, rounded once: the fused (2^23 + b) k - 2^23 k is exactly b k
    const T kk = vconst<T>(k), off = vconst<T>(-8388608.0f * k);
    m.rx = vfma(bytes_of<T>(t0.x, t1.x, 0), kk, off);
    m.ry = vfma(bytes_of<T>(t0.x, t1.x, 1), kk, off);
    m.rz = vfma(bytes_of<T>(t0.x, t1.x, 2), kk, off);
    m.rough = vfma(vconst<T>(0.95f), vfma(bytes_of<T>(t0.x, t1.x, 3), kk, off), vconst<T>(0.05f));
    // 2b - 255 exactly: (2^23 + b) - (2^23 + 127) = b - 127, then 2 (b - 127) - 1
    const T X = vfma(vconst<T>(2.0f), vsub(bytes_of<T>(t0.y, t1.y, 0), vconst<T>(8388735.0f)), vconst<T>(-1.0f));
    const T Y = vfma(vconst<T>(2.0f), vsub(bytes_of<T>(t0.y, t1.y, 1), vconst<T>(8388735.0f)), vconst<T>(-1.0f));
    const T XY = vfma(Y, Y, vmul(X, X));                              // exact integer
    const T R = vsub(vconst<T>(65025.0f), XY);                        // exact integer radicand
    // R > 0: scale 1/255 and z = sqrt(R)/255; otherwise scale 1/|(X, Y)| and z = 0
    auto sc = [](float r, float xy) { return r > 0.0f ? 1.0f / 255.0f : rsqrt_approx(xy); };
    auto zz = [](float r) { return r > 0.0f ? __fmul_rn(__fmul_rn(r, rsqrt_approx(r)), 1.0f / 255.0f) : 0.0f; };
    T scale, z;
    if constexpr (sizeof(T) == sizeof(float)) {
        scale = sc(lo(R), lo(XY));
        z = zz(lo(R));
    } else {
        const float2 r = upk2(R.v), xy = upk2(XY.v);
        scale = f2(sc(r.x, xy.x), sc(r.y, xy.y));
        z = f2(zz(r.x), zz(r.y));
    }
    m.nx = vmul(X, scale);
    m.ny = vmul(Y, scale);
    m.nz = z;
    return m;
}
__device__ __forceinline__ Material mat_of(const MatT<float>& m) {
    Material r;
    r.rho = make_float3(m.rx, m.ry, m.rz);
    r.rough = m.rough;
    r.n = make_float3(m.nx, m.ny, m.nz);
    return r;
}
__device__ __forceinline__ Material decode_rgba8(uint2 t, bool has_normal) {
    if (has_normal) return mat_of(decode_rgba8n_t<float>(t));
    Material m;
    const float k = 1.0f / 255.0f;
    m.rho = make_float3(byte_times(t.x, 0, k), byte_times(t.x, 1, k), byte_times(t.x, 2, k));
    m.rough = __fmaf_rn(0.95f, byte_times(t.x, 3, k), 0.05f);
    m.n = make_float3(0.f, 0.f, 1.f);
    return m;
}
// Decoded channels (albedo RGB, roughness, normal X and Y, each in [0,1] up to decoding
// error) -> material: clamped albedo, roughness 0.05 + 0.95 r, normal (2x-1, 2y-1, z)
// normalised.  Used by the learned and the DCT-compressed textures.
__device__ __forceinline__ Material material_from_channels(const float y[8]) {
    Material m;
    m.rho = make_float3(__saturatef(y[0]), __saturatef(y[1]), __saturatef(y[2]));
    m.rough = fmaf(0.95f, __saturatef(y[3]), 0.05f);
    const float x = fmaf(2.0f, __saturatef(y[4]), -1.0f), yy = fmaf(2.0f, __saturatef(y[5]), -1.0f);
    const float z2 = 1.0f - x * x - yy * yy;
    // z2 > 0: (x, y, sqrt z2) is a unit vector already; otherwise z = 0 and (x, y), which is
    // then at least unit length, is normalised
    if (z2 > 0.0f) {
        m.n = make_float3(x, yy, z2 * rsqrt_approx(z2));
    } else {
        const float inv = rsqrt_approx(x * x + yy * yy);
        m.n = make_float3(x * inv, yy * inv, 0.0f);
    }
    return m;
}

__device__ __forceinline__ Material decode_rgba32f(float4 t) {
    Material m;
    m.rho = make_float3(t.x, t.y, t.z);
    m.rough = t.w;
    m.n = make_float3(0.f, 0.f, 1.f);
    return m;
}

// ---------------------------------------------------------------- DCT-compressed texels
// 8 x 8 blocks of six channel words (supplement "Texture compression"): per channel the
// six lowest frequencies (u + v <= 2) of the orthonormal 2-D DCT-II, DC in bits 0-6
// (q * 8/127), AC terms (1,0), (0,1), (2,0), (1,1), (0,2) in 5-bit fields ((q - 15) * 2/15);
// blocks are 32 bytes (24 used), row-major per level.
struct DctRaw {
    uint4 a;     // channel words 0-3 (albedo RGB, roughness)
    uint2 b;     // channel words 4-5 (normal X, Y)
    int lx, ly;  // texel position inside the block
};
__device__ __forceinline__ DctRaw load_dct(const unsigned char* level, int w, int ix, int iy) {
    const uint32_t w8 = ((uint32_t)w + 7u) >> 3;
    const uint32_t blk = ((uint32_t)iy >> 3) * w8 + ((uint32_t)ix >> 3);
    const uint4* p = reinterpret_cast<const uint4*>(level) + (size_t)blk * 2;
    DctRaw r;
    r.a = __ldg(p);
    r.b = __ldg(reinterpret_cast<const uint2*>(p + 1));
    r.lx = ix & 7;
    r.ly = iy & 7;
    return r;
}
// one channel: q0/127 + (2/15) [a1 a0 (q1 cx1 + q2 cy1 + q3 cx2 + q5 cy2) + a1 a1 q4 cx1 cy1],
// a0 = 1/(2 sqrt 2), a1 = 1/2 (the orthonormal scale factors)
__device__ __forceinline__ float dct_channel(uint32_t w, float cx1, float cx2, float cy1, float cy2) {
    const float q1 = (float)((int)((w >> 7) & 31u) - 15), q2 = (float)((int)((w >> 12) & 31u) - 15);
    const float q3 = (float)((int)((w >> 17) & 31u) - 15), q4 = (float)((int)((w >> 22) & 31u) - 15);
    const float q5 = (float)((int)((w >> 27) & 31u) - 15);
    const float s10 = 0.17677669529663688f * (2.0f / 15.0f), s11 = 0.25f * (2.0f / 15.0f);
    float f = fmaf(q1, cx1, q2 * cy1);
    f = fmaf(q3, cx2, f);
    f = fmaf(q5, cy2, f);
    return fmaf(f, s10, fmaf(q4 * s11, cx1 * cy1, (float)(w & 127u) * (1.0f / 127.0f)));
}
__device__ __forceinline__ Material decode_dct(const DctRaw& r) {
    // cos((2x+1) pi / 16) per axis, and cos(2 theta) = 2 cos^2 theta - 1
    const float cx1 = cospif((float)(2 * r.lx + 1) * 0.0625f), cy1 = cospif((float)(2 * r.ly + 1) * 0.0625f);
    const float cx2 = fmaf(2.0f * cx1, cx1, -1.0f), cy2 = fmaf(2.0f * cy1, cy1, -1.0f);
    float y[8];
    y[0] = dct_channel(r.a.x, cx1, cx2, cy1, cy2);
    y[1] = dct_channel(r.a.y, cx1, cx2, cy1, cy2);
    y[2] = dct_channel(r.a.z, cx1, cx2, cy1, cy2);
    y[3] = dct_channel(r.a.w, cx1, cx2, cy1, cy2);
    y[4] = dct_channel(r.b.x, cx1, cx2, cy1, cy2);
    y[5] = dct_channel(r.b.y, cx1, cx2, cy1, cy2);
    y[6] = y[7] = 0.0f;
    return material_from_channels(y);
}

}  // namespace stf
