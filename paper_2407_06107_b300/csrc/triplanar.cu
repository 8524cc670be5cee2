// Triplanar filter + shade kernels (sm_103a).
//
// Triplanar mapping (Sec. 5 "Triplanar mapping"; Sec. 4.4 material graphs) looks textures up
// three times, at the surface point projected along x, y and z, and blends the three results
// with weights from the surface normal.  The blend is a weighted sum, so Eq. stochastic-sum
// applies to it as it does to the filter taps: BLEND_STOCHASTIC draws one plane per sample
// with probability b_i and evaluates that plane's lookup alone (weight b_i / p_i = 1).  With
// the 1-tap filter a sample then reads one texel instead of three (or 3 x 8 for trilinear
// N-tap).
//
// Blend weights b_i = |n_i|^4 / sum_j |n_j|^4, FP32 in a fixed order (they decide the plane
// pick); a normal whose weights all vanish maps to the z plane.  Plane i's lookup is the 2-D
// lookup of the filter kernels at (u, v) = scale * (the two other coordinates of P), with the
// derivatives of P projected the same way: jitter in that footprint, stochastic level,
// separable picks.  Every plane of a sample uses the same uniforms (stream 0, and stream 1 for
// positivization); the plane pick uses the fifth uniform of stream 1.
#include "stf_kernels.h"
#include "stf_device.cuh"
#include "stf_lookup.cuh"

namespace stf {

struct TriTex { FetchCtx t[3]; };

// unnormalised blend weights w_i = (n_i^2)^2 and their sum (w[3] = 0 pads the pick array)
__device__ __forceinline__ float tri_weights(float nx, float ny, float nz, float w[4]) {
    const float ax = __fmul_rn(nx, nx), ay = __fmul_rn(ny, ny), az = __fmul_rn(nz, nz);
    w[0] = __fmul_rn(ax, ax);
    w[1] = __fmul_rn(ay, ay);
    w[2] = __fmul_rn(az, az);
    w[3] = 0.0f;
    return __fadd_rn(__fadd_rn(w[0], w[1]), w[2]);
}

// plane i's 2-D query and its level: plane 0 reads (y, z), plane 1 (x, z), plane 2 (x, y)
struct PlaneQ { float u, v, dudx, dvdx, dudy, dvdy; int l0; float fr; };

__device__ __forceinline__ PlaneQ plane_query(int i, float3 P, float3 DX, float3 DY, bool has_d, float s,
                                              const FetchCtx& T, uint32_t flags) {
    PlaneQ p;
    p.u = __fmul_rn(i == 0 ? P.y : P.x, s);
    p.v = __fmul_rn(i == 2 ? P.y : P.z, s);
    float lam = 0.0f;
    p.dudx = p.dvdx = p.dudy = p.dvdy = 0.0f;
    if (has_d) {
        p.dudx = __fmul_rn(i == 0 ? DX.y : DX.x, s);
        p.dvdx = __fmul_rn(i == 2 ? DX.y : DX.z, s);
        p.dudy = __fmul_rn(i == 0 ? DY.y : DY.x, s);
        p.dvdy = __fmul_rn(i == 2 ? DY.y : DY.z, s);
        if (T.levels > 1) lam = lod_aniso(p.dudx, p.dvdx, p.dudy, p.dvdy, (float)T.w[0], (float)T.h[0], T.levels);
    }
    if (flags & FLAG_LOD0) lam = 0.0f;
    p.l0 = (int)floorf(lam);
    p.fr = __fsub_rn(lam, (float)p.l0);
    return p;
}

// One sample of one plane, weighted by `scale`.  The N-tap filter-before mode adds the
// plane's filtered material into fm (shaded once after all planes) and returns zero.
// pk (nullable) receives the plane's two pick slots.
template <int FILTER, int MODE, int TF>
__device__ __forceinline__ float3 plane_sample(const FetchCtx& T, const PlaneQ& p, uint32_t s, int kside,
                                               uint32_t flags, bool has_d, const U5& A, const U5& B, float scale,
                                               int shade_mode, const ShadeConst& SC, Material& fm, uint32_t* pk) {
    float x = p.u, y = p.v;
    if (has_d) jitter(s, kside, flags, A, p.dudx, p.dvdx, p.dudy, p.dvdy, &x, &y);
    if constexpr (MODE == M_STOCHASTIC) {
        const Pick1 k = pick_1tap<FILTER, TF>(T, x, y, p.l0, p.fr, A, false);
        const float3 f = shade<clamp_rough<TF>()>(shade_mode, fetch_t<TF>(T, k.lvl, k.ix, k.iy), SC);
        if (pk) { pk[0] = pack_pick(k.lvl, k.ix, k.iy); pk[1] = NO_PICK; }
        const float w = scale * k.wt;
        return make_float3(w * f.x, w * f.y, w * f.z);
    } else if constexpr (MODE == M_POSITIVIZED) {
        uint32_t k0, k1;
        const float3 e = positivized_sample<FILTER, TF>(T, x, y, p.l0, p.fr, A, B, shade_mode, SC, &k0, &k1);
        if (pk) { pk[0] = k0; pk[1] = k1; }
        return make_float3(scale * e.x, scale * e.y, scale * e.z);
    } else {
        float3 fsum = make_float3(0.f, 0.f, 0.f);
        ntap_accumulate<FILTER, MODE, TF>(T, x, y, p.l0, p.fr, scale, shade_mode, SC, fm, fsum);
        return fsum;
    }
}

// Resident 256-thread blocks per SM: 4 (<= 64 registers); 3 for positivization and the DCT
// N-tap sums, which spill at 64.
template <int MODE, int V, int TF>
constexpr int tri_min_blocks() {
    return (MODE == M_POSITIVIZED || (TF == TF_DCT && MODE != M_STOCHASTIC)) ? 3
           : (MODE == M_STOCHASTIC && V != KV_GENERAL) ? 5 : 4;
}

template <int FILTER, int MODE, int BLEND, int V, int TF>
__global__ void __launch_bounds__(256, tri_min_blocks<MODE, V, TF>())
k_triplanar(TriplanarArgs a, const __grid_constant__ TriTex TT, ShadeConst SC, RoundKeys K) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const uint64_t q = a.order ? (uint64_t)__ldg(a.order + i) : i;
    const uint32_t flags = V == KV_GENERAL ? a.flags : variant_flags(V);
    uint32_t* const picks = V == KV_GENERAL ? a.picks : nullptr;
    const bool has_d = a.has_derivs != 0;
    // the point and result streams are touched once: loaded and stored evict-first
    const float3 P = make_float3(__ldcs(a.px + q), __ldcs(a.py + q), __ldcs(a.pz + q));
    const float3 N = make_float3(__ldcs(a.nx + q), __ldcs(a.ny + q), __ldcs(a.nz + q));
    float3 DX = make_float3(0.f, 0.f, 0.f), DY = DX;
    if (has_d) {
        DX = make_float3(__ldcs(a.dxx + q), __ldcs(a.dxy + q), __ldcs(a.dxz + q));
        DY = make_float3(__ldcs(a.dyx + q), __ldcs(a.dyy + q), __ldcs(a.dyz + q));
    }
    if (isnan(P.x) || isnan(P.y) || isnan(P.z) || isnan(N.x) || isnan(N.y) || isnan(N.z) || isnan(DX.x) ||
        isnan(DX.y) || isnan(DX.z) || isnan(DY.x) || isnan(DY.y) || isnan(DY.z))
        atomicOr(a.status, DEV_NAN_INPUT);
    float w[4];
    const float W = tri_weights(N.x, N.y, N.z, w);
    const uint64_t id = a.id_base + q;
    const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
    const bool lat = (MODE == M_STOCHASTIC || MODE == M_POSITIVIZED) && (flags & FLAG_LATTICE);
    constexpr bool NEED_B = BLEND == BLEND_STOCHASTIC || MODE == M_POSITIVIZED;
    I5 LA{}, LB{};
    if (lat) {   // per-query lattice offsets of the pick uniforms (and of the plane pick)
        LA = ints5(philox(id_lo, id_hi, 0xFFFFFFFFu, 0u, K));
        if (NEED_B) LB = ints5(philox(id_lo, id_hi, 0xFFFFFFFFu, 1u, K));
    }
    float3 acc = make_float3(0.f, 0.f, 0.f);
    for (uint32_t s = 0; s < a.spp; ++s) {
        // stream 0: (jitter x, jitter y, level, pick x, pick y); stream 1: (positive class,
        // negative pick x, negative pick y, negative class, plane)
        U5 A = uniforms5(philox(id_lo, id_hi, s, 0u, K));
        U5 B{};
        const uint32_t lshift = lat ? lattice_shift(s, a.spp, 24) : 0u;
        if (lat) {
#pragma unroll
            for (int k = 2; k < 5; ++k) A.u[k] = lattice(LA.f[k], lshift, 24);
        }
        if (NEED_B) {
            B = uniforms5(philox(id_lo, id_hi, s, 1u, K));
            if (lat) {
#pragma unroll
                for (int k = 0; k < 5; ++k) B.u[k] = lattice(LB.f[k], lshift, 24);
            }
        }
        uint32_t* pk = picks ? picks + (q * a.spp + s) * 6 : nullptr;
        if (pk) {
#pragma unroll
            for (int k = 0; k < 6; ++k) pk[k] = NO_PICK;
        }
        Material fm = zero_material();
        float3 est = make_float3(0.f, 0.f, 0.f);
        if constexpr (BLEND == BLEND_STOCHASTIC) {
            const int pl = W > 0.0f ? cdf_pick<3>(w, B.u[4], 0, nullptr) : 2;
            const FetchCtx& T = TT.t[pl];
            const PlaneQ p = plane_query(pl, P, DX, DY, has_d, a.scale, T, flags);
            est = plane_sample<FILTER, MODE, TF>(T, p, s, a.kside, flags, has_d, A, B, 1.0f, a.shade, SC, fm,
                                                 pk ? pk + 2 * pl : nullptr);
        } else {
#pragma unroll 1
            for (int pl = 0; pl < 3; ++pl) {
                float bw = 1.0f;
                if (W > 0.0f) {
                    const float wp = pl == 0 ? w[0] : pl == 1 ? w[1] : w[2];
                    if (!(wp > 0.0f)) continue;
                    bw = __fdiv_rn(wp, W);
                } else if (pl != 2) {
                    continue;
                }
                const FetchCtx& T = TT.t[pl];
                const PlaneQ p = plane_query(pl, P, DX, DY, has_d, a.scale, T, flags);
                const float3 e = plane_sample<FILTER, MODE, TF>(T, p, s, a.kside, flags, has_d, A, B, bw, a.shade,
                                                                SC, fm, pk ? pk + 2 * pl : nullptr);
                est.x += e.x; est.y += e.y; est.z += e.z;
            }
        }
        if (MODE == M_NTAP_BEFORE) est = shade_filtered(a.shade, fm, SC);
        acc.x += est.x; acc.y += est.y; acc.z += est.z;
    }
    const float inv_spp = 1.0f / (float)a.spp;
    __stcs(a.r + q, acc.x * inv_spp);
    __stcs(a.g + q, acc.y * inv_spp);
    __stcs(a.b + q, acc.z * inv_spp);
}

// The fully stochastic lookup at one sample per point with no flags, split at the texel
// load: the first half picks the plane and the texel and issues the load, the second decodes,
// shades and stores.  A thread runs the first half of two points before the second half of
// either, so two gathers are in flight per thread.  Same arithmetic as k_triplanar.
template <int TF> struct TriPick { typename RawOf<TF>::type raw; float wt; int plane; };

template <int FILTER, int TF>
__device__ __forceinline__ TriPick<TF> tri_pick_1spp(const TriplanarArgs& a, const TriTex& TT, const RoundKeys& K,
                                                     uint64_t q) {
    const bool has_d = a.has_derivs != 0;
    // the point and result streams are touched once: loaded and stored evict-first
    const float3 P = make_float3(__ldcs(a.px + q), __ldcs(a.py + q), __ldcs(a.pz + q));
    const float3 N = make_float3(__ldcs(a.nx + q), __ldcs(a.ny + q), __ldcs(a.nz + q));
    float3 DX = make_float3(0.f, 0.f, 0.f), DY = DX;
    if (has_d) {
        DX = make_float3(__ldcs(a.dxx + q), __ldcs(a.dxy + q), __ldcs(a.dxz + q));
        DY = make_float3(__ldcs(a.dyx + q), __ldcs(a.dyy + q), __ldcs(a.dyz + q));
    }
    if (isnan(P.x) || isnan(P.y) || isnan(P.z) || isnan(N.x) || isnan(N.y) || isnan(N.z) || isnan(DX.x) ||
        isnan(DX.y) || isnan(DX.z) || isnan(DY.x) || isnan(DY.y) || isnan(DY.z))
        atomicOr(a.status, DEV_NAN_INPUT);
    float w[4];
    const float W = tri_weights(N.x, N.y, N.z, w);
    const uint64_t id = a.id_base + q;
    const uint32_t id_lo = (uint32_t)id, id_hi = (uint32_t)(id >> 32);
    const U5 A = uniforms5(philox(id_lo, id_hi, 0u, 0u, K));
    const U5 B = uniforms5(philox(id_lo, id_hi, 0u, 1u, K));
    TriPick<TF> r;
    r.plane = W > 0.0f ? cdf_pick<3>(w, B.u[4], 0, nullptr) : 2;
    const FetchCtx& T = TT.t[r.plane];
    const PlaneQ p = plane_query(r.plane, P, DX, DY, has_d, a.scale, T, 0u);
    float x = p.u, y = p.v;
    if (has_d) jitter(0u, 1, 0u, A, p.dudx, p.dvdx, p.dudy, p.dvdy, &x, &y);
    const Pick1 k = pick_1tap<FILTER, TF>(T, x, y, p.l0, p.fr, A, false);
    r.raw = load_raw<TF>(T, k.lvl, k.ix, k.iy);
    r.wt = k.wt;
    return r;
}

template <int TF>
__device__ __forceinline__ void tri_finish_1spp(const TriplanarArgs& a, const TriTex& TT, const ShadeConst& SC,
                                                const TriPick<TF>& r, uint64_t q) {
    const float3 f = shade<clamp_rough<TF>()>(a.shade, decode_raw<TF>(TT.t[r.plane], r.raw), SC);
    __stcs(a.r + q, r.wt * f.x);
    __stcs(a.g + q, r.wt * f.y);
    __stcs(a.b + q, r.wt * f.z);
}

template <int FILTER, int TF>
__global__ void __launch_bounds__(256, 5)
k_triplanar_1spp_pair(TriplanarArgs a, const __grid_constant__ TriTex TT, ShadeConst SC, RoundKeys K) {
    const uint64_t half = (a.n + 1) / 2;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    const uint64_t j = i + half;
    const bool two = j < a.n;
    const uint64_t q0 = a.order ? (uint64_t)__ldg(a.order + i) : i;
    const uint64_t q1 = two ? (a.order ? (uint64_t)__ldg(a.order + j) : j) : q0;
    const TriPick<TF> r0 = tri_pick_1spp<FILTER, TF>(a, TT, K, q0);
    TriPick<TF> r1{};
    if (two) r1 = tri_pick_1spp<FILTER, TF>(a, TT, K, q1);
    tri_finish_1spp<TF>(a, TT, SC, r0, q0);
    if (two) tri_finish_1spp<TF>(a, TT, SC, r1, q1);
}

template <int FILTER, int MODE, int BLEND, int V, int TF>
static cudaError_t launch_tri_one(const TriplanarArgs& a, const TriTex& TT, cudaStream_t st) {
    const uint64_t blocks = (a.n + 255) / 256;
    const int grid = (int)(blocks < 0x7FFFFFFFull ? (blocks ? blocks : 1) : 0x7FFFFFFFull);
    k_triplanar<FILTER, MODE, BLEND, V, TF><<<grid, 256, 0, st>>>(a, TT, make_shade_const(), expand_key(a.seed));
    return cudaGetLastError();
}

template <int FILTER, int TF>
static cudaError_t launch_tri_pair(const TriplanarArgs& a, const TriTex& TT, cudaStream_t st) {
    const uint64_t blocks = ((a.n + 1) / 2 + 255) / 256;
    const int grid = (int)(blocks < 0x7FFFFFFFull ? (blocks ? blocks : 1) : 0x7FFFFFFFull);
    k_triplanar_1spp_pair<FILTER, TF><<<grid, 256, 0, st>>>(a, TT, make_shade_const(), expand_key(a.seed));
    return cudaGetLastError();
}

template <int FILTER, int MODE, int BLEND>
static cudaError_t launch_tri_fmb(const TriplanarArgs& a, const TriTex& TT, cudaStream_t st) {
    const bool dct = TT.t[0].fmt == FMT_DCT;
    const bool rgba8n = texture_family(TT.t[0]) == TF_RGBA8N && texture_family(TT.t[1]) == TF_RGBA8N &&
                        texture_family(TT.t[2]) == TF_RGBA8N;
    if constexpr (MODE == M_STOCHASTIC && BLEND == BLEND_STOCHASTIC) {
        // one sample, no flags, no picks: two points per thread
        if (a.spp == 1 && kernel_variant(a.flags, a.picks) == KV_PLAIN) {
            if (dct) return launch_tri_pair<FILTER, TF_DCT>(a, TT, st);
            return rgba8n ? launch_tri_pair<FILTER, TF_RGBA8N>(a, TT, st) : launch_tri_pair<FILTER, TF_BASIC>(a, TT, st);
        }
    }
    if (dct) {
        if (kernel_variant(a.flags, a.picks) == KV_PLAIN) return launch_tri_one<FILTER, MODE, BLEND, KV_PLAIN, TF_DCT>(a, TT, st);
        return launch_tri_one<FILTER, MODE, BLEND, KV_GENERAL, TF_DCT>(a, TT, st);
    }
    switch (kernel_variant(a.flags, a.picks)) {
        case KV_PLAIN:
            if (rgba8n) return launch_tri_one<FILTER, MODE, BLEND, KV_PLAIN, TF_RGBA8N>(a, TT, st);
            return launch_tri_one<FILTER, MODE, BLEND, KV_PLAIN, TF_BASIC>(a, TT, st);
        case KV_LATTICE:
            if constexpr (MODE == M_STOCHASTIC || MODE == M_POSITIVIZED) {
                if (rgba8n) return launch_tri_one<FILTER, MODE, BLEND, KV_LATTICE, TF_RGBA8N>(a, TT, st);
                return launch_tri_one<FILTER, MODE, BLEND, KV_LATTICE, TF_BASIC>(a, TT, st);
            }
            break;
        default: break;
    }
    return launch_tri_one<FILTER, MODE, BLEND, KV_GENERAL, TF_BASIC>(a, TT, st);
}

template <int FILTER, int MODE>
static cudaError_t launch_tri_fm(const TriplanarArgs& a, const TriTex& TT, cudaStream_t st) {
    return a.blend == BLEND_STOCHASTIC ? launch_tri_fmb<FILTER, MODE, BLEND_STOCHASTIC>(a, TT, st)
                                       : launch_tri_fmb<FILTER, MODE, BLEND_FULL>(a, TT, st);
}

template <int FILTER>
static cudaError_t launch_tri_f(const TriplanarArgs& a, const TriTex& TT, cudaStream_t st) {
    switch (a.mode) {
        case M_NTAP_BEFORE: return launch_tri_fm<FILTER, M_NTAP_BEFORE>(a, TT, st);
        case M_NTAP_AFTER: return launch_tri_fm<FILTER, M_NTAP_AFTER>(a, TT, st);
        case M_STOCHASTIC: return launch_tri_fm<FILTER, M_STOCHASTIC>(a, TT, st);
        case M_POSITIVIZED:
            if constexpr (is_signed(FILTER)) return launch_tri_fm<FILTER, M_POSITIVIZED>(a, TT, st);
            return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_triplanar(const TriplanarArgs& a, const TexView tv[3], cudaStream_t st) {
    TriTex TT;
    for (int i = 0; i < 3; ++i) TT.t[i] = make_fetch_ctx(tv[i]);
    switch (a.filter) {
        case F_LINEAR: return launch_tri_f<F_LINEAR>(a, TT, st);
        case F_BSPLINE: return launch_tri_f<F_BSPLINE>(a, TT, st);
        case F_CATMULL_ROM: return launch_tri_f<F_CATMULL_ROM>(a, TT, st);
        case F_MITCHELL: return launch_tri_f<F_MITCHELL>(a, TT, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stf
