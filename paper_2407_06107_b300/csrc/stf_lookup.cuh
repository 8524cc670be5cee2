// One 2-D texture lookup, step by step: texel load and decode per storage format, the LOD
// of a derivative footprint, the screen-space jitter, and the per-sample filters (a 1-tap
// stochastic pick, positivization's two picks, the N-tap sums).  The 2-D kernels and the
// triplanar kernels (three such lookups per query) are built from these.
#pragma once
#include "stf_kernels.h"
#include "stf_device.cuh"

namespace stf {

// A texel as loaded: RGBA32F uses all four words, RGBA8 + RG8 the first two.  Loading and
// decoding are separate so that a sample's load can be issued before the previous
// sample is shaded.
__device__ __forceinline__ uint4 load_texel(const FetchCtx& T, int lvl, int ix, int iy) {
    // a level has at most 16384^2 = 2^28 texels: the index fits 32 bits
    const uint32_t idx = (uint32_t)iy * (uint32_t)T.w[lvl] + (uint32_t)ix;
    if (T.fmt == FMT_RGBA32F) return __ldg(reinterpret_cast<const uint4*>(T.base + T.off[lvl]) + idx);
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(T.base + T.off[lvl]) + idx);
    return make_uint4(t.x, t.y, 0u, 0u);
}
__device__ __forceinline__ Material decode_texel(const FetchCtx& T, uint4 r) {
    if (T.fmt == FMT_RGBA32F)
        return decode_rgba32f(make_float4(__uint_as_float(r.x), __uint_as_float(r.y), __uint_as_float(r.z), __uint_as_float(r.w)));
    return decode_rgba8(make_uint2(r.x, r.y), T.has_normal != 0);
}
__device__ __forceinline__ Material fetch(const FetchCtx& T, int lvl, int ix, int iy) {
    return decode_texel(T, load_texel(T, lvl, ix, iy));
}

// Texture-format family of a kernel instantiation: BASIC (RGBA32F or RGBA8 + RG8, told apart
// at run time), RGBA8N (RGBA8 with its RG8 normal map, fixed at compile time: no format tests
// per texel) or DCT (compressed blocks, decoded per texel).  A loaded texel's type and its
// decode depend on the family, so the DCT path adds no registers to the others.
enum { TF_BASIC = 0, TF_DCT = 1, TF_RGBA8N = 2 };
template <int TF> struct RawOf { using type = uint4; };
template <> struct RawOf<TF_DCT> { using type = DctRaw; };
template <> struct RawOf<TF_RGBA8N> { using type = uint2; };

// Whether a decoded texel's roughness needs clamping to [0.05, 1] before shading: an RGBA32F
// texel holds any value; the other formats decode to 0.05 + 0.95 x with x in [0, 1].
template <int TF> constexpr bool clamp_rough() { return TF == TF_BASIC; }

// the family a texture's kernels may use: RGBA8N for RGBA8 textures with a normal map whose
// levels all have power-of-two sides (wrap addressing is then a mask)
inline int texture_family(const FetchCtx& T) {
    if (T.fmt == FMT_DCT) return TF_DCT;
    if (T.fmt != FMT_RGBA8 || !T.has_normal) return TF_BASIC;
    for (int l = 0; l < T.levels; ++l)
        if ((T.w[l] & (T.w[l] - 1)) != 0 || (T.h[l] & (T.h[l] - 1)) != 0) return TF_BASIC;
    return TF_RGBA8N;
}

// wrap addressing of index i on an axis of n texels: a mask for the RGBA8N family's
// power-of-two levels, the general modulo otherwise
template <int TF>
__device__ __forceinline__ int wrap_t(int i, int n) {
    if constexpr (TF == TF_RGBA8N) return i & (n - 1);
    else return wrap_index(i, n);
}

template <int TF>
__device__ __forceinline__ typename RawOf<TF>::type load_raw(const FetchCtx& T, int lvl, int ix, int iy) {
    if constexpr (TF == TF_DCT) {
        return load_dct(T.base + T.off[lvl], T.w[lvl], ix, iy);
    } else if constexpr (TF == TF_RGBA8N) {
        const uint32_t idx = (uint32_t)iy * (uint32_t)T.w[lvl] + (uint32_t)ix;
        return __ldg(reinterpret_cast<const uint2*>(T.base + T.off[lvl]) + idx);
    } else {
        return load_texel(T, lvl, ix, iy);
    }
}
template <int TF>
__device__ __forceinline__ Material decode_raw(const FetchCtx& T, const typename RawOf<TF>::type& r) {
    if constexpr (TF == TF_DCT) return decode_dct(r);
    else if constexpr (TF == TF_RGBA8N) return decode_rgba8(r, true);
    else return decode_texel(T, r);
}
template <int TF>
__device__ __forceinline__ Material fetch_t(const FetchCtx& T, int lvl, int ix, int iy) {
    return decode_raw<TF>(T, load_raw<TF>(T, lvl, ix, iy));
}

__device__ __forceinline__ uint32_t pack_pick(int lvl, int ix, int iy) {
    return ((uint32_t)lvl << 28) | ((uint32_t)iy << 14) | (uint32_t)ix;
}

// LOD from the derivative footprint: log2 of the minor axis in level-0 texels with the
// anisotropy capped at 64 (supplement listing computeLodAniso), clamped to [0, L-1].
__device__ __forceinline__ float lod_aniso(float dudx, float dvdx, float dudy, float dvdy,
                                           float W, float H, int levels) {
    const float ax = __fmul_rn(dudx, W), ay = __fmul_rn(dvdx, H);
    const float bx = __fmul_rn(dudy, W), by = __fmul_rn(dvdy, H);
    const float la = __fmaf_rn(ay, ay, __fmul_rn(ax, ax));
    const float lb = __fmaf_rn(by, by, __fmul_rn(bx, bx));
    float mn = la, mx = lb;
    if (mn > mx) { mn = lb; mx = la; }
    float minl = sqrtf(mn);
    const float maxl = sqrtf(mx);
    if (minl > 0.0f && __fmul_rn(minl, 64.0f) < maxl) minl = __fmul_rn(maxl, 1.0f / 64.0f);
    const float l = log2f(minl);
    return fminf(fmaxf(l, 0.0f), (float)(levels - 1));
}

// Screen-space jitter of sample s inside the derivative footprint (Sec. 4.2.1): a uniform
// offset in [-1/2, 1/2)^2, or the centre of cell s of a kside x kside grid (stratified).
__device__ __forceinline__ void jitter(uint32_t s, int kside, uint32_t flags, const U5& A, float dudx, float dvdx,
                                       float dudy, float dvdy, float* x, float* y) {
    float jx, jy;
    if (flags & FLAG_STRATIFIED) {
        jx = __fsub_rn(__fdiv_rn(__fadd_rn((float)(s % kside), 0.5f), (float)kside), 0.5f);
        jy = __fsub_rn(__fdiv_rn(__fadd_rn((float)(s / kside), 0.5f), (float)kside), 0.5f);
    } else {
        jx = __fsub_rn(A.u[0], 0.5f);
        jy = __fsub_rn(A.u[1], 0.5f);
    }
    *x = __fmaf_rn(jy, dudy, __fmaf_rn(jx, dudx, *x));
    *y = __fmaf_rn(jy, dvdy, __fmaf_rn(jx, dvdx, *y));
}


// Both axes' raster positions at once in packed FP32 pairs: the same values as axis_pos on x
// and on y (one rounding per lane)
__device__ __forceinline__ void axis_pos2(float x, float y, float W, float H, AxisPos* ax, AxisPos* ay) {
    const float2 p = upk2(vfma(f2(x, y), f2(W, H), vconst<F2>(-0.5f)).v);
    const float fx = floorf(p.x), fy = floorf(p.y);
    const float2 t = upk2(vsub(f2(p.x, p.y), f2(fx, fy)).v);
    *ax = {(int)fx, t.x};
    *ay = {(int)fy, t.y};
}

// ---------------------------------------------------------------- per-sample filters
// Each takes the (jittered) position (x, y) in texture coordinates, the query's level floor
// l0 and fraction fr, and the sample's uniforms.

// 1-tap stochastic pick: stochastic level floor(lambda) + [xi < frac(lambda)] (supplement
// "Linear Filters"), per-axis weights, per-axis CDF picks (Sec. 2.2 "Sampling arrays",
// separable FRS Sec. 4.1); wt = sign * S_x * S_y for a signed filter, else 1 (Eq.
// stochastic-sum).  reuse: one uniform drives the level and both axes, remapped per decision.
struct Pick1 { int lvl, ix, iy; float wt; };

template <int FILTER, int TF = TF_BASIC>
__device__ __forceinline__ Pick1 pick_1tap(const FetchCtx& T, float x, float y, int l0, float fr, const U5& A,
                                           bool reuse) {
    constexpr int NT = ntaps(FILTER), T0 = tap0(FILTER);
    int lvl = l0 + ((A.u[2] < fr) ? 1 : 0);
    float ru = A.u[2];
    if (reuse) {
        float r2;
        lvl = l0 + level_reuse(A.u[2], fr, &r2);
        ru = r2;
    }
    lvl = min(lvl, T.levels - 1);
    const int W = T.w[lvl], H = T.h[lvl];
    AxisPos ax, ay;
    if constexpr (TF == TF_RGBA8N && !is_signed(FILTER)) {   // packed: faster for the positive filters
        axis_pos2(x, y, (float)W, (float)H, &ax, &ay);
    } else {
        ax = axis_pos(x, (float)W);
        ay = axis_pos(y, (float)H);
    }
    Pick1 p;
    p.lvl = lvl;
    p.wt = 1.0f;
    if constexpr (!is_signed(FILTER)) {
        if (!reuse) {   // a positive filter's pick needs no weights: its CDF in closed form
            int kx, ky;
            if constexpr (TF == TF_RGBA8N) {
                pick_positive2<FILTER>(ax.t, ay.t, A.u[3], A.u[4], &kx, &ky);
            } else {
                kx = pick_positive<FILTER>(ax.t, A.u[3]);
                ky = pick_positive<FILTER>(ay.t, A.u[4]);
            }
            p.ix = wrap_t<TF>(ax.i0 + T0 + kx, W);
            p.iy = wrap_t<TF>(ay.i0 + T0 + ky, H);
            return p;
        }
    }
    float wx[4], wy[4];
    axis_pick_weights<FILTER>(ax.t, wx);
    axis_pick_weights<FILTER>(ay.t, wy);
    float Sx, Sy;
    int kx, ky;
    bool nx = false, ny = false;     // sign of the picked weight per axis
    if (reuse) {
        float uy, dummy;
        kx = cdf_pick_reuse<NT>(wx, ru, &uy);
        ky = cdf_pick_reuse<NT>(wy, uy, &dummy);
        if (is_signed(FILTER)) {
            cdf_pick<NT>(wx, 0.0f, 0, &Sx); cdf_pick<NT>(wy, 0.0f, 0, &Sy);
            // the sign of the picked weight, selected without dynamic register indexing
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                nx = (k == kx) ? (wx[k] < 0.0f) : nx;
                ny = (k == ky) ? (wy[k] < 0.0f) : ny;
            }
        }
    } else if (is_signed(FILTER)) {
        kx = cdf_pick_sign<NT, true>(wx, A.u[3], &Sx, &nx);
        ky = cdf_pick_sign<NT, true>(wy, A.u[4], &Sy, &ny);
    } else {
        kx = cdf_pick<NT>(wx, A.u[3], 0, &Sx);
        ky = cdf_pick<NT>(wy, A.u[4], 0, &Sy);
    }
    p.ix = wrap_t<TF>(ax.i0 + T0 + kx, W);
    p.iy = wrap_t<TF>(ay.i0 + T0 + ky, H);
    if (is_signed(FILTER)) {
        p.wt = Sx * Sy;
        if constexpr (pick_weight_scale<FILTER>() != 1.0f) p.wt = __fmul_rn(p.wt, pick_weight_scale<FILTER>());
        if (nx != ny) p.wt = -p.wt;
    }
    return p;
}

// Positivization (Sec. 2.2): one texel from the positive set and one from the negative set
// of the separable weights, est = W+ f(t+) - W- f(t-).  Stream 1 uniforms B: (positive
// class, negative pick x, negative pick y, negative class).  Both loads are issued before
// either texel is shaded.  pk_pos / pk_neg receive the packed picks (NO_PICK: none).
template <int FILTER, int TF>
__device__ __forceinline__ float3 positivized_sample(const FetchCtx& T, float x, float y, int l0, float fr,
                                                     const U5& A, const U5& B, int shade_mode, const ShadeConst& SC,
                                                     uint32_t* pk_pos, uint32_t* pk_neg) {
    constexpr int NT = ntaps(FILTER), T0 = tap0(FILTER);
    const int lvl = min(l0 + ((A.u[2] < fr) ? 1 : 0), T.levels - 1);
    const int W = T.w[lvl], H = T.h[lvl];
    const AxisPos ax = axis_pos(x, (float)W), ay = axis_pos(y, (float)H);
    float wx[4], wy[4];
    axis_weights<FILTER>(ax.t, wx);
    axis_weights<FILTER>(ay.t, wy);
    // the 4-tap signed filters' class sums and picks from their sign structure (signed_axis4),
    // the others' from the class CDFs; the values are the same either way
    constexpr bool S4 = NT == 4 && is_signed(FILTER);
    SignedAxis4 sx{}, sy{};
    float Px, Nx, Py, Ny;
    if constexpr (S4) {
        sx = signed_axis4(wx); sy = signed_axis4(wy);
        Px = sx.P; Nx = sx.N; Py = sy.P; Ny = sy.N;
    } else {
        cdf_pick<NT>(wx, 0.0f, +1, &Px); cdf_pick<NT>(wx, 0.0f, -1, &Nx);
        cdf_pick<NT>(wy, 0.0f, +1, &Py); cdf_pick<NT>(wy, 0.0f, -1, &Ny);
    }
    auto pick = [&](const float w[4], const SignedAxis4& sa, float xi, int cls) {
        if constexpr (S4) return signed_pick4(sa, xi, cls);
        else return cdf_pick<NT>(w, xi, cls, nullptr);
    };
    const float Wp = __fmaf_rn(Nx, Ny, __fmul_rn(Px, Py));
    const float Wn = __fmaf_rn(Nx, Py, __fmul_rn(Px, Ny));
    const int cp = (__fmul_rn(B.u[0], Wp) < __fmul_rn(Px, Py)) ? +1 : -1;
    const int kx = pick(wx, sx, A.u[3], cp);
    const int ky = pick(wy, sy, A.u[4], cp);
    const int ix = wrap_t<TF>(ax.i0 + T0 + kx, W), iy = wrap_t<TF>(ay.i0 + T0 + ky, H);
    const typename RawOf<TF>::type raw_p = load_raw<TF>(T, lvl, ix, iy);
    uint32_t negpick = NO_PICK;
    typename RawOf<TF>::type raw_n{};
    if (Wn > 0.0f) {
        const int cn = (__fmul_rn(B.u[3], Wn) < __fmul_rn(Px, Ny)) ? +1 : -1;
        const int qx = pick(wx, sx, B.u[1], cn);
        const int qy = pick(wy, sy, B.u[2], -cn);
        const int jx = wrap_t<TF>(ax.i0 + T0 + qx, W), jy = wrap_t<TF>(ay.i0 + T0 + qy, H);
        raw_n = load_raw<TF>(T, lvl, jx, jy);
        negpick = pack_pick(lvl, jx, jy);
    }
    const float3 f = shade<clamp_rough<TF>()>(shade_mode, decode_raw<TF>(T, raw_p), SC);
    float3 est = make_float3(Wp * f.x, Wp * f.y, Wp * f.z);
    if (Wn > 0.0f) {
        const float3 g = shade<clamp_rough<TF>()>(shade_mode, decode_raw<TF>(T, raw_n), SC);
        est.x = fmaf(-Wn, g.x, est.x);
        est.y = fmaf(-Wn, g.y, est.y);
        est.z = fmaf(-Wn, g.z, est.z);
    }
    *pk_pos = pack_pick(lvl, ix, iy);
    *pk_neg = negpick;
    return est;
}

// N-tap: every tap of levels floor(lambda) and floor(lambda) + 1, each weighted by
// scale * level weight * w_x * w_y.  Filter-before (MODE M_NTAP_BEFORE) adds the decoded
// materials into fm (Eq. filter-before-shading); filter-after adds the shaded taps into fsum
// (Eq. filtering-after-shading).
template <int FILTER, int MODE, int TF>
__device__ __forceinline__ void ntap_accumulate(const FetchCtx& T, float x, float y, int l0, float fr, float scale,
                                                int shade_mode, const ShadeConst& SC, Material& fm, float3& fsum) {
    constexpr int NT = ntaps(FILTER), T0 = tap0(FILTER);
#pragma unroll 1
    for (int li = 0; li < 2; ++li) {
        const int lvl = l0 + li;
        const float wl = scale * (li == 0 ? __fsub_rn(1.0f, fr) : fr);
        if (wl == 0.0f || lvl >= T.levels) continue;
        const int W = T.w[lvl], H = T.h[lvl];
        const AxisPos ax = axis_pos(x, (float)W), ay = axis_pos(y, (float)H);
        float wx[4], wy[4];
        axis_weights<FILTER>(ax.t, wx);
        axis_weights<FILTER>(ay.t, wy);
        // the window's wrapped columns and rows: one full wrap per axis, then +1 steps
        int cx[4], ry[4];
        cx[0] = wrap_t<TF>(ax.i0 + T0, W);
        ry[0] = wrap_t<TF>(ay.i0 + T0, H);
#pragma unroll
        for (int k = 1; k < NT; ++k) {
            cx[k] = cx[k - 1] + 1 == W ? 0 : cx[k - 1] + 1;
            ry[k] = ry[k - 1] + 1 == H ? 0 : ry[k - 1] + 1;
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int iy = ry[j];
            const float wyl = wl * wy[j];
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const float w = wyl * wx[i];
                // a zero weight adds nothing to finite texels; RGBA8 and DCT decodes are always
                // finite, RGBA32F ones need not be, and 0 * inf must not enter the sum
                if (TF == TF_BASIC && w == 0.0f) continue;
                const int ix = cx[i];
                const Material m = fetch_t<TF>(T, lvl, ix, iy);
                if (MODE == M_NTAP_BEFORE) {
                    fm.rho.x = fmaf(w, m.rho.x, fm.rho.x);
                    fm.rho.y = fmaf(w, m.rho.y, fm.rho.y);
                    fm.rho.z = fmaf(w, m.rho.z, fm.rho.z);
                    fm.rough = fmaf(w, m.rough, fm.rough);
                    fm.n.x = fmaf(w, m.n.x, fm.n.x);
                    fm.n.y = fmaf(w, m.n.y, fm.n.y);
                    fm.n.z = fmaf(w, m.n.z, fm.n.z);
                } else {
                    const float3 f = shade<clamp_rough<TF>()>(shade_mode, m, SC);
                    fsum.x = fmaf(w, f.x, fsum.x);
                    fsum.y = fmaf(w, f.y, fsum.y);
                    fsum.z = fmaf(w, f.z, fsum.z);
                }
            }
        }
    }
}

__device__ __forceinline__ Material zero_material() {
    Material fm;
    fm.rho = make_float3(0.f, 0.f, 0.f);
    fm.rough = 0.f;
    fm.n = make_float3(0.f, 0.f, 0.f);
    return fm;
}

// Filter-before-shading's last step: renormalise the filtered normal (+z if it vanished)
// and shade the filtered material once.
__device__ __forceinline__ float3 shade_filtered(int shade_mode, Material fm, const ShadeConst& SC) {
    const float ln2 = dot3(fm.n, fm.n);
    if (ln2 > 0.0f) {
        const float inv = 1.0f / sqrtf(ln2);
        fm.n = make_float3(fm.n.x * inv, fm.n.y * inv, fm.n.z * inv);
    } else {
        fm.n = make_float3(0.f, 0.f, 1.f);
    }
    return shade(shade_mode, fm, SC);
}

}  // namespace stf
