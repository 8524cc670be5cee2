// FP64 CPU oracle for stochastic texture filtering -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, obviously-correct restatement of what the paper's method computes
// (Pharr, Wronski, Salvi, Fajardo 2024, "Filtering After Shading With Stochastic
// Texture Filtering").  Only tests/, the smoke check and bench.py's CPU-baseline leg
// may load this library; the CUDA product path never does, and the two share no code.
//
// Structure of one lookup (2-D):
//   * screen-space jitter of the lookup point inside the pixel footprint (Sec. 4.2.1,
//     Fig. 6), the stochastic MIP level (Sec. 4.2.1; supplement "Real-time anisotropic
//     filtering", and the stochastic lerp of supplement Sec. "Linear Filters"),
//   * separable filter weights from the 1-D kernels of supplement Sec. "Filter Kernels"
//     (tent, Keys cubic, cubic B-spline) and Mitchell-Netravali BC(1/3,1/3),
//   * the estimators: filter-before-shading (Eq. filter-before-shading), exact
//     filter-after-shading (Eq. filtering-after-shading), single-tap stochastic
//     estimator (Eq. stochastic-sum with CDF inversion, Sec. 2.2 "Sampling arrays") and
//     positivization (Sec. 2.2 "Positivization").
//
// Precision.  Everything that *decides an integer* (which MIP level, which texel) is
// evaluated in FP32 as the paper's listings do (they are float code), with a fixed
// operation order; multiply-add chains use explicit single-rounded fmaf and nothing else
// is contracted.  Every *value* (filter weights used
// for sums, shading, transmittance, averages) is FP64.  For every decision the oracle
// also takes the same decision from FP64 quantities and reports the distance of the
// uniform to the nearest FP64 CDF boundary, so that tests can check that FP32 and FP64
// decisions differ only next to a boundary.
//
// Parity status of each function: see the pins in tests/test_oracle_*.py.
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw 2011), keyed by
// (seed, query/pixel id, sample, stream); the uniform is the top 24 bits * 2^-24.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <thread>
#include <vector>

#include "oracle_internal.h"

namespace {

// ------------------------------------------------------------------ enums (API values)
enum { F_LINEAR = 0, F_BSPLINE = 1, F_CATMULL_ROM = 2, F_MITCHELL = 3, F_EWA = 4,
       F_GAUSS = 5, F_GAUSS_BOX = 6, F_FIS_LINEAR = 7, F_FIS_BSPLINE = 8, F_FIS_GAUSS = 9 };
enum { M_NTAP_BEFORE = 0, M_NTAP_AFTER = 1, M_STOCHASTIC = 2, M_POSITIVIZED = 3 };
enum { S_GGX_LAMBERT = 0, S_LINEAR = 1 };
enum { FLAG_STRATIFIED = 1u, FLAG_LATTICE = 2u, FLAG_REUSE = 4u, FLAG_LOD0 = 8u };
enum { FMT_RGBA32F = 0, FMT_RGBA8 = 1, FMT_NEURAL = 2, FMT_DCT = 3 };
enum { ADDR_WRAP = 0, ADDR_CLAMP = 1 };
const uint32_t NO_PICK = 0xFFFFFFFFu;

// ------------------------------------------------------------------ Philox4x32-10
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   // round multipliers
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   // Weyl key increments
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * x0, p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void draw(uint64_t seed, uint64_t id, uint32_t sample, uint32_t stream, uint32_t out[4]) {
    uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), sample, stream};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    philox4x32_10(c, k, out);
}

// uniform in [0,1) on the 2^-24 grid; exactly representable in float and double
inline float unif(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }

// Five 24-bit uniforms from one Philox output: the high 24 bits of each word, and a fifth
// assembled from the low bytes of words 0, 1 and 2 (bits no other uniform uses).
void uniforms5(const uint32_t w[4], float u[5]) {
    for (int i = 0; i < 4; ++i) u[i] = unif(w[i]);
    uint32_t f = ((w[0] & 0xFFu) << 16) | ((w[1] & 0xFFu) << 8) | (w[2] & 0xFFu);
    u[4] = (float)f * 5.9604644775390625e-8f;
}

// Integer forms of uniforms5 (24-bit numerators) and uniforms6 (21-bit numerators).
void ints5(const uint32_t w[4], uint32_t f[5]) {
    for (int i = 0; i < 4; ++i) f[i] = w[i] >> 8;
    f[4] = ((w[0] & 0xFFu) << 16) | ((w[1] & 0xFFu) << 8) | (w[2] & 0xFFu);
}
void ints6(const uint32_t w[4], uint32_t f[6]) {
    for (int i = 0; i < 4; ++i) f[i] = w[i] >> 11;
    f[4] = (w[0] & 0x7FFu) | ((w[1] & 0x3FFu) << 11);
    f[5] = (w[2] & 0x7FFu) | ((w[3] & 0x3FFu) << 11);
}
// Randomly shifted lattice over the spp samples of one query (FLAG_LATTICE): sample s of
// spp takes frac(s/spp + phi), phi a per-query Philox offset; in exact integer arithmetic
// on the 2^bits grid.  Each value is uniform; the spp values are stratified.
float lattice(uint32_t phi, uint32_t s, uint32_t spp, int bits) {
    uint32_t mask = (1u << bits) - 1u;
    uint32_t shift = (uint32_t)(((uint64_t)s << bits) / spp);
    return (float)((phi + shift) & mask) * std::ldexp(1.0f, -bits);
}

// Six 21-bit uniforms from one Philox output (two volume march steps, three each).
void uniforms6(const uint32_t w[4], float u[6]) {
    const float k = 4.76837158203125e-7f;   // 2^-21
    for (int i = 0; i < 4; ++i) u[i] = (float)(w[i] >> 11) * k;
    u[4] = (float)((w[0] & 0x7FFu) | ((w[1] & 0x3FFu) << 11)) * k;
    u[5] = (float)((w[2] & 0x7FFu) | ((w[3] & 0x3FFu) << 11)) * k;
}

// ------------------------------------------------------------------ 1-D kernels, FP64
// supplement "Filter Kernels": tent K1, Keys cubic K3(a), cubic B-spline K_bs;
// Mitchell & Netravali (1988) BC family (cited beside K3 in the supplement).
double k_tent(double d) { d = std::fabs(d); return d < 1.0 ? 1.0 - d : 0.0; }
double k_bspline(double d) {
    d = std::fabs(d);
    if (d <= 1.0) return (4.0 - 3.0 * d * d * (2.0 - d)) / 6.0;
    if (d <= 2.0) { double e = 2.0 - d; return e * e * e / 6.0; }
    return 0.0;
}
double k_keys(double a, double d) {
    d = std::fabs(d);
    if (d < 1.0) return (a + 2.0) * d * d * d - (a + 3.0) * d * d + 1.0;
    if (d < 2.0) return a * d * d * d - 5.0 * a * d * d + 8.0 * a * d - 4.0 * a;
    return 0.0;
}
double k_bc(double B, double C, double d) {
    d = std::fabs(d);
    if (d < 1.0)
        return ((12.0 - 9.0 * B - 6.0 * C) * d * d * d + (-18.0 + 12.0 * B + 6.0 * C) * d * d +
                (6.0 - 2.0 * B)) / 6.0;
    if (d < 2.0)
        return ((-B - 6.0 * C) * d * d * d + (6.0 * B + 30.0 * C) * d * d +
                (-12.0 * B - 48.0 * C) * d + (8.0 * B + 24.0 * C)) / 6.0;
    return 0.0;
}
// The filters the lookups use, with the signed cubics written as products of their root
// factors: the same polynomials as k_keys(-1/2) and k_bc(1/3, 1/3), but a value next to a
// root keeps its relative precision (the expanded outer piece cancels near its double root
// at |d| = 2, and the ratio of such small weights decides a positivized class choice).
//   Keys a:   inner (d-1)((a+2) d^2 - d - 1), outer a (d-1)(d-2)^2
//   BC(B, C): outer (d-2)^2 ((-B-6C) d + 2B + 6C) / 6; for B = C = 1/3, (d-2)^2 (8-7d) / 18;
//             the inner piece stays above B/6 = 1/18 and keeps its expanded form.
double kernel64(int f, double d) {
    switch (f) {
        case F_LINEAR: return k_tent(d);
        case F_BSPLINE: return k_bspline(d);
        case F_CATMULL_ROM: {
            d = std::fabs(d);
            if (d < 1.0) return (d - 1.0) * (1.5 * d * d - d - 1.0);
            if (d < 2.0) return -0.5 * (d - 1.0) * (d - 2.0) * (d - 2.0);
            return 0.0;
        }
        case F_MITCHELL: {
            d = std::fabs(d);
            if (d < 1.0) return k_bc(1.0 / 3.0, 1.0 / 3.0, d);
            if (d < 2.0) return (d - 2.0) * (d - 2.0) * (8.0 - 7.0 * d) / 18.0;
            return 0.0;
        }
    }
    return 0.0;
}
int ntaps(int f) { return f == F_LINEAR ? 2 : 4; }
int first_tap(int f) { return f == F_LINEAR ? 0 : -1; }   // offset of tap 0 from floor(p)
bool signed_filter(int f) { return f == F_CATMULL_ROM || f == F_MITCHELL; }

// ------------------------------------------------------------------ FP32 decision weights
// Per-axis weights in float at the four tap distances 1+t, t, 1-t, 2-t (cubic) or 1-t, t
// (tent), in the forms a float implementation should use: the B-spline polynomials of the
// paper's bicubic/tricubic listings, and for the two signed cubics the pieces factored at
// their roots, so that a weight close to zero keeps its relative precision (the expanded
// outer polynomial loses it near the double root at |x| = 2, and only the ratio of such
// small weights decides the class choice of a positivized negative sample).  With s = 1-t:
//   Keys a = -1/2 (Catmull-Rom): outer a (x-1)(x-2)^2, inner (x-1)(3x^2/2 - x - 1)
//     w0 = -t s^2 / 2, w1 = s (1 + t (1 - 3t/2)), w2 = t (1 + s (1 - 3s/2)), w3 = -s t^2 / 2
//   Mitchell-Netravali BC(1/3, 1/3): outer (x-2)^2 (8 - 7x) / 18, inner 7x^3/6 - 2x^2 + 8/9
//     w0 = s^2 (1 - 7t) / 18, w3 = t^2 (7t - 6) / 18, w1, w2 the inner piece at t and s
//     (it stays above 1/18, so its Horner form loses nothing).
// Single-rounded fmaf is reproducible on any IEEE machine.  Used only to take decisions.
int weights32(int f, float t, float w[4]) {
    if (f == F_LINEAR) { w[0] = 1.0f - t; w[1] = t; return 2; }
    if (f == F_BSPLINE) {
        const float s = 1.0f / 6.0f;
        float t2 = t * t;
        float a;
        // the listing's polynomials in Horner form with fused multiply-adds:
        //   (1-t)^3, t^2 (3t - 6) + 4, t (t (3 - 3t) + 3) + 1, t^3, each times 1/6
        float omt = 1.0f - t;
        w[0] = s * ((omt * omt) * omt);
        a = std::fmaf(3.0f, t, -6.0f); w[1] = s * std::fmaf(t2, a, 4.0f);
        a = std::fmaf(-3.0f, t, 3.0f); a = std::fmaf(t, a, 3.0f); w[2] = s * std::fmaf(t, a, 1.0f);
        w[3] = s * (t2 * t);
        return 4;
    }
    const float s = 1.0f - t, t2 = t * t, s2 = s * s;
    if (f == F_CATMULL_ROM) {
        w[0] = (-0.5f * t) * s2;
        w[1] = s * std::fmaf(t, std::fmaf(-1.5f, t, 1.0f), 1.0f);
        w[2] = t * std::fmaf(s, std::fmaf(-1.5f, s, 1.0f), 1.0f);
        w[3] = (-0.5f * s) * t2;
        return 4;
    }
    // Mitchell B = C = 1/3
    const float k18 = 1.0f / 18.0f, c3 = 7.0f / 6.0f, c2 = -2.0f, c0 = 8.0f / 9.0f;
    w[0] = (s2 * std::fmaf(-7.0f, t, 1.0f)) * k18;
    w[1] = std::fmaf(std::fmaf(c3, t, c2) * t, t, c0);
    w[2] = std::fmaf(std::fmaf(c3, s, c2) * s, s, c0);
    w[3] = (t2 * std::fmaf(7.0f, t, -6.0f)) * k18;
    return 4;
}

// FP32 weights for a pick, where only their ratios matter: the B-spline's polynomials without
// the common factor 1/6, in the same operation order (the CDF inversion divides the factor out,
// and a positive filter's estimate carries weight 1); the other filters' weights32.
int pick_weights32(int f, float t, float w[4]) {
    if (f != F_BSPLINE) return weights32(f, t, w);
    const float t2 = t * t, omt = 1.0f - t;
    w[0] = (omt * omt) * omt;
    w[1] = std::fmaf(t2, std::fmaf(3.0f, t, -6.0f), 4.0f);
    w[2] = std::fmaf(t, std::fmaf(t, std::fmaf(-3.0f, t, 3.0f), 3.0f), 1.0f);
    w[3] = t2 * t;
    return 4;
}

// CDF inversion ("Sampling arrays"): first k with xi * S < prefix_k, S = sum |w|,
// restricted to taps of a sign class (cls = 0 all, +1 w > 0, -1 w < 0).
int pick32(const float* w, int n, float xi, int cls, float* total) {
    float C[4], acc = 0.0f;
    for (int k = 0; k < n; ++k) {
        bool in = cls == 0 || (cls > 0 ? w[k] > 0.0f : w[k] < 0.0f);
        acc = acc + (in ? std::fabs(w[k]) : 0.0f);
        C[k] = acc;
    }
    if (total) *total = acc;
    float target = xi * acc;
    for (int k = 0; k < n; ++k) if (target < C[k]) return k;
    return n - 1;
}
// Sample reuse (FLAG_REUSE): the same CDF pick, and the uniform remapped into the chosen
// interval, u' = (xi S - C_{k-1}) / (C_k - C_{k-1}) -- Eq. uniform-sample-reuse applied to a
// sampling array, as the bicubic listing's SampleDiscrete returns it.  FP32.
int pick32_reuse(const float* w, int n, float xi, float* remapped) {
    float C[4], acc = 0.0f;
    for (int k = 0; k < n; ++k) { acc = acc + std::fabs(w[k]); C[k] = acc; }
    float target = xi * acc;
    int k = n - 1;
    for (int j = n - 2; j >= 0; --j) if (target < C[j]) k = j;
    float lo = k > 0 ? C[k - 1] : 0.0f;
    *remapped = (target - lo) / (C[k] - lo);
    return k;
}
// Level decision with reuse: level+1 if xi < f, xi' = xi / f, else xi' = (xi - f) / (1 - f).
int level_reuse(float xi, float f, float* remapped) {
    if (xi < f) { *remapped = xi / f; return 1; }
    *remapped = (xi - f) / (1.0f - f);
    return 0;
}

// Same decision from FP64 weights; also the distance of xi to the nearest interior
// boundary of the FP64 CDF.
int pick64(const double* w, int n, double xi, int cls, double* bdist) {
    double S = 0.0, C[4];
    for (int k = 0; k < n; ++k) {
        bool in = cls == 0 || (cls > 0 ? w[k] > 0.0 : w[k] < 0.0);
        S += in ? std::fabs(w[k]) : 0.0;
        C[k] = S;
    }
    int pick = n - 1;
    bool found = false;
    double bd = 1e30;
    for (int k = 0; k < n; ++k) {
        double ck = S > 0 ? C[k] / S : 1.0;
        if (k < n - 1) bd = std::min(bd, std::fabs(xi - ck));
        if (!found && xi < ck) { pick = k; found = true; }
    }
    if (bdist) *bdist = std::min(*bdist, bd);
    return pick;
}

// Sample reuse in FP64: the pick of pick64 over all taps, and the uniform remapped into the
// chosen interval, xi' = (xi - c_{k-1}) / (c_k - c_{k-1}) on the normalised CDF c; *width =
// c_k - c_{k-1}.  `scale` is the width of the interval the incoming xi was itself remapped
// from, so scale * |xi - c_j| is the distance of the original uniform to this boundary.
int pick64_reuse(const double* w, int n, double xi, double* remapped, double* width, double scale,
                 double* bdist) {
    double S = 0.0, C[4];
    for (int k = 0; k < n; ++k) { S += std::fabs(w[k]); C[k] = S; }
    int pick = n - 1;
    bool found = false;
    double lo = 0.0, hi = 1.0, prev = 0.0, bd = 1e30;
    for (int k = 0; k < n; ++k) {
        const double ck = k == n - 1 ? 1.0 : C[k] / S;
        if (k < n - 1) bd = std::min(bd, scale * std::fabs(xi - ck));
        if (!found && xi < ck) { pick = k; found = true; lo = prev; hi = ck; }
        prev = ck;
    }
    if (!found) { lo = n > 1 ? C[n - 2] / S : 0.0; hi = 1.0; }
    *width = hi - lo;
    *remapped = (xi - lo) / (hi - lo);
    if (bdist) *bdist = std::min(*bdist, bd);
    return pick;
}

// ------------------------------------------------------------------ shading, FP64
// GGX (Trowbridge-Reitz) microfacet specular + Lambert diffuse, times the cosine
// factor: f_hat = [rho/pi + D G2 F / (4 nl nv)] nl.  The paper evaluates a Disney BRDF
// through this f_hat (Sec. 3); this restatement fixes l, v and F0 (see the design notes).
const double PI = 3.14159265358979323846;
struct V3 { double x, y, z; };
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline V3 normalize(V3 a) { double l = std::sqrt(dot(a, a)); return {a.x / l, a.y / l, a.z / l}; }
// fixed light and view directions, given as FP32 constants
const V3 LDIR = {(double)0.48f, (double)0.36f, (double)0.80f};
const V3 VDIR = {(double)-0.28f, (double)0.0f, (double)0.96f};
const double F0_DIELECTRIC = (double)0.04f;
const double ALPHA_MIN = (double)0.05f, ALPHA_MAX = 1.0;

double ggx_D(double a2, double nh, double s2) {     // s2 = |n x h|^2 = 1 - nh^2
    double q = a2 * nh * nh + s2;
    return a2 / (PI * q * q);
}
double smith_lambda(double a2, double tan2) { return 0.5 * (std::sqrt(1.0 + a2 * tan2) - 1.0); }

void ggx_eval(V3 n, V3 l, V3 v, double alpha, const double rho[3], double F0, double out[3]) {
    double nl = dot(n, l), nv = dot(n, v);
    if (!(nl > 0.0) || !(nv > 0.0)) { out[0] = out[1] = out[2] = 0.0; return; }
    double a = std::min(std::max(alpha, ALPHA_MIN), ALPHA_MAX), a2 = a * a;
    V3 h = normalize({l.x + v.x, l.y + v.y, l.z + v.z});
    V3 nxh = cross(n, h), nxl = cross(n, l), nxv = cross(n, v);
    double D = ggx_D(a2, dot(n, h), dot(nxh, nxh));
    double G = 1.0 / (1.0 + smith_lambda(a2, dot(nxl, nxl) / (nl * nl)) +
                      smith_lambda(a2, dot(nxv, nxv) / (nv * nv)));
    double vh = dot(v, h), m = 1.0 - vh;
    double F = F0 + (1.0 - F0) * m * m * m * m * m;
    double spec = D * G * F / (4.0 * nv);   // (D G F / (4 nl nv)) * nl
    for (int c = 0; c < 3; ++c) out[c] = rho[c] * nl / PI + spec;
}

// decoded material sample
struct Mat { double rho[3]; double rough; V3 n; };

void shade(int mode, const Mat& m, double out[3]) {
    if (mode == S_LINEAR) { for (int c = 0; c < 3; ++c) out[c] = m.rho[c]; return; }
    ggx_eval(m.n, LDIR, VDIR, m.rough, m.rho, F0_DIELECTRIC, out);
}

// ------------------------------------------------------------------ textures
struct Tex {
    int format, levels, address;
    int width[16], height[16];
    const void* data[16];
    const uint8_t* normal[16];
};

int wrapi(int i, int n, int addr) {
    if (addr == ADDR_CLAMP) return std::min(std::max(i, 0), n - 1);
    int r = i % n;
    return r < 0 ? r + n : r;
}

inline double clamp01(double x) { return std::min(std::max(x, 0.0), 1.0); }

// Map the 8 decoded channels of a learned texel to the material: albedo RGB, roughness,
// tangent-space normal XY (z reconstructed); channels 6 and 7 (metalness, height) are not
// used by the shade.
Mat material_from_channels(const double y[8]) {
    Mat m;
    for (int c = 0; c < 3; ++c) m.rho[c] = clamp01(y[c]);
    m.rough = 0.05 + 0.95 * clamp01(y[3]);
    double x = 2.0 * clamp01(y[4]) - 1.0, yy = 2.0 * clamp01(y[5]) - 1.0;
    double z = std::sqrt(std::max(0.0, 1.0 - x * x - yy * yy));
    double l = std::sqrt(x * x + yy * yy + z * z);
    m.n = l > 0 ? V3{x / l, yy / l, z / l} : V3{0.0, 0.0, 1.0};
    return m;
}

// DCT-compressed texel (supplement "Texture compression"): the inverse orthonormal 2-D DCT-II
// of one 8 x 8 block, restricted to the six stored frequencies u + v <= 2, evaluated at the
// texel's position (x, y) in the block.  Word layout: DC in bits 0-6 (q * 8/127), then the
// AC terms (1,0), (0,1), (2,0), (1,1), (0,2) in 5-bit fields ((q - 15) * 2/15).
double dct_texel(uint32_t w, int x, int y) {
    const double pi = 3.14159265358979323846;
    auto alpha = [](int k) { return k == 0 ? 1.0 / (2.0 * std::sqrt(2.0)) : 0.5; };
    auto basis = [&](int u, int v) {
        return alpha(u) * alpha(v) * std::cos((2 * x + 1) * u * pi / 16.0) * std::cos((2 * y + 1) * v * pi / 16.0);
    };
    double f = (double)(w & 127u) * (8.0 / 127.0) * basis(0, 0);
    const int uv[5][2] = {{1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
    for (int j = 0; j < 5; ++j) {
        const int q = (int)((w >> (7 + 5 * j)) & 31u) - 15;
        f += (double)q * (2.0 / 15.0) * basis(uv[j][0], uv[j][1]);
    }
    return f;
}

Mat fetch(const Tex& T, int lvl, int ix, int iy, double* rdist = nullptr) {
    Mat m;
    if (T.format == FMT_DCT) {        // six channels: albedo RGB, roughness, normal X, Y
        const int W8 = (T.width[lvl] + 7) / 8;
        const uint32_t* blk = (const uint32_t*)T.data[lvl] + ((size_t)(iy / 8) * W8 + (size_t)(ix / 8)) * 8;
        double y[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 6; ++c) y[c] = dct_texel(blk[c], ix % 8, iy % 8);
        return material_from_channels(y);
    }
    if (T.format == FMT_NEURAL) {     // learned texel: one MLP decode
        double y[8];
        orc::neural_decode(*(const orc::NeuralTex*)T.data[0], ix, iy, y, rdist);
        return material_from_channels(y);
    }
    size_t o = (size_t)iy * T.width[lvl] + ix;
    if (T.format == FMT_RGBA32F) {
        const float* p = (const float*)T.data[lvl] + 4 * o;
        m.rho[0] = p[0]; m.rho[1] = p[1]; m.rho[2] = p[2]; m.rough = p[3];
    } else {
        const uint8_t* p = (const uint8_t*)T.data[lvl] + 4 * o;
        for (int c = 0; c < 3; ++c) m.rho[c] = p[c] / 255.0;
        m.rough = 0.05 + 0.95 * (p[3] / 255.0);
    }
    if (T.normal[lvl]) {
        const uint8_t* q = T.normal[lvl] + 2 * o;
        double x = 2.0 * q[0] / 255.0 - 1.0, y = 2.0 * q[1] / 255.0 - 1.0;
        double z = std::sqrt(std::max(0.0, 1.0 - x * x - y * y));
        m.n = normalize({x, y, z});
    } else {
        m.n = {0.0, 0.0, 1.0};
    }
    return m;
}
inline uint32_t pack2d(int lvl, int ix, int iy) {
    return ((uint32_t)lvl << 28) | ((uint32_t)iy << 14) | (uint32_t)ix;
}

struct Queries {
    uint64_t n;
    const float *u, *v, *dudx, *dvdx, *dudy, *dvdy;   // derivs nullable (all or none)
};

// LOD from the screen-space derivatives: minor ellipse axis, anisotropy capped at 64
// (Sec. 4.2.1; supplement listing "computeLodAniso"), clamped to [0, L-1].
// FP32 as in the listing (decision precision), plus the FP64 value for boundary checks.
void lod(const Tex& T, const Queries& Q, uint64_t q, float* lam32, double* lam64) {
    if (!Q.dudx || T.levels <= 1) { *lam32 = 0.0f; *lam64 = 0.0; return; }
    float W = (float)T.width[0], H = (float)T.height[0];
    float ax = Q.dudx[q] * W, ay = Q.dvdx[q] * H, bx = Q.dudy[q] * W, by = Q.dvdy[q] * H;
    float la = std::fmaf(ay, ay, ax * ax);
    float lb = std::fmaf(by, by, bx * bx);
    float mn = la, mx = lb;
    if (mn > mx) { mn = lb; mx = la; }
    float minl = std::sqrt(mn), maxl = std::sqrt(mx);
    if (minl > 0.0f && minl * 64.0f < maxl) minl = maxl * (1.0f / 64.0f);
    float l = std::log2(minl);
    l = std::fmin(std::fmax(l, 0.0f), (float)(T.levels - 1));
    *lam32 = l;
    double A = (double)Q.dudx[q] * W, B = (double)Q.dvdx[q] * H;
    double C = (double)Q.dudy[q] * W, D = (double)Q.dvdy[q] * H;
    double a2 = A * A + B * B, b2 = C * C + D * D;
    double mn64 = std::sqrt(std::min(a2, b2)), mx64 = std::sqrt(std::max(a2, b2));
    if (mn64 > 0.0 && mn64 * 64.0 < mx64) mn64 = mx64 / 64.0;
    double l64 = std::log2(mn64);
    *lam64 = std::fmin(std::fmax(l64, 0.0), (double)(T.levels - 1));
}

struct Out {
    double* rgb;        // n*3
    uint32_t* picks;    // n*spp*2 or null (FP32 decisions)
    uint32_t* picks64;  // n*spp*2 or null (FP64 decisions)
    double* bdist;      // n or null: min distance of any uniform to an FP64 boundary
    double* mag;        // n*3 or null: mean over samples of sum |term| (scale of the sum)
    double* rdist;      // n or null: min relative distance of a BF16 decision to a boundary
};

// per level: FP32 texel position and tap geometry on one axis
struct Axis { int i0; float t; double pos; };
Axis axis_at(float x, int res) {
    float p = std::fmaf(x, (float)res, -0.5f);
    float fl = std::floor(p);
    return {(int)fl, p - fl, (double)p};
}

// ------------------------------------------------------------------ EWA
// Elliptically weighted average over a Gaussian (Greene and Heckbert 1986; Heckbert 1989),
// as the supplement's "Stochastic EWA" evaluates it, following pbrt.
//   * The ellipse is the implicit A s^2 + B s t + C t^2 < 1 in the texel space of the
//     chosen level (texel centres at integers, s = x W - 1/2).
//   * It is built from the two screen-space derivative vectors, each plus a one-texel
//     reconstruction term, with the minor axis stretched to major/64 when the eccentricity
//     exceeds 64 (the same cap as the LOD).
//   * Weights are exp(-2 r^2) - exp(-2), read from a 128-entry table at floor(128 r^2).
// The geometry and the table lookups decide which texels take part and with which
// weight, so they are FP32 with a fixed operation order (fmaf written out); every sum is
// FP64.  The bounding box's half-extents are capped at EWA_MAX_HALF texels (only a
// footprint many times larger than the coarsest level reaches the cap).
const int EWA_LUT_N = 128;
const float EWA_MAX_HALF = 256.0f;

const float* ewa_table() {
    static const std::vector<float> lut = [] {
        std::vector<float> t(EWA_LUT_N);
        for (int i = 0; i < EWA_LUT_N; ++i) {
            const double r2 = (double)i / (double)(EWA_LUT_N - 1);
            t[i] = (float)(std::exp(-2.0 * r2) - std::exp(-2.0));
        }
        return t;
    }();
    return lut.data();
}

struct Ewa {
    float cx, cy, A, B, C;
    int s0, s1, t0, t1;
    bool ok;
};

Ewa ewa_setup(float x, float y, float dudx, float dvdx, float dudy, float dvdy, int W, int H) {
    Ewa e{};
    e.cx = std::fmaf(x, (float)W, -0.5f);
    e.cy = std::fmaf(y, (float)H, -0.5f);
    float ax = dudx * (float)W, ay = dvdx * (float)H;   // screen x axis, in texels
    float bx = dudy * (float)W, by = dvdy * (float)H;   // screen y axis
    float la = std::fmaf(ay, ay, ax * ax), lb = std::fmaf(by, by, bx * bx);
    if (la < lb) { std::swap(ax, bx); std::swap(ay, by); std::swap(la, lb); }   // a: major axis
    const float lmaj = std::sqrt(la), lmin = std::sqrt(lb);
    if (lmin > 0.0f && lmin * 64.0f < lmaj) {
        const float sc = lmaj / (lmin * 64.0f);
        bx = bx * sc;
        by = by * sc;
    }
    float A = std::fmaf(ay, ay, std::fmaf(by, by, 1.0f));
    float B = -2.0f * std::fmaf(ax, ay, bx * by);
    float C = std::fmaf(ax, ax, std::fmaf(bx, bx, 1.0f));
    const float iF = 1.0f / std::fmaf(A, C, -0.25f * (B * B));
    A = A * iF; B = B * iF; C = C * iF;
    const float det = std::fmaf(4.0f * A, C, -(B * B));
    const float iD = 2.0f * (1.0f / det);
    const float hs = iD * std::sqrt(det * C), ht = iD * std::sqrt(A * det);
    e.A = A; e.B = B; e.C = C;
    e.ok = std::isfinite(e.cx) && std::isfinite(e.cy) && std::isfinite(hs) && std::isfinite(ht) &&
           std::fabs(e.cx) < 16777216.0f && std::fabs(e.cy) < 16777216.0f;
    if (!e.ok) return e;
    const float fx = std::floor(e.cx), fy = std::floor(e.cy);
    e.s0 = (int)std::ceil(std::fmax(e.cx - hs, fx - EWA_MAX_HALF));
    e.s1 = (int)std::floor(std::fmin(e.cx + hs, fx + EWA_MAX_HALF));
    e.t0 = (int)std::ceil(std::fmax(e.cy - ht, fy - EWA_MAX_HALF));
    e.t1 = (int)std::floor(std::fmin(e.cy + ht, fy + EWA_MAX_HALF));
    return e;
}

float ewa_weight(const Ewa& e, int s, int t) {
    const float ss = (float)s - e.cx, tt = (float)t - e.cy;
    const float r2 = std::fmaf(e.A * ss, ss, std::fmaf(e.B * ss, tt, (e.C * tt) * tt));
    if (!(r2 < 1.0f)) return 0.0f;
    const int idx = std::min((int)(r2 * (float)EWA_LUT_N), EWA_LUT_N - 1);
    return ewa_table()[idx];
}

// EWA lookups of one query (no screen-space jitter: the ellipse is the footprint).
//   * N-tap modes: both MIP levels, each normalised by its own weight sum, blended linearly.
//   * Stochastic: the stochastic level, then one texel by weighted reservoir sampling over the
//     box in raster order (t outer, s inner).  The uniform is remapped after every decision, as
//     in the listing.  bdist records the smallest |u - p| over the decisions.
void run_query_ewa(const Tex& T, const Queries& Q, uint64_t q, uint64_t id, int mode, int smode, uint32_t spp,
                   uint64_t seed, float lam32, double lam64, double bd, Out& O) {
    const int l0 = (int)std::floor(lam32);
    const float fr = lam32 - (float)l0;
    const float du0 = Q.dudx ? Q.dudx[q] : 0.0f, dv0 = Q.dudx ? Q.dvdx[q] : 0.0f;
    const float du1 = Q.dudx ? Q.dudy[q] : 0.0f, dv1 = Q.dudx ? Q.dvdy[q] : 0.0f;
    const float x = Q.u[q], y = Q.v[q];
    double acc[3] = {0, 0, 0}, mag[3] = {0, 0, 0};
    double rd = 1.0;
    for (uint32_t s = 0; s < spp; ++s) {
        uint32_t r0[4];
        draw(seed, id, s, 0, r0);
        float a[5];
        uniforms5(r0, a);
        uint32_t* pk = O.picks ? O.picks + (q * spp + s) * 2 : nullptr;
        uint32_t* pk64 = O.picks64 ? O.picks64 + (q * spp + s) * 2 : nullptr;
        if (pk) pk[0] = pk[1] = NO_PICK;
        if (pk64) pk64[0] = pk64[1] = NO_PICK;
        double est[3] = {0, 0, 0};
        if (mode == M_STOCHASTIC) {
            int lvl = std::min(l0 + ((a[2] < fr) ? 1 : 0), T.levels - 1);
            if (lam64 > 0.0 && lam64 < T.levels - 1) bd = std::min(bd, std::fabs((double)a[2] - (lam64 - std::floor(lam64))));
            const int W = T.width[lvl], H = T.height[lvl];
            const Ewa e = ewa_setup(x, y, du0, dv0, du1, dv1, W, H);
            float u = a[3], sum = 0.0f;
            int ps = 0, pt = 0;
            bool any = false;
            if (e.ok) {
                for (int t = e.t0; t <= e.t1; ++t)
                    for (int si = e.s0; si <= e.s1; ++si) {
                        const float w = ewa_weight(e, si, t);
                        if (!(w > 0.0f)) continue;
                        sum = sum + w;
                        const float p = w / sum;
                        if (any) bd = std::min(bd, std::fabs((double)u - (double)p));
                        if (u < p) { ps = si; pt = t; any = true; u = u / p; }
                        else u = (u - p) / (1.0f - p);
                    }
            }
            if (any) {
                const int ix = wrapi(ps, W, T.address), iy = wrapi(pt, H, T.address);
                double o[3];
                shade(smode, fetch(T, lvl, ix, iy, &rd), o);
                for (int c = 0; c < 3; ++c) { est[c] = o[c]; mag[c] += std::fabs(o[c]); }
                if (pk) pk[0] = pack2d(lvl, ix, iy);
                if (pk64) pk64[0] = pack2d(lvl, ix, iy);
            }
        } else {
            const double wl[2] = {1.0 - (double)fr, (double)fr};
            Mat fm{}; fm.n = {0, 0, 0};
            double fsum[3] = {0, 0, 0};
            for (int li = 0; li < 2; ++li) {
                const int lvl = l0 + li;
                if (wl[li] == 0.0 || lvl >= T.levels) continue;
                const int W = T.width[lvl], H = T.height[lvl];
                const Ewa e = ewa_setup(x, y, du0, dv0, du1, dv1, W, H);
                if (!e.ok) continue;
                double S = 0.0, mb[7] = {0, 0, 0, 0, 0, 0, 0}, ma[3] = {0, 0, 0}, mm[3] = {0, 0, 0};
                for (int t = e.t0; t <= e.t1; ++t)
                    for (int si = e.s0; si <= e.s1; ++si) {
                        const double w = ewa_weight(e, si, t);
                        if (!(w > 0.0)) continue;
                        S += w;
                        const Mat m = fetch(T, lvl, wrapi(si, W, T.address), wrapi(t, H, T.address), &rd);
                        if (mode == M_NTAP_BEFORE) {
                            for (int c = 0; c < 3; ++c) mb[c] += w * m.rho[c];
                            mb[3] += w * m.rough;
                            mb[4] += w * m.n.x; mb[5] += w * m.n.y; mb[6] += w * m.n.z;
                        } else {
                            double o[3];
                            shade(smode, m, o);
                            for (int c = 0; c < 3; ++c) { ma[c] += w * o[c]; mm[c] += std::fabs(w * o[c]); }
                        }
                    }
                if (!(S > 0.0)) continue;
                const double k = wl[li] / S;
                if (mode == M_NTAP_BEFORE) {
                    for (int c = 0; c < 3; ++c) fm.rho[c] += k * mb[c];
                    fm.rough += k * mb[3];
                    fm.n.x += k * mb[4]; fm.n.y += k * mb[5]; fm.n.z += k * mb[6];
                } else {
                    for (int c = 0; c < 3; ++c) { fsum[c] += k * ma[c]; mag[c] += k * mm[c]; }
                }
            }
            if (mode == M_NTAP_BEFORE) {
                const double ln = std::sqrt(dot(fm.n, fm.n));
                fm.n = ln > 0 ? V3{fm.n.x / ln, fm.n.y / ln, fm.n.z / ln} : V3{0, 0, 1};
                shade(smode, fm, est);
                for (int c = 0; c < 3; ++c) mag[c] += std::fabs(est[c]);
            } else {
                for (int c = 0; c < 3; ++c) est[c] = fsum[c];
            }
        }
        for (int c = 0; c < 3; ++c) acc[c] += est[c];
    }
    for (int c = 0; c < 3; ++c) O.rgb[q * 3 + c] = acc[c] / (double)spp;
    if (O.mag) for (int c = 0; c < 3; ++c) O.mag[q * 3 + c] = mag[c] / (double)spp;
    if (O.rdist) O.rdist[q] = rd;
    if (O.bdist) O.bdist[q] = bd;
}

// ------------------------------------------------------------------ Gaussian filters and FIS
// Sec. 4.2 "Filter Importance Sampling" and the supplement's Gaussian listings.
//   F_GAUSS      the Gaussian exp(-d^2 / (2 sigma^2)) at texel centres, normalised.
//                STOCHASTIC: filter reservoir sampling over the listing's 4 x 4 window (offsets
//                -1..2 from floor(p)), taken as separable CDF picks (the weights factor per
//                axis; the same distribution as the listing's 16-tap reservoir); the estimate is
//                the picked texel's shade.  N-tap: the window |i - p| <= ceil(5 sigma) + 1.
//   F_GAUSS_BOX  the Gaussian convolved with the unit box, per axis
//                Phi((i + 1/2 - p) / sigma) - Phi((i - 1/2 - p) / sigma): the filter that FIS with
//                a nearest lookup realises.  N-tap only.
//   F_FIS_*      FIS (STOCHASTIC only): a continuous offset o in texels, then the nearest texel
//                floor(x W + o).  LINEAR: o = u - 1/2 (box, hence the tent); BSPLINE: o = u1 + u2
//                + u3 - 3/2 (the quadratic B-spline, hence the cubic one, by the Cox-de Boor
//                recursion); GAUSS: o = sigma * Box-Muller(1 - u_a, u_b) (1 - u keeps the log
//                finite when u = 0).
// Decisions are FP32 in a fixed order (the Box-Muller transcendentals as double, rounded to
// float); bdist reports the distance of each decision to its FP64 boundary (for FIS, of the
// sample position to a texel edge, in texels).
double phi64(double z) { return 0.5 * std::erfc(-z / std::sqrt(2.0)); }

void gauss_weights32(float t, float inv_s2, float w[4]) {
    for (int k = 0; k < 4; ++k) {
        const float d = t - (float)(k - 1);
        w[k] = std::exp((-0.5f * (d * d)) * inv_s2);
    }
}

void run_query_gauss(const Tex& T, const Queries& Q, uint64_t q, uint64_t id, int filter, int mode, int smode,
                     uint32_t spp, uint64_t seed, uint32_t flags, float sigma, float lam32, double lam64, Out& O) {
    const int l0 = (int)std::floor(lam32);
    const float fr = lam32 - (float)l0;
    const double fr64 = lam64 - std::floor(lam64);
    const float inv_s2 = 1.0f / (sigma * sigma);
    const double sg = (double)sigma;
    double bd = 1e30;
    if (lam64 > 0.0 && lam64 < T.levels - 1) bd = std::fabs(lam64 - std::nearbyint(lam64));
    int kside = 1;
    if (flags & FLAG_STRATIFIED) kside = (int)std::lround(std::sqrt((double)spp));
    double acc[3] = {0, 0, 0}, mag[3] = {0, 0, 0};
    double rd = 1.0;
    for (uint32_t s = 0; s < spp; ++s) {
        uint32_t r0[4], r1[4];
        draw(seed, id, s, 0, r0);
        draw(seed, id, s, 1, r1);
        float a[5], b[5];
        uniforms5(r0, a);
        uniforms5(r1, b);
        float x = Q.u[q], y = Q.v[q];
        if (Q.dudx) {
            float jx, jy;
            if (flags & FLAG_STRATIFIED) {
                jx = ((float)(s % kside) + 0.5f) / (float)kside - 0.5f;
                jy = ((float)(s / kside) + 0.5f) / (float)kside - 0.5f;
            } else {
                jx = a[0] - 0.5f;
                jy = a[1] - 0.5f;
            }
            x = std::fmaf(jy, Q.dudy[q], std::fmaf(jx, Q.dudx[q], x));
            y = std::fmaf(jy, Q.dvdy[q], std::fmaf(jx, Q.dvdx[q], y));
        }
        uint32_t* pk = O.picks ? O.picks + (q * spp + s) * 2 : nullptr;
        uint32_t* pk64 = O.picks64 ? O.picks64 + (q * spp + s) * 2 : nullptr;
        if (pk) pk[0] = pk[1] = NO_PICK;
        if (pk64) pk64[0] = pk64[1] = NO_PICK;
        double est[3] = {0, 0, 0};
        if (mode == M_STOCHASTIC) {
            const int lvl = std::min(l0 + ((a[2] < fr) ? 1 : 0), T.levels - 1);
            if (lam64 > 0.0 && lam64 < T.levels - 1) bd = std::min(bd, std::fabs((double)a[2] - fr64));
            const int W = T.width[lvl], H = T.height[lvl];
            int ix, iy;
            if (filter == F_GAUSS) {
                const Axis ax = axis_at(x, W), ay = axis_at(y, H);
                float wx[4], wy[4];
                gauss_weights32(ax.t, inv_s2, wx);
                gauss_weights32(ay.t, inv_s2, wy);
                double wx64[4], wy64[4];
                for (int k = 0; k < 4; ++k) {
                    const double dx = ax.pos - (double)(ax.i0 - 1 + k), dy = ay.pos - (double)(ay.i0 - 1 + k);
                    wx64[k] = std::exp(-0.5 * dx * dx / (sg * sg));
                    wy64[k] = std::exp(-0.5 * dy * dy / (sg * sg));
                }
                const int kx = pick32(wx, 4, a[3], 0, nullptr), ky = pick32(wy, 4, a[4], 0, nullptr);
                pick64(wx64, 4, a[3], 0, &bd);
                pick64(wy64, 4, a[4], 0, &bd);
                ix = ax.i0 - 1 + kx;
                iy = ay.i0 - 1 + ky;
            } else {
                float ox, oy;
                double ox64, oy64;
                if (filter == F_FIS_LINEAR) {
                    ox = a[3] - 0.5f; oy = a[4] - 0.5f;
                    ox64 = (double)a[3] - 0.5; oy64 = (double)a[4] - 0.5;
                } else if (filter == F_FIS_BSPLINE) {
                    ox = ((a[3] + b[0]) + b[1]) - 1.5f;
                    oy = ((a[4] + b[2]) + b[3]) - 1.5f;
                    ox64 = ((double)a[3] + b[0] + b[1]) - 1.5;
                    oy64 = ((double)a[4] + b[2] + b[3]) - 1.5;
                } else {
                    const double pi = 3.14159265358979323846;
                    const float lg = (float)std::log((double)(1.0f - a[3]));
                    const float r = std::sqrt(-2.0f * lg);
                    const float c = (float)std::cos(2.0 * pi * (double)a[4]), sn = (float)std::sin(2.0 * pi * (double)a[4]);
                    ox = sigma * (r * c);
                    oy = sigma * (r * sn);
                    const double r64 = std::sqrt(-2.0 * std::log(1.0 - (double)a[3]));
                    ox64 = sg * r64 * std::cos(2.0 * pi * (double)a[4]);
                    oy64 = sg * r64 * std::sin(2.0 * pi * (double)a[4]);
                }
                const float sx = std::fmaf(x, (float)W, ox), sy = std::fmaf(y, (float)H, oy);
                ix = (int)std::floor(sx);
                iy = (int)std::floor(sy);
                const double sx64 = (double)x * W + ox64, sy64 = (double)y * H + oy64;
                bd = std::min(bd, std::min(std::fabs(sx64 - std::nearbyint(sx64)), std::fabs(sy64 - std::nearbyint(sy64))));
            }
            const int wx_ = wrapi(ix, W, T.address), wy_ = wrapi(iy, H, T.address);
            double o[3];
            shade(smode, fetch(T, lvl, wx_, wy_, &rd), o);
            for (int c = 0; c < 3; ++c) { est[c] = o[c]; mag[c] += std::fabs(o[c]); }
            if (pk) pk[0] = pack2d(lvl, wx_, wy_);
            if (pk64) pk64[0] = pack2d(lvl, wx_, wy_);
        } else {
            // N-tap: the window around p on both levels, each axis normalised
            const double wl[2] = {1.0 - (double)fr, (double)fr};
            const int R = (int)std::ceil(5.0 * sg) + 1;
            Mat fm{}; fm.n = {0, 0, 0};
            double fsum[3] = {0, 0, 0};
            for (int li = 0; li < 2; ++li) {
                const int lvl = l0 + li;
                if (wl[li] == 0.0 || lvl >= T.levels) continue;
                const int W = T.width[lvl], H = T.height[lvl];
                const Axis ax = axis_at(x, W), ay = axis_at(y, H);
                std::vector<double> wx(2 * R + 2), wy(2 * R + 2);
                double sx = 0, sy = 0;
                for (int k = 0; k < 2 * R + 2; ++k) {
                    const double dx = (double)(ax.i0 - R + k) - ax.pos, dy = (double)(ay.i0 - R + k) - ay.pos;
                    if (filter == F_GAUSS) {
                        wx[k] = std::exp(-0.5 * dx * dx / (sg * sg));
                        wy[k] = std::exp(-0.5 * dy * dy / (sg * sg));
                    } else {
                        wx[k] = phi64((dx + 0.5) / sg) - phi64((dx - 0.5) / sg);
                        wy[k] = phi64((dy + 0.5) / sg) - phi64((dy - 0.5) / sg);
                    }
                    sx += wx[k]; sy += wy[k];
                }
                for (int j = 0; j < 2 * R + 2; ++j)
                    for (int i = 0; i < 2 * R + 2; ++i) {
                        const double w = wl[li] * (wx[i] / sx) * (wy[j] / sy);
                        if (w == 0.0) continue;
                        const Mat m = fetch(T, lvl, wrapi(ax.i0 - R + i, W, T.address), wrapi(ay.i0 - R + j, H, T.address), &rd);
                        if (mode == M_NTAP_BEFORE) {
                            for (int c = 0; c < 3; ++c) fm.rho[c] += w * m.rho[c];
                            fm.rough += w * m.rough;
                            fm.n.x += w * m.n.x; fm.n.y += w * m.n.y; fm.n.z += w * m.n.z;
                        } else {
                            double o[3];
                            shade(smode, m, o);
                            for (int c = 0; c < 3; ++c) { fsum[c] += w * o[c]; mag[c] += std::fabs(w * o[c]); }
                        }
                    }
            }
            if (mode == M_NTAP_BEFORE) {
                const double ln = std::sqrt(dot(fm.n, fm.n));
                fm.n = ln > 0 ? V3{fm.n.x / ln, fm.n.y / ln, fm.n.z / ln} : V3{0, 0, 1};
                shade(smode, fm, est);
                for (int c = 0; c < 3; ++c) mag[c] += std::fabs(est[c]);
            } else {
                for (int c = 0; c < 3; ++c) est[c] = fsum[c];
            }
        }
        for (int c = 0; c < 3; ++c) acc[c] += est[c];
    }
    for (int c = 0; c < 3; ++c) O.rgb[q * 3 + c] = acc[c] / (double)spp;
    if (O.mag) for (int c = 0; c < 3; ++c) O.mag[q * 3 + c] = mag[c] / (double)spp;
    if (O.rdist) O.rdist[q] = rd;
    if (O.bdist) O.bdist[q] = bd;
}

// The same decisions as the FP64 estimate, taken in FP32 the way a float implementation
// takes them (fmaf weights, float CDF sums and compares): diagnostics only.  pk[0] is the
// positive (or only) pick, pk[1] the negative pick of positivization.
void picks_fp32(const Tex& T, int filter, int mode, uint32_t flags, float x, float y, int l0, float fr,
                const float a[5], const float b[5], uint32_t* pk) {
    const int nt = ntaps(filter), ft = first_tap(filter);
    const float xl = a[2];
    float ru = a[2];
    int lvl = l0 + ((xl < fr) ? 1 : 0);
    if (flags & FLAG_REUSE) { float r2; lvl = l0 + level_reuse(xl, fr, &r2); ru = r2; }
    lvl = std::min(lvl, T.levels - 1);
    const int W = T.width[lvl], H = T.height[lvl];
    const Axis ax = axis_at(x, W), ay = axis_at(y, H);
    float wx[4], wy[4];
    pick_weights32(filter, ax.t, wx);
    pick_weights32(filter, ay.t, wy);
    auto pack = [&](int kx, int ky) {
        return pack2d(lvl, wrapi(ax.i0 + ft + kx, W, T.address), wrapi(ay.i0 + ft + ky, H, T.address));
    };
    if (mode == M_STOCHASTIC) {
        int kx, ky;
        if (flags & FLAG_REUSE) {
            float uy, dummy;
            kx = pick32_reuse(wx, nt, ru, &uy);
            ky = pick32_reuse(wy, nt, uy, &dummy);
        } else {
            kx = pick32(wx, nt, a[3], 0, nullptr);
            ky = pick32(wy, nt, a[4], 0, nullptr);
        }
        pk[0] = pack(kx, ky);
        return;
    }
    float Px, Nx, Py, Ny;
    pick32(wx, nt, 0.0f, +1, &Px); pick32(wx, nt, 0.0f, -1, &Nx);
    pick32(wy, nt, 0.0f, +1, &Py); pick32(wy, nt, 0.0f, -1, &Ny);
    const float Wp = std::fmaf(Nx, Ny, Px * Py);
    const float Wn = std::fmaf(Nx, Py, Px * Ny);
    const int cp = (b[0] * Wp < Px * Py) ? +1 : -1;
    pk[0] = pack(pick32(wx, nt, a[3], cp, nullptr), pick32(wy, nt, a[4], cp, nullptr));
    if (Wn > 0.0f) {
        const int cn = (b[3] * Wn < Px * Ny) ? +1 : -1;
        pk[1] = pack(pick32(wx, nt, b[1], cn, nullptr), pick32(wy, nt, b[2], -cn, nullptr));
    }
}

// keep (nullable, [spp]): samples with keep[s] == 0 add nothing (and report no picks) but
// still count in the mean; the triplanar blend uses it to give each plane its own samples.
void run_query(const Tex& T, const Queries& Q, uint64_t q, uint64_t id, int filter, int mode, int smode,
               uint32_t spp, uint64_t seed, uint32_t flags, float sigma, Out& O, const uint8_t* keep = nullptr) {
    float lam32; double lam64;
    lod(T, Q, q, &lam32, &lam64);
    if (flags & FLAG_LOD0) { lam32 = 0.0f; lam64 = 0.0; }   // finest level only (no MIP prefiltering)
    if (filter >= F_GAUSS) {
        run_query_gauss(T, Q, q, id, filter, mode, smode, spp, seed, flags, sigma, lam32, lam64, O);
        return;
    }
    if (filter == F_EWA) {
        double bd0 = 1e30;
        if (lam64 > 0.0 && lam64 < T.levels - 1) bd0 = std::fabs(lam64 - std::nearbyint(lam64));
        run_query_ewa(T, Q, q, id, mode, smode, spp, seed, lam32, lam64, bd0, O);
        return;
    }
    int l0 = (int)std::floor(lam32);
    float fr = lam32 - (float)l0;
    int l0_64 = (int)std::floor(lam64);
    double fr64 = lam64 - l0_64;
    double bd = 1e30;
    if (lam64 > 0.0 && lam64 < T.levels - 1) bd = std::min(bd, std::fabs(lam64 - std::nearbyint(lam64)));
    int nt = ntaps(filter), ft = first_tap(filter);
    bool sgn = signed_filter(filter);
    double acc[3] = {0, 0, 0}, mag[3] = {0, 0, 0};
    double rd = 1.0;
    int kside = 1;
    if (flags & FLAG_STRATIFIED) { kside = (int)std::lround(std::sqrt((double)spp)); }

    for (uint32_t s = 0; s < spp; ++s) {
        // stream 0: (jitter x, jitter y, level, pick x, pick y); stream 1 (positivization):
        // (positive class, negative pick x, negative pick y, negative class, -)
        uint32_t r0[4], r1[4];
        draw(seed, id, s, 0, r0);
        draw(seed, id, s, 1, r1);
        float a[5], b[5];
        uniforms5(r0, a);
        uniforms5(r1, b);
        if (flags & FLAG_LATTICE) {
            // pick uniforms (level, pick x/y, class and negative picks) from a shifted
            // lattice across the samples; the jitter stays independent per sample
            uint32_t z0[4], z1[4], f0[5], f1[5];
            draw(seed, id, 0xFFFFFFFFu, 0, z0);
            draw(seed, id, 0xFFFFFFFFu, 1, z1);
            ints5(z0, f0);
            ints5(z1, f1);
            for (int k = 2; k < 5; ++k) a[k] = lattice(f0[k], s, spp, 24);
            for (int k = 0; k < 4; ++k) b[k] = lattice(f1[k], s, spp, 24);
        }
        // screen-space jitter inside the pixel footprint (FP32, fixed order)
        float x = Q.u[q], y = Q.v[q];
        if (Q.dudx) {
            float jx, jy;
            if (flags & FLAG_STRATIFIED) {
                jx = ((float)(s % kside) + 0.5f) / (float)kside - 0.5f;
                jy = ((float)(s / kside) + 0.5f) / (float)kside - 0.5f;
            } else {
                jx = a[0] - 0.5f;
                jy = a[1] - 0.5f;
            }
            x = std::fmaf(jy, Q.dudy[q], std::fmaf(jx, Q.dudx[q], x));
            y = std::fmaf(jy, Q.dvdy[q], std::fmaf(jx, Q.dvdx[q], y));
        }
        uint32_t* pk = O.picks ? O.picks + (q * spp + s) * 2 : nullptr;
        uint32_t* pk64 = O.picks64 ? O.picks64 + (q * spp + s) * 2 : nullptr;
        if (pk) pk[0] = pk[1] = NO_PICK;
        if (pk64) pk64[0] = pk64[1] = NO_PICK;
        if (keep && !keep[s]) continue;
        double est[3] = {0, 0, 0};

        if (mode == M_NTAP_BEFORE || mode == M_NTAP_AFTER) {
            // exact sum over both MIP levels (FP64 lambda) and the full 2-D tap grid, FP64 weights
            double wl[2] = {1.0 - fr64, fr64};
            Mat fm{}; fm.n = {0, 0, 0};
            double fsum[3] = {0, 0, 0};
            for (int li = 0; li < 2; ++li) {
                int lvl = l0_64 + li;
                if (wl[li] == 0.0 || lvl >= T.levels) continue;
                int W = T.width[lvl], H = T.height[lvl];
                Axis ax = axis_at(x, W), ay = axis_at(y, H);
                for (int j = 0; j < nt; ++j) {
                    int iy = ay.i0 + ft + j;
                    double wy = kernel64(filter, ay.pos - (double)iy);
                    for (int i = 0; i < nt; ++i) {
                        int ix = ax.i0 + ft + i;
                        double w = wl[li] * kernel64(filter, ax.pos - (double)ix) * wy;
                        if (w == 0.0) continue;
                        Mat m = fetch(T, lvl, wrapi(ix, W, T.address), wrapi(iy, H, T.address), &rd);
                        if (mode == M_NTAP_BEFORE) {
                            for (int c = 0; c < 3; ++c) fm.rho[c] += w * m.rho[c];
                            fm.rough += w * m.rough;
                            fm.n.x += w * m.n.x; fm.n.y += w * m.n.y; fm.n.z += w * m.n.z;
                        } else {
                            double o[3];
                            shade(smode, m, o);
                            for (int c = 0; c < 3; ++c) { fsum[c] += w * o[c]; mag[c] += std::fabs(w * o[c]); }
                        }
                    }
                }
            }
            if (mode == M_NTAP_BEFORE) {
                double ln = std::sqrt(dot(fm.n, fm.n));
                fm.n = ln > 0 ? V3{fm.n.x / ln, fm.n.y / ln, fm.n.z / ln} : V3{0, 0, 1};
                shade(smode, fm, est);
                for (int c = 0; c < 3; ++c) mag[c] += std::fabs(est[c]);
            } else {
                for (int c = 0; c < 3; ++c) est[c] = fsum[c];
            }
        } else {
            // Stochastic estimate (Eq. stochastic filtering; positivization, Sec. 2.2).  The
            // FP64 decisions define it: the level floor(lambda) + [xi < frac(lambda)] (the
            // stochastic lerp), then per axis the first tap whose normalised |w| prefix
            // exceeds the uniform, all from FP64 weights at the exact texel position.  The
            // same decisions taken in FP32 (float weights and CDF) are reported as `picks`,
            // for diagnostics only; the estimate never depends on them.
            const int L = T.levels;
            const float xl = a[2];
            // FLAG_REUSE: the level's uniform, remapped into the chosen interval, drives the
            // next decision; `scale` maps a distance in the remapped uniform back to the
            // original one, so `bd` stays a distance of the drawn uniform to a boundary
            double ru64 = xl, scale = 1.0;
            int lvl64;
            if (flags & FLAG_REUSE) {
                const bool up = (double)xl < fr64;
                lvl64 = l0_64 + (up ? 1 : 0);
                ru64 = up ? (double)xl / fr64 : ((double)xl - fr64) / (1.0 - fr64);
                scale = up ? fr64 : 1.0 - fr64;
            } else {
                lvl64 = l0_64 + (((double)xl < fr64) ? 1 : 0);
            }
            if (lam64 > 0.0 && lam64 < L - 1) bd = std::min(bd, std::fabs((double)xl - fr64));
            lvl64 = std::min(lvl64, L - 1);
            const int W = T.width[lvl64], H = T.height[lvl64];
            const Axis ax = axis_at(x, W), ay = axis_at(y, H);
            double wx64[4], wy64[4];
            for (int k = 0; k < nt; ++k) {
                wx64[k] = kernel64(filter, ax.pos - (double)(ax.i0 + ft + k));
                wy64[k] = kernel64(filter, ay.pos - (double)(ay.i0 + ft + k));
            }
            auto texel = [&](int kx, int ky) {
                return std::make_pair(wrapi(ax.i0 + ft + kx, W, T.address), wrapi(ay.i0 + ft + ky, H, T.address));
            };
            auto value = [&](std::pair<int, int> t, double o[3]) { shade(smode, fetch(T, lvl64, t.first, t.second, &rd), o); };
            if (mode == M_STOCHASTIC) {
                int kx, ky;
                if (flags & FLAG_REUSE) {
                    double s1, s2, r1, r2;
                    kx = pick64_reuse(wx64, nt, ru64, &r1, &s1, scale, &bd);
                    ky = pick64_reuse(wy64, nt, r1, &r2, &s2, scale * s1, &bd);
                } else {
                    kx = pick64(wx64, nt, a[3], 0, &bd);
                    ky = pick64(wy64, nt, a[4], 0, &bd);
                }
                const auto t = texel(kx, ky);
                double o[3];
                value(t, o);
                double Wt = 1.0;     // W = sum |w| with the picked tap's sign (Eq. stochastic-sum)
                if (sgn) {
                    double sx = 0, sy = 0;
                    for (int k = 0; k < nt; ++k) { sx += std::fabs(wx64[k]); sy += std::fabs(wy64[k]); }
                    Wt = sx * sy * ((wx64[kx] < 0) != (wy64[ky] < 0) ? -1.0 : 1.0);
                }
                for (int c = 0; c < 3; ++c) { est[c] = Wt * o[c]; mag[c] += std::fabs(est[c]); }
                if (pk64) pk64[0] = pack2d(lvl64, t.first, t.second);
            } else {   // positivization: one sample from each sign set (Sec. 2.2)
                double Px = 0, Nx = 0, Py = 0, Ny = 0;
                for (int k = 0; k < nt; ++k) {
                    (wx64[k] > 0 ? Px : Nx) += std::fabs(wx64[k]);
                    (wy64[k] > 0 ? Py : Ny) += std::fabs(wy64[k]);
                }
                const double Wp = Px * Py + Nx * Ny, Wn = Px * Ny + Nx * Py;
                // positive set: class (+,+) with probability Px Py / W+, else (-,-)
                const double xc = b[0];
                const int cp = (xc < Px * Py / Wp) ? +1 : -1;
                if (Nx * Ny > 0) bd = std::min(bd, std::fabs(xc - Px * Py / Wp));
                const auto tp = texel(pick64(wx64, nt, a[3], cp, &bd), pick64(wy64, nt, a[4], cp, &bd));
                double o[3];
                value(tp, o);
                for (int c = 0; c < 3; ++c) { est[c] = Wp * o[c]; mag[c] += std::fabs(est[c]); }
                if (pk64) pk64[0] = pack2d(lvl64, tp.first, tp.second);
                // negative set: class (+,-) with probability Px Ny / W-, else (-,+)
                if (Wn > 0) {
                    const double xn = b[3];
                    const int cn = (xn < Px * Ny / Wn) ? +1 : -1;
                    if (Px * Ny > 0 && Nx * Py > 0) bd = std::min(bd, std::fabs(xn - Px * Ny / Wn));
                    const auto tn = texel(pick64(wx64, nt, b[1], cn, &bd), pick64(wy64, nt, b[2], -cn, &bd));
                    value(tn, o);
                    for (int c = 0; c < 3; ++c) { est[c] -= Wn * o[c]; mag[c] += std::fabs(Wn * o[c]); }
                    if (pk64) pk64[1] = pack2d(lvl64, tn.first, tn.second);
                }
            }
            if (pk) picks_fp32(T, filter, mode, flags, x, y, l0, fr, a, b, pk);
        }
        for (int c = 0; c < 3; ++c) acc[c] += est[c];
    }
    for (int c = 0; c < 3; ++c) O.rgb[q * 3 + c] = acc[c] / (double)spp;
    if (O.mag) for (int c = 0; c < 3; ++c) O.mag[q * 3 + c] = mag[c] / (double)spp;
    if (O.rdist) O.rdist[q] = rd;
    if (O.bdist) O.bdist[q] = bd;
}

// ------------------------------------------------------------------ triplanar mapping
// Sec. 5 "Triplanar mapping" and Sec. 4.4 (material graphs): the lookups at the surface point
// projected along x, y and z are blended with weights b_i = |n_i|^4 / sum_j |n_j|^4.  The
// blend is a weighted sum of three values, so Eq. stochastic-sum applies to it.
//   plane i reads texture i at (u, v) = scale * (P_y, P_z), (P_x, P_z), (P_x, P_y) for
//   i = 0, 1, 2; the derivatives of P project the same way; each plane's lookup is run_query
//   on that 2-D query with the query's own id (so every plane sees the same uniforms);
//   blend FULL: sum_i b_i L_i over the planes with b_i > 0; filter-before blends the planes'
//   filtered materials (both levels, all taps) and shades once;
//   blend STOCHASTIC: sample s looks up one plane, drawn ~ b from the fifth uniform of
//   stream 1 (on the lattice with FLAG_LATTICE in the stochastic modes), weight 1.
// FP32: the plane coordinates and derivatives (one product each), the weights n_i^2 squared,
// their sum and the plane pick; FP64: the blend values b_i.  A normal whose FP32 weights
// all vanish takes plane 2 alone.
struct TriQueries {
    uint64_t n;
    const float *px, *py, *pz, *nx, *ny, *nz;
    const float *dxx, *dxy, *dxz, *dyx, *dyy, *dyz;   // dP/dx, dP/dy (all or none)
};

struct PlaneQuery { float u, v, d[4]; };

PlaneQuery plane_query(const TriQueries& Q, uint64_t q, int i, float scale) {
    const float P[3] = {Q.px[q], Q.py[q], Q.pz[q]};
    const int a = i == 0 ? 1 : 0, b = i == 2 ? 1 : 2;
    PlaneQuery p{P[a] * scale, P[b] * scale, {0.0f, 0.0f, 0.0f, 0.0f}};
    if (Q.dxx) {
        const float dx[3] = {Q.dxx[q], Q.dxy[q], Q.dxz[q]}, dy[3] = {Q.dyx[q], Q.dyy[q], Q.dyz[q]};
        p.d[0] = dx[a] * scale; p.d[1] = dx[b] * scale;
        p.d[2] = dy[a] * scale; p.d[3] = dy[b] * scale;
    }
    return p;
}

// the filter-before sum of one plane at (x, y): every tap of levels floor(lambda) and
// floor(lambda) + 1 (FP64 lambda) with FP64 weights, scaled by wb, added into fm
void ntap_material(const Tex& T, float x, float y, double lam64, int filter, double wb, Mat& fm, double* rd) {
    const int l0 = (int)std::floor(lam64);
    const double fr = lam64 - (double)l0;
    const double wl[2] = {1.0 - fr, fr};
    const int nt = ntaps(filter), ft = first_tap(filter);
    for (int li = 0; li < 2; ++li) {
        const int lvl = l0 + li;
        if (wl[li] == 0.0 || lvl >= T.levels) continue;
        const int W = T.width[lvl], H = T.height[lvl];
        const Axis ax = axis_at(x, W), ay = axis_at(y, H);
        for (int j = 0; j < nt; ++j) {
            const int iy = ay.i0 + ft + j;
            const double wy = kernel64(filter, ay.pos - (double)iy);
            for (int i = 0; i < nt; ++i) {
                const int ix = ax.i0 + ft + i;
                const double w = wb * wl[li] * kernel64(filter, ax.pos - (double)ix) * wy;
                if (w == 0.0) continue;
                const Mat m = fetch(T, lvl, wrapi(ix, W, T.address), wrapi(iy, H, T.address), rd);
                for (int c = 0; c < 3; ++c) fm.rho[c] += w * m.rho[c];
                fm.rough += w * m.rough;
                fm.n.x += w * m.n.x; fm.n.y += w * m.n.y; fm.n.z += w * m.n.z;
            }
        }
    }
}

void run_query_triplanar(const Tex* const T[3], const TriQueries& TQ, uint64_t q, uint64_t id, float scale,
                         int filter, int mode, int blend, int smode, uint32_t spp, uint64_t seed, uint32_t flags,
                         Out& O) {
    const float nrm[3] = {TQ.nx[q], TQ.ny[q], TQ.nz[q]};
    float w32[3];
    double b64[3], W64 = 0.0;
    for (int i = 0; i < 3; ++i) {
        const float a2 = nrm[i] * nrm[i];
        w32[i] = a2 * a2;
        const double d = (double)nrm[i];
        W64 += d * d * d * d;
    }
    const float W32 = (w32[0] + w32[1]) + w32[2];
    for (int i = 0; i < 3; ++i) {
        const double d = (double)nrm[i];
        b64[i] = W32 > 0.0f ? (w32[i] > 0.0f ? d * d * d * d / W64 : 0.0) : (i == 2 ? 1.0 : 0.0);
    }
    PlaneQuery pq[3];
    for (int i = 0; i < 3; ++i) pq[i] = plane_query(TQ, q, i, scale);
    const bool has_d = TQ.dxx != nullptr;
    auto plane_queries = [&](int i) {
        return Queries{1, &pq[i].u, &pq[i].v, has_d ? &pq[i].d[0] : nullptr, has_d ? &pq[i].d[1] : nullptr,
                       has_d ? &pq[i].d[2] : nullptr, has_d ? &pq[i].d[3] : nullptr};
    };
    double acc[3] = {0, 0, 0}, mag[3] = {0, 0, 0}, bd = 1e30, rd = 1.0;
    uint32_t* pk = O.picks ? O.picks + q * spp * 6 : nullptr;
    uint32_t* pk64 = O.picks64 ? O.picks64 + q * spp * 6 : nullptr;
    if (pk) for (uint32_t k = 0; k < spp * 6; ++k) pk[k] = NO_PICK;
    if (pk64) for (uint32_t k = 0; k < spp * 6; ++k) pk64[k] = NO_PICK;

    if (blend == 0 && mode == M_NTAP_BEFORE) {
        // one filtered material over all planes and taps, shaded once per sample
        int kside = 1;
        if (flags & FLAG_STRATIFIED) kside = (int)std::lround(std::sqrt((double)spp));
        for (uint32_t s = 0; s < spp; ++s) {
            uint32_t r0[4];
            draw(seed, id, s, 0, r0);
            float a[5];
            uniforms5(r0, a);
            Mat fm{}; fm.n = {0, 0, 0};
            for (int i = 0; i < 3; ++i) {
                if (b64[i] == 0.0) continue;
                const Queries Qi = plane_queries(i);
                float lam32; double lam64;
                lod(*T[i], Qi, 0, &lam32, &lam64);
                if (flags & FLAG_LOD0) { lam32 = 0.0f; lam64 = 0.0; }
                if (lam64 > 0.0 && lam64 < T[i]->levels - 1) bd = std::min(bd, std::fabs(lam64 - std::nearbyint(lam64)));
                float x = pq[i].u, y = pq[i].v;
                if (has_d) {   // the screen-space jitter of run_query, in this plane's footprint
                    float jx, jy;
                    if (flags & FLAG_STRATIFIED) {
                        jx = ((float)(s % kside) + 0.5f) / (float)kside - 0.5f;
                        jy = ((float)(s / kside) + 0.5f) / (float)kside - 0.5f;
                    } else {
                        jx = a[0] - 0.5f;
                        jy = a[1] - 0.5f;
                    }
                    x = std::fmaf(jy, pq[i].d[2], std::fmaf(jx, pq[i].d[0], x));
                    y = std::fmaf(jy, pq[i].d[3], std::fmaf(jx, pq[i].d[1], y));
                }
                ntap_material(*T[i], x, y, lam64, filter, b64[i], fm, &rd);
            }
            const double ln = std::sqrt(dot(fm.n, fm.n));
            fm.n = ln > 0 ? V3{fm.n.x / ln, fm.n.y / ln, fm.n.z / ln} : V3{0, 0, 1};
            double est[3];
            shade(smode, fm, est);
            for (int c = 0; c < 3; ++c) { acc[c] += est[c]; mag[c] += std::fabs(est[c]); }
        }
        for (int c = 0; c < 3; ++c) O.rgb[q * 3 + c] = acc[c] / (double)spp;
        if (O.mag) for (int c = 0; c < 3; ++c) O.mag[q * 3 + c] = mag[c] / (double)spp;
        if (O.bdist) O.bdist[q] = bd;
        if (O.rdist) O.rdist[q] = rd;
        return;
    }

    // which samples each plane evaluates, and with what blend factor
    std::vector<uint8_t> keep(3 * (size_t)spp, 1);
    double factor[3] = {b64[0], b64[1], b64[2]};
    if (blend == 1) {
        const bool lat = (mode == M_STOCHASTIC || mode == M_POSITIVIZED) && (flags & FLAG_LATTICE);
        uint32_t f1[5] = {0, 0, 0, 0, 0};
        if (lat) { uint32_t z1[4]; draw(seed, id, 0xFFFFFFFFu, 1, z1); ints5(z1, f1); }
        for (uint32_t s = 0; s < spp; ++s) {
            uint32_t r1[4];
            draw(seed, id, s, 1, r1);
            float b[5];
            uniforms5(r1, b);
            if (lat) b[4] = lattice(f1[4], s, spp, 24);
            int plane = 2;
            if (W32 > 0.0f) {
                plane = pick32(w32, 3, b[4], 0, nullptr);
                pick64(b64, 3, (double)b[4], 0, &bd);
            }
            for (int i = 0; i < 3; ++i) keep[i * (size_t)spp + s] = plane == i;
        }
        factor[0] = factor[1] = factor[2] = 1.0;
    }
    std::vector<uint32_t> lp(2 * (size_t)spp), lp64(2 * (size_t)spp);
    for (int i = 0; i < 3; ++i) {
        if (blend == 0 && b64[i] == 0.0) continue;
        bool any = false;
        for (uint32_t s = 0; s < spp; ++s) any |= keep[i * (size_t)spp + s] != 0;
        if (!any) continue;
        const Queries Qi = plane_queries(i);
        double rgb1[3], mag1[3], bd1 = 1e30, rd1 = 1.0;
        Out O1{rgb1, pk ? lp.data() : nullptr, pk64 ? lp64.data() : nullptr, &bd1, mag1, &rd1};
        run_query(*T[i], Qi, 0, id, filter, mode, smode, spp, seed, flags, 0.0f, O1,
                  blend == 1 ? &keep[i * (size_t)spp] : nullptr);
        for (int c = 0; c < 3; ++c) { acc[c] += factor[i] * rgb1[c]; mag[c] += factor[i] * mag1[c]; }
        bd = std::min(bd, bd1);
        rd = std::min(rd, rd1);
        for (uint32_t s = 0; s < spp; ++s)
            for (int k = 0; k < 2; ++k) {
                if (pk) pk[(s * 3 + i) * 2 + k] = lp[s * 2 + k];
                if (pk64) pk64[(s * 3 + i) * 2 + k] = lp64[s * 2 + k];
            }
    }
    for (int c = 0; c < 3; ++c) O.rgb[q * 3 + c] = acc[c];
    if (O.mag) for (int c = 0; c < 3; ++c) O.mag[q * 3 + c] = mag[c];
    if (O.bdist) O.bdist[q] = bd;
    if (O.rdist) O.rdist[q] = rd;
}

// ------------------------------------------------------------------ volume march
// FP16 -> double, exact (IEEE 754 binary16)
double half_to_double(uint16_t h) {
    int e = (h >> 10) & 0x1F, m = h & 0x3FF;
    double s = (h & 0x8000) ? -1.0 : 1.0;
    if (e == 0) return s * std::ldexp((double)m, -24);
    if (e == 31) return m ? NAN : s * INFINITY;
    return s * std::ldexp((double)(m | 0x400), e - 25);
}

struct Vol { int nx, ny, nz; const uint16_t* data; float sigma_scale; };

inline uint32_t pack3d(int x, int y, int z) { return ((uint32_t)z << 20) | ((uint32_t)y << 10) | (uint32_t)x; }

// One pixel sample of the 128-step (or `steps`) ray march through the unit cube with
// per-step transmittance exp(-sigma dt) (Sec. 5 "Offline rendering": density filtered by
// trilinear or tricubic B-spline, stochastically or with all taps).
double march_sample(const Vol& V, const float* cam, uint32_t W, uint32_t H, uint32_t steps,
                    int filter, int mode, uint64_t seed, uint32_t flags, uint32_t spp,
                    uint64_t pix, uint32_t s, uint32_t* picks, uint32_t* picks64, double* bd) {
    uint32_t px = (uint32_t)(pix % W), py = (uint32_t)(pix / W);
    float jx, jy;
    if (flags & FLAG_STRATIFIED) {
        int k = (int)std::lround(std::sqrt((double)spp));
        jx = ((float)(s % k) + 0.5f) / (float)k;
        jy = ((float)(s / k) + 0.5f) / (float)k;
    } else {
        uint32_t r[4];
        draw(seed, pix, s, 0, r);
        jx = unif(r[0]); jy = unif(r[1]);
    }
    float sx = std::fmaf((float)px + jx, 2.0f / (float)W, -1.0f);
    float sy = std::fmaf(-((float)py + jy), 2.0f / (float)H, 1.0f);
    const float *e = cam, *f = cam + 3, *r = cam + 6, *u = cam + 9;
    float d[3];
    for (int a = 0; a < 3; ++a) d[a] = std::fmaf(sy, u[a], std::fmaf(sx, r[a], f[a]));
    float l2 = std::fmaf(d[2], d[2], std::fmaf(d[1], d[1], d[0] * d[0]));
    float inv = 1.0f / std::sqrt(l2);
    for (int a = 0; a < 3; ++a) d[a] = d[a] * inv;
    float tmin = 0.0f, tmax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0f) {
            float id = 1.0f / d[a];
            float t1 = (0.0f - e[a]) * id, t2 = (1.0f - e[a]) * id;
            tmin = std::fmax(tmin, std::fmin(t1, t2));
            tmax = std::fmin(tmax, std::fmax(t1, t2));
        } else if (e[a] < 0.0f || e[a] > 1.0f) {
            tmax = -1.0f;
        }
    }
    if (!(tmin < tmax)) {
        if (picks) for (uint32_t k = 0; k < steps; ++k) picks[k] = NO_PICK;
        if (picks64) for (uint32_t k = 0; k < steps; ++k) picks64[k] = NO_PICK;
        return 1.0;
    }
    float dt = (tmax - tmin) / (float)steps;
    const int res[3] = {V.nx, V.ny, V.nz};
    int nt = ntaps(filter), ft = first_tap(filter);
    double sig = (double)V.sigma_scale, dt64 = (double)dt;
    double sum_sigma = 0.0, prod = 1.0;
    for (uint32_t k = 0; k < steps; ++k) {
        float tk = std::fmaf((float)k + 0.5f, dt, tmin);
        Axis ax[3];
        for (int a = 0; a < 3; ++a) {
            float p = std::fmaf(tk, d[a], e[a]);
            ax[a] = axis_at(p, res[a]);
        }
        auto vox = [&](int ix, int iy, int iz) {
            ix = wrapi(ix, V.nx, ADDR_CLAMP); iy = wrapi(iy, V.ny, ADDR_CLAMP); iz = wrapi(iz, V.nz, ADDR_CLAMP);
            return half_to_double(V.data[((size_t)iz * V.ny + iy) * V.nx + ix]);
        };
        if (mode == M_STOCHASTIC) {
            // steps 2p and 2p+1 share stream p+1: six 21-bit uniforms, three per step
            uint32_t rr[4];
            float u6[6];
            if (flags & FLAG_LATTICE) {
                uint32_t f6[6];
                draw(seed, pix, 0xFFFFFFFFu, (k >> 1) + 1, rr);
                ints6(rr, f6);
                for (int j = 0; j < 6; ++j) u6[j] = lattice(f6[j], s, spp, 21);
            } else {
                draw(seed, pix, s, (k >> 1) + 1, rr);
                uniforms6(rr, u6);
            }
            const float* uk = u6 + 3 * (k & 1);
            // per axis the first tap whose normalised FP64 |w| prefix exceeds the uniform
            // (these decisions define the estimate); FLAG_REUSE: x, y, z from one uniform,
            // remapped into each chosen interval.  The FP32 decisions go to `picks` only.
            int kk[3], kk64[3];
            float ru = uk[0];
            double ru64 = uk[0], scale = 1.0;
            for (int a = 0; a < 3; ++a) {
                float w[4];
                double w64[4];
                pick_weights32(filter, ax[a].t, w);
                for (int j = 0; j < nt; ++j) w64[j] = kernel64(filter, ax[a].pos - (double)(ax[a].i0 + ft + j));
                if (flags & FLAG_REUSE) {
                    kk[a] = pick32_reuse(w, nt, ru, &ru);
                    double r, width;
                    kk64[a] = pick64_reuse(w64, nt, ru64, &r, &width, scale, bd);
                    ru64 = r;
                    scale *= width;
                } else {
                    kk[a] = pick32(w, nt, uk[a], 0, nullptr);
                    kk64[a] = pick64(w64, nt, uk[a], 0, bd);
                }
            }
            auto packv = [&](const int* kq) {
                return pack3d(wrapi(ax[0].i0 + ft + kq[0], V.nx, ADDR_CLAMP), wrapi(ax[1].i0 + ft + kq[1], V.ny, ADDR_CLAMP),
                              wrapi(ax[2].i0 + ft + kq[2], V.nz, ADDR_CLAMP));
            };
            sum_sigma += sig * vox(ax[0].i0 + ft + kk64[0], ax[1].i0 + ft + kk64[1], ax[2].i0 + ft + kk64[2]);
            if (picks) picks[k] = packv(kk);
            if (picks64) picks64[k] = packv(kk64);
        } else {
            double fsig = 0.0, favg = 0.0;
            for (int c = 0; c < nt; ++c) {
                int iz = ax[2].i0 + ft + c;
                double wz = kernel64(filter, ax[2].pos - (double)iz);
                for (int b = 0; b < nt; ++b) {
                    int iy = ax[1].i0 + ft + b;
                    double wy = kernel64(filter, ax[1].pos - (double)iy);
                    for (int a = 0; a < nt; ++a) {
                        int ix = ax[0].i0 + ft + a;
                        double w = kernel64(filter, ax[0].pos - (double)ix) * wy * wz;
                        if (w == 0.0) continue;
                        double sv = sig * vox(ix, iy, iz);
                        fsig += w * sv;
                        favg += w * std::exp(-sv * dt64);
                    }
                }
            }
            sum_sigma += fsig;
            prod *= favg;
            if (picks) picks[k] = NO_PICK;
            if (picks64) picks64[k] = NO_PICK;
        }
    }
    if (mode == M_NTAP_AFTER) return prod;
    return std::exp(-sum_sigma * dt64);
}

template <class F>
void parallel_for(uint64_t n, int nthreads, F fn) {
    if (nthreads <= 1 || n < 64) { for (uint64_t i = 0; i < n; ++i) fn(i); return; }
    std::vector<std::thread> th;
    uint64_t chunk = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        th.emplace_back([=]() { for (uint64_t i = b; i < e; ++i) fn(i); });
    }
    for (auto& x : th) x.join();
}

}  // namespace

// ===================================================================== C entry points
extern "C" {

typedef struct {
    int format, levels, address;
    int width[16], height[16];
    const void* data[16];
    const uint8_t* normal[16];
} orc_texture;

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

double orc_kernel(int filter, double d) { return kernel64(filter, d); }
double orc_kernel_bc(double B, double Cc, double d) { return k_bc(B, Cc, d); }
double orc_kernel_keys(double a, double d) { return k_keys(a, d); }

int orc_weights32(int filter, float t, float* w) { return weights32(filter, t, w); }

// EWA pieces for the pins: the weight table, and the weights of an ellipse's bounding box
// (box[4] = s0, s1, t0, t1; w gets (s1-s0+1)*(t1-t0+1) weights, t outer), or -1 if the box
// holds more than cap weights
// raw DCT decode of one channel word at (x, y) in its 8 x 8 block (for the pins)
double orc_dct_texel(uint32_t word, int x, int y) { return dct_texel(word, x, y); }

void orc_ewa_table(float* out) { std::memcpy(out, ewa_table(), sizeof(float) * EWA_LUT_N); }
int orc_ewa_box(float x, float y, float dudx, float dvdx, float dudy, float dvdy, int W, int H, int* box,
                float* w, int cap) {
    const Ewa e = ewa_setup(x, y, dudx, dvdx, dudy, dvdy, W, H);
    if (!e.ok) return -2;
    box[0] = e.s0; box[1] = e.s1; box[2] = e.t0; box[3] = e.t1;
    const long n = (long)(e.s1 - e.s0 + 1) * (long)(e.t1 - e.t0 + 1);
    if (n > cap) return -1;
    int k = 0;
    for (int t = e.t0; t <= e.t1; ++t)
        for (int s = e.s0; s <= e.s1; ++s) w[k++] = ewa_weight(e, s, t);
    return k;
}

// FP32 CDF pick (cls 0 = all taps, +1 positive taps, -1 negative taps)
int orc_pick32(const float* w, int n, float xi, int cls) { return pick32(w, n, xi, cls, nullptr); }
int orc_pick32_reuse(const float* w, int n, float xi, float* remapped) { return pick32_reuse(w, n, xi, remapped); }

// FP64 CDF pick over an arbitrary array of up to 64 non-negative weights
int orc_pick_array(const double* w, int n, double xi) {
    double S = 0; for (int k = 0; k < n; ++k) S += std::fabs(w[k]);
    double acc = 0;
    for (int k = 0; k < n; ++k) { acc += std::fabs(w[k]); if (xi < acc / S) return k; }
    return n - 1;
}

// general GGX + Lambert evaluation (f_hat including the cosine factor)
void orc_ggx_eval(const double* n, const double* l, const double* v, double alpha,
                  const double* rho, double F0, double* out) {
    ggx_eval({n[0], n[1], n[2]}, {l[0], l[1], l[2]}, {v[0], v[1], v[2]}, alpha, rho, F0, out);
}
double orc_ggx_D(double alpha, double nh) { double a2 = alpha * alpha; return ggx_D(a2, nh, 1.0 - nh * nh); }
double orc_smith_lambda(double alpha, double tan2) { return smith_lambda(alpha * alpha, tan2); }

// the fixed-direction shade used by the texture path: rho[n*3], rough[n], nrm[n*3]
void orc_shade_batch(uint64_t n, int smode, const double* rho, const double* rough,
                     const double* nrm, double* out) {
    for (uint64_t i = 0; i < n; ++i) {
        Mat m;
        for (int c = 0; c < 3; ++c) m.rho[c] = rho[3 * i + c];
        m.rough = rough[i];
        m.n = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        shade(smode, m, out + 3 * i);
    }
}

// decoded texel (for tests): rho[3], rough, n[3]
void orc_fetch(const orc_texture* t, int lvl, int ix, int iy, double* out7) {
    Tex T; std::memcpy(&T, t, sizeof(Tex));
    Mat m = fetch(T, lvl, ix, iy);
    out7[0] = m.rho[0]; out7[1] = m.rho[1]; out7[2] = m.rho[2]; out7[3] = m.rough;
    out7[4] = m.n.x; out7[5] = m.n.y; out7[6] = m.n.z;
}

int orc_filter_shade(const orc_texture* tex, uint64_t n, const float* u, const float* v,
                     const float* dudx, const float* dvdx, const float* dudy, const float* dvdy,
                     const uint64_t* ids, int filter, int mode, int smode, uint32_t spp, uint64_t seed,
                     uint32_t flags, double* rgb, uint32_t* picks, uint32_t* picks64, double* bdist,
                     double* mag, double* rdist, int nthreads, float sigma) {
    if (!tex || !u || !v || !rgb || spp == 0 || filter < 0 || filter > 9 || mode < 0 || mode > 3) return 1;
    if (filter >= F_GAUSS) {
        if (!(sigma > 0.0f) || sigma > 8.0f || mode == M_POSITIVIZED) return 1;
        if (flags & ~(uint32_t)(FLAG_STRATIFIED | FLAG_LOD0)) return 1;
        if (filter == F_GAUSS_BOX && mode == M_STOCHASTIC) return 1;
        if (filter >= F_FIS_LINEAR && mode != M_STOCHASTIC) return 1;
    }
    if (tex->levels < 1 || tex->levels > 16) return 1;
    if ((mode == M_POSITIVIZED) && !signed_filter(filter)) return 1;
    if (filter == F_EWA && (flags & ~(uint32_t)FLAG_LOD0)) return 1;   // EWA: no jitter, lattice or reuse
    if ((flags & FLAG_REUSE) && mode == M_POSITIVIZED) return 1;
    if (flags & FLAG_STRATIFIED) {
        long k = std::lround(std::sqrt((double)spp));
        if ((uint32_t)(k * k) != spp) return 1;
    }
    Tex T; std::memcpy(&T, tex, sizeof(Tex));
    Queries Q{n, u, v, dudx, dvdx, dudy, dvdy};
    Out O{rgb, picks, picks64, bdist, mag, rdist};
    parallel_for(n, nthreads, [&](uint64_t q) {
        run_query(T, Q, q, ids ? ids[q] : q, filter, mode, smode, spp, seed, flags, sigma, O);
    });
    return 0;
}

// triplanar filter + shade: tex points at three textures (planes 0, 1, 2); rgb[n*3];
// picks / picks64 (nullable) [n][spp][3][2]
int orc_triplanar_shade(const orc_texture* tex, uint64_t n, const float* px, const float* py, const float* pz,
                        const float* nx, const float* ny, const float* nz, const float* dxx, const float* dxy,
                        const float* dxz, const float* dyx, const float* dyy, const float* dyz,
                        const uint64_t* ids, float scale, int filter, int mode, int blend, int smode, uint32_t spp,
                        uint64_t seed, uint32_t flags, double* rgb, uint32_t* picks, uint32_t* picks64,
                        double* bdist, double* mag, int nthreads) {
    if (!tex || !px || !py || !pz || !nx || !ny || !nz || !rgb || spp == 0) return 1;
    if (filter < 0 || filter > 3 || mode < 0 || mode > 3 || (blend != 0 && blend != 1)) return 1;
    if (mode == M_POSITIVIZED && !signed_filter(filter)) return 1;
    if (flags & ~(uint32_t)(FLAG_STRATIFIED | FLAG_LATTICE | FLAG_LOD0)) return 1;
    if (!std::isfinite(scale) || scale == 0.0f) return 1;
    if (flags & FLAG_STRATIFIED) {
        long k = std::lround(std::sqrt((double)spp));
        if ((uint32_t)(k * k) != spp) return 1;
    }
    Tex T[3];
    const Tex* Tp[3];
    for (int i = 0; i < 3; ++i) {
        if (tex[i].levels < 1 || tex[i].levels > 16) return 1;
        std::memcpy(&T[i], &tex[i], sizeof(Tex));
        Tp[i] = &T[i];
    }
    TriQueries Q{n, px, py, pz, nx, ny, nz, dxx, dxy, dxz, dyx, dyy, dyz};
    Out O{rgb, picks, picks64, bdist, mag, nullptr};
    parallel_for(n, nthreads, [&](uint64_t q) {
        run_query_triplanar(Tp, Q, q, ids ? ids[q] : q, scale, filter, mode, blend, smode, spp, seed, flags, O);
    });
    return 0;
}

int orc_march(int nx, int ny, int nz, const uint16_t* data, float sigma_scale, const float* cam,
              uint32_t W, uint32_t H, uint32_t steps, int filter, int mode, uint32_t spp,
              uint64_t seed, uint32_t flags, uint64_t pix_begin, uint64_t pix_count,
              const uint64_t* pix_ids, double* T, uint32_t* picks, uint32_t* picks64, double* bdist,
              int nthreads) {
    if (!data || !cam || !T || spp == 0 || steps == 0) return 1;
    if (!(filter == F_LINEAR || filter == F_BSPLINE) || mode == M_POSITIVIZED) return 1;
    Vol V{nx, ny, nz, data, sigma_scale};
    parallel_for(pix_count, nthreads, [&](uint64_t i) {
        uint64_t pix = pix_ids ? pix_ids[i] : pix_begin + i;
        double acc = 0.0, bd = 1e30;
        for (uint32_t s = 0; s < spp; ++s) {
            uint32_t* pk = picks ? picks + (i * spp + s) * steps : nullptr;
            uint32_t* pk64 = picks64 ? picks64 + (i * spp + s) * steps : nullptr;
            acc += march_sample(V, cam, W, H, steps, filter, mode, seed, flags, spp, pix, s, pk, pk64, &bd);
        }
        T[i] = acc / spp;
        if (bdist) bdist[i] = bd;
    });
    return 0;
}

}  // extern "C"
