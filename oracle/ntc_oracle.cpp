// FP64 oracle of the learned (neural-texture) form -- TEST INFRASTRUCTURE ONLY.
//
// The paper names neural texture compression among the representations whose per-texel
// decode is expensive, so that stochastic filtering's single decode per lookup pays off
// (Sec. 1, Sec. 2 related work, Sec. 5 compressed-texture results); it specifies no
// network.  The network restated here:
//   * features: 4 latent grids (8 channels each) sampled bilinearly (wrap) at the centre
//     of the decoded texel, concatenated to 32 values, rounded to BF16; the bilinear step
//     is evaluated in FP32 with a fixed operation order because it decides the BF16 code;
//   * MLP 32 -> 64 (ReLU) -> 64 (ReLU) -> 8, BF16 weights, FP32 biases; the hidden
//     activations are rounded to BF16 (they are the operands of the next BF16 GEMM);
//   * MSE loss on the 8 target channels (byte/255), analytic backward, Adam (Kingma & Ba
//     2015, with bias correction).
// Codecs: FP16, BF16 and FP8 E4M3 (OCP 8-bit float: bias 7, no infinities, max 448,
// saturating) by round-to-nearest-even on the real line.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <vector>

#include "oracle_internal.h"

namespace orc {

// ------------------------------------------------------------------ codecs
// round v to the nearest value with p significant bits and exponent >= emin (ties to
// even); |result| > vmax -> saturate (sat) or +-inf
double round_float(double v, int p, int emin, double vmax, bool sat) {
    if (v == 0.0 || std::isnan(v)) return v;
    int e;
    std::frexp(std::fabs(v), &e);       // |v| = m 2^e, m in [0.5, 1)
    e = std::max(e - 1, emin);          // exponent of the leading bit, clamped to the subnormal range
    double quantum = std::ldexp(1.0, e - (p - 1));
    double q = v / quantum;
    double r = std::floor(q);
    double d = q - r;
    if (d > 0.5 || (d == 0.5 && std::fmod(r, 2.0) != 0.0)) r += 1.0;
    double out = r * quantum;
    if (std::fabs(out) > vmax) out = sat ? std::copysign(vmax, v) : std::copysign(INFINITY, v);
    return out;
}
double to_bf16(double v) { return round_float(v, 8, -126, 3.3895313892515355e38, false); }
double to_fp16(double v) { return round_float(v, 11, -14, 65504.0, false); }
double to_e4m3(double v) { return round_float(v, 4, -6, 448.0, true); }

double half_value(uint16_t h) {
    int e = (h >> 10) & 0x1F, m = h & 0x3FF;
    double s = (h & 0x8000) ? -1.0 : 1.0;
    if (e == 0) return s * std::ldexp((double)m, -24);
    if (e == 31) return m ? NAN : s * INFINITY;
    return s * std::ldexp((double)(m | 0x400), e - 25);
}
double e4m3_value(uint8_t c) {
    int s = c >> 7, e = (c >> 3) & 0xF, m = c & 7;
    if (e == 15 && m == 7) return NAN;
    double v = e == 0 ? std::ldexp((double)m, -9) : std::ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

// ------------------------------------------------------------------ features
double NeuralTex::latent(int g, int x, int y, int c) const {
    size_t o = ((size_t)y * res[g] + x) * 8 + c;
    if (latent_fmt == 0) return half_value(((const uint16_t*)grid[g])[o]);
    if (latent_fmt == 1) return e4m3_value(((const uint8_t*)grid[g])[o]) * (double)scale[g];
    return ((const float*)grid[g])[o];
}

static int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

struct Tap { int x, y; float w; };

// bilinear taps of grid g at the centre of texel (ix, iy) of the tex_res^2 texture (FP32)
static void taps(const NeuralTex& N, int ix, int iy, int g, Tap t[4]) {
    float s = (float)N.res[g] / (float)N.tex_res;
    float px = std::fmaf((float)ix + 0.5f, s, -0.5f);
    float py = std::fmaf((float)iy + 0.5f, s, -0.5f);
    float fx = std::floor(px), fy = std::floor(py);
    float tx = px - fx, ty = py - fy, ux = 1.0f - tx, uy = 1.0f - ty;
    int x0 = wrapi((int)fx, N.res[g]), y0 = wrapi((int)fy, N.res[g]);
    int x1 = wrapi((int)fx + 1, N.res[g]), y1 = wrapi((int)fy + 1, N.res[g]);
    t[0] = {x0, y0, ux * uy}; t[1] = {x1, y0, tx * uy};
    t[2] = {x0, y1, ux * ty}; t[3] = {x1, y1, tx * ty};
}

// interpolated latent features, FP32 fixed order with fused multiply-adds:
// fma(w11, d, fma(w01, c, fma(w10, b, w00 a)))
void features32(const NeuralTex& N, int ix, int iy, float f[32]) {
    for (int g = 0; g < 4; ++g) {
        Tap t[4];
        taps(N, ix, iy, g, t);
        for (int c = 0; c < 8; ++c) {
            float v = t[0].w * (float)N.latent(g, t[0].x, t[0].y, c);
            for (int k = 1; k < 4; ++k) v = std::fmaf(t[k].w, (float)N.latent(g, t[k].x, t[k].y, c), v);
            f[8 * g + c] = v;
        }
    }
}

// Margin of the BF16 rounding of a pre-activation v = b + sum_i w_i x_i: the distance of
// v to the nearest BF16 rounding midpoint divided by S = |b| + sum_i |w_i x_i|.  An FP32
// accumulation of the same (exact) products in another order differs from v by about
// sqrt(K) 2^-24 S, so a margin below a few times that may round the other way.
static double bf16_margin(double v, double S) {
    if (v == 0.0 || S == 0.0) return 1.0;
    int e;
    std::frexp(std::fabs(v), &e);
    double quantum = std::ldexp(1.0, (e - 1) - 7);
    double q = std::fabs(v) / quantum;
    double frac = q - std::floor(q);
    return std::fabs(frac - 0.5) * quantum / S;
}

void mlp_forward(const Mlp& M, const double x[32], double h1[64], double h2[64], double y[8],
                 double* rdist, bool round_hidden) {
    for (int o = 0; o < 64; ++o) {
        double z = M.b1[o], S = std::fabs(M.b1[o]);
        for (int i = 0; i < 32; ++i) { z += M.W1[o * 32 + i] * x[i]; S += std::fabs(M.W1[o * 32 + i] * x[i]); }
        if (rdist && z > 0) *rdist = std::min(*rdist, bf16_margin(z, S) / std::sqrt(33.0));
        h1[o] = z > 0 ? (round_hidden ? to_bf16(z) : z) : 0.0;
    }
    for (int o = 0; o < 64; ++o) {
        double z = M.b2[o], S = std::fabs(M.b2[o]);
        for (int i = 0; i < 64; ++i) { z += M.W2[o * 64 + i] * h1[i]; S += std::fabs(M.W2[o * 64 + i] * h1[i]); }
        if (rdist && z > 0) *rdist = std::min(*rdist, bf16_margin(z, S) / std::sqrt(65.0));
        h2[o] = z > 0 ? (round_hidden ? to_bf16(z) : z) : 0.0;
    }
    for (int o = 0; o < 8; ++o) {
        double z = M.b3[o];
        for (int i = 0; i < 64; ++i) z += M.W3[o * 64 + i] * h2[i];
        y[o] = z;
    }
}

void neural_decode(const NeuralTex& N, int ix, int iy, double y[8], double* rdist) {
    float f[32];
    features32(N, ix, iy, f);
    double x[32], h1[64], h2[64];
    for (int i = 0; i < 32; ++i) x[i] = to_bf16(f[i]);   // same FP32 features on both sides
    mlp_forward(*N.mlp, x, h1, h2, y, rdist, true);
}

// The network's exact value at texel (ix, iy): FP64 bilinear features of the latents as
// stored in N (the FP32 master values for the exact form) and an FP64 forward pass of the
// MLP in N with no BF16 rounding anywhere -- the reference the quantised inference forms
// (BF16 weights and activations, FP16 or FP8 latents) are measured against.
void neural_decode_exact(const NeuralTex& N, int ix, int iy, double y[8]) {
    double x[32];
    for (int g = 0; g < 4; ++g) {
        const double s = (double)N.res[g] / (double)N.tex_res;
        const double px = ((double)ix + 0.5) * s - 0.5, py = ((double)iy + 0.5) * s - 0.5;
        const double fx = std::floor(px), fy = std::floor(py), tx = px - fx, ty = py - fy;
        const int x0 = wrapi((int)fx, N.res[g]), y0 = wrapi((int)fy, N.res[g]);
        const int x1 = wrapi((int)fx + 1, N.res[g]), y1 = wrapi((int)fy + 1, N.res[g]);
        for (int c = 0; c < 8; ++c)
            x[8 * g + c] = (1 - tx) * (1 - ty) * N.latent(g, x0, y0, c) + tx * (1 - ty) * N.latent(g, x1, y0, c) +
                           (1 - tx) * ty * N.latent(g, x0, y1, c) + tx * ty * N.latent(g, x1, y1, c);
    }
    double h1[64], h2[64];
    mlp_forward(*N.mlp, x, h1, h2, y, nullptr, false);
}

}  // namespace orc

// ===================================================================== C entry points
extern "C" {

double orc_round_bf16(double v) { return orc::to_bf16(v); }
double orc_round_fp16(double v) { return orc::to_fp16(v); }
double orc_round_e4m3(double v) { return orc::to_e4m3(v); }
double orc_e4m3_value(uint8_t c) { return orc::e4m3_value(c); }

void orc_ntc_features(const orc::NeuralTex* N, uint64_t n, const int32_t* ix, const int32_t* iy, float* out) {
    for (uint64_t i = 0; i < n; ++i) orc::features32(*N, ix[i], iy[i], out + 32 * i);
}

// decode n texels: y[n*8] (FP64); rdist[n] (nullable): the smallest BF16 rounding margin of
// the hidden activations, |v - midpoint| / (sqrt(K) sum|w x|)
void orc_ntc_decode(const orc::NeuralTex* N, uint64_t n, const int32_t* ix, const int32_t* iy,
                    double* y, double* rdist) {
    for (uint64_t i = 0; i < n; ++i) {
        double rd = 1.0;
        orc::neural_decode(*N, ix[i], iy[i], y + 8 * i, &rd);
        if (rdist) rdist[i] = rd;
    }
}

// exact FP64 decode of n texels (see neural_decode_exact): y[n*8]
void orc_ntc_decode_exact(const orc::NeuralTex* N, uint64_t n, const int32_t* ix, const int32_t* iy, double* y) {
    for (uint64_t i = 0; i < n; ++i) orc::neural_decode_exact(*N, ix[i], iy[i], y + 8 * i);
}

// Loss and gradients of one training batch.  Latents are FP32 master values (latent_fmt
// 2).  round_bf16 selects where BF16 operands stand in for exact values:
//   0: nowhere (exact FP64 forward and backward);
//   1: the forward GEMMs' operands (features, FP32 master weights, hidden activations);
//   2: as 1, and also the backward GEMMs' operands dy, dh2 (.) [h2 > 0] and
//      dh1 (.) [h1 > 0], each rounded once where it is formed, then used for the weight,
//      bias and input gradients alike (a BF16 tensor-core backward).
// Every rounding is treated as identity when differentiating.  targets: tex_res^2 x 8
// bytes.  Gradients are ACCUMULATED into the double arrays.
double orc_ntc_loss_grad(const orc::NeuralTex* N, const float* W1, const float* b1, const float* W2,
                         const float* b2, const float* W3, const float* b3, const uint8_t* targets,
                         uint64_t n, const int32_t* ix, const int32_t* iy, int round_bf16,
                         double* dW1, double* db1, double* dW2, double* db2, double* dW3, double* db3,
                         double* const* dlat) {
    std::vector<double> w1(64 * 32), w2(64 * 64), w3(8 * 64);
    auto rnd = [&](double v) { return round_bf16 ? orc::to_bf16(v) : v; };
    auto rndb = [&](double v) { return round_bf16 >= 2 ? orc::to_bf16(v) : v; };
    for (int i = 0; i < 64 * 32; ++i) w1[i] = rnd(W1[i]);
    for (int i = 0; i < 64 * 64; ++i) w2[i] = rnd(W2[i]);
    for (int i = 0; i < 8 * 64; ++i) w3[i] = rnd(W3[i]);
    std::vector<double> vb1(b1, b1 + 64), vb2(b2, b2 + 64), vb3(b3, b3 + 8);
    orc::Mlp M{w1.data(), vb1.data(), w2.data(), vb2.data(), w3.data(), vb3.data()};
    double loss = 0.0;
    const double inv = 1.0 / (8.0 * (double)n);
    for (uint64_t s = 0; s < n; ++s) {
        float f[32];
        orc::features32(*N, ix[s], iy[s], f);
        double x[32], h1[64], h2[64], y[8];
        for (int i = 0; i < 32; ++i) x[i] = round_bf16 ? orc::to_bf16(f[i]) : (double)f[i];
        orc::mlp_forward(M, x, h1, h2, y, nullptr, round_bf16 != 0);
        const uint8_t* t = targets + ((size_t)iy[s] * N->tex_res + ix[s]) * 8;
        double dy[8], dh2[64], dh1[64], dx[32];
        for (int o = 0; o < 8; ++o) {
            double e = y[o] - t[o] / 255.0;
            loss += e * e * inv;
            dy[o] = rndb(2.0 * e * inv);
            db3[o] += dy[o];
            for (int i = 0; i < 64; ++i) dW3[o * 64 + i] += dy[o] * h2[i];
        }
        for (int i = 0; i < 64; ++i) {
            double a = 0.0;
            for (int o = 0; o < 8; ++o) a += w3[o * 64 + i] * dy[o];
            dh2[i] = h2[i] > 0 ? rndb(a) : 0.0;
            db2[i] += dh2[i];
        }
        for (int o = 0; o < 64; ++o)
            for (int i = 0; i < 64; ++i) dW2[o * 64 + i] += dh2[o] * h1[i];
        for (int i = 0; i < 64; ++i) {
            double a = 0.0;
            for (int o = 0; o < 64; ++o) a += w2[o * 64 + i] * dh2[o];
            dh1[i] = h1[i] > 0 ? rndb(a) : 0.0;
            db1[i] += dh1[i];
        }
        for (int o = 0; o < 64; ++o)
            for (int i = 0; i < 32; ++i) dW1[o * 32 + i] += dh1[o] * x[i];
        for (int i = 0; i < 32; ++i) {
            double a = 0.0;
            for (int o = 0; o < 64; ++o) a += w1[o * 32 + i] * dh1[o];
            dx[i] = a;
        }
        for (int g = 0; g < 4; ++g) {
            orc::Tap tp[4];
            orc::taps(*N, ix[s], iy[s], g, tp);
            for (int k = 0; k < 4; ++k)
                for (int c = 0; c < 8; ++c)
                    dlat[g][((size_t)tp[k].y * N->res[g] + tp[k].x) * 8 + c] += (double)tp[k].w * dx[8 * g + c];
        }
    }
    return loss;
}

// Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
void orc_adam(uint64_t n, double* p, const double* g, double* m, double* v, int t, double lr,
              double beta1, double beta2, double eps) {
    double c1 = 1.0 - std::pow(beta1, t), c2 = 1.0 - std::pow(beta2, t);
    for (uint64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
    }
}

}  // extern "C"
