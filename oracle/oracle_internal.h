// Shared declarations between the two oracle translation units (test infrastructure).
#pragma once
#include <cstdint>

namespace orc {

struct Mlp {              // FP64 copies of the (BF16-valued) weights; row-major [out][in]
    const double *W1, *b1, *W2, *b2, *W3, *b3;
};

struct NeuralTex {
    int tex_res;          // decoded texture is tex_res x tex_res texels
    int res[4];           // latent grid resolutions
    int latent_fmt;       // 0: FP16 codes, 1: FP8 E4M3 codes x scale[g], 2: FP32 values
    const void* grid[4];  // [res][res][8] per grid
    float scale[4];
    const Mlp* mlp;
    double latent(int g, int x, int y, int c) const;
};

void neural_decode(const NeuralTex& N, int ix, int iy, double y[8], double* rdist);
double to_bf16(double v);

}  // namespace orc
