// Host check of the hoisted Philox forms used by the lookup and march kernels: PhiloxS
// (counter words fixed except the sample) and PhiloxT (fixed except the last word) must return
// exactly philox() of the same counter, and philox() must give the Random123 known answer for
// the zero counter and key.  Built with nvcc as host code; exits 0 when every check holds.
#include <cstdio>
#include <random>

#include "../../paper_2407_06107_b300/csrc/stf_device.cuh"

using namespace stf;

int main() {
    std::mt19937_64 g(7);
    long bad = 0;
    for (int it = 0; it < 200000; ++it) {
        const RoundKeys K = expand_key(g());
        uint32_t a = (uint32_t)g(), b = (uint32_t)g(), c = (uint32_t)g(), d = (uint32_t)g();
        if (it & 1) { b = 0; c &= 15; d &= 3; }     // small ids, sample and stream indices too
        const uint4 r0 = philox(a, b, c, d, K);
        const uint4 r1 = PhiloxS(a, b, d, K)(c, K);
        const uint4 r2 = PhiloxT(a, b, c, K)(d, K);
        bad += r1.x != r0.x || r1.y != r0.y || r1.z != r0.z || r1.w != r0.w;
        bad += r2.x != r0.x || r2.y != r0.y || r2.z != r0.z || r2.w != r0.w;
    }
    const RoundKeys K0 = expand_key(0);
    const uint4 z = philox(0, 0, 0, 0, K0);
    const bool kat = z.x == 0x6627e8d5u && z.y == 0xe169c58du && z.z == 0xbc57ac4cu && z.w == 0x9b00dbd8u;
    std::printf("mismatches %ld kat %d\n", bad, (int)kat);
    return (bad == 0 && kat) ? 0 : 1;
}
