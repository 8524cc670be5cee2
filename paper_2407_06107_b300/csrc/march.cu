// Volume ray march kernels (sm_103a): trilinear (8 taps) / tricubic B-spline (64 taps)
// density reconstruction, per-step transmittance exp(-sigma dt), stochastic 1-tap vs
// N-tap (Sec. 5 "Offline rendering"; FRS for the 3-D B-spline, Sec. 4.1, and the
// tricubic listing of the supplement).
//
// One thread owns one pixel and all its samples.  Ray setup and sample positions are
// FP32 with a fixed operation order (they decide which voxel is picked).  Estimators:
//   stochastic : T = exp(-dt * sigma_scale * sum_k d_pick,k), the densities summed in
//                exact 2^-24 fixed point, so one expf per ray carries the only rounding;
//   N-tap after: T = prod_k sum_i w_i exp(-sigma_i dt), an FMA-compensated product of
//                1 - sum_i w_i (1 - exp(-sigma_i dt)) (exactly 1 in empty space);
//   N-tap before: T = exp(-dt sum_k sum_i w_i sigma_i), compensated summation over k.
#include "stf_kernels.h"
#include "stf_device.cuh"

namespace stf {

__device__ __forceinline__ float vox(const MarchArgs& a, int x, int y, int z) {
    x = clamp_index(x, a.nx); y = clamp_index(y, a.ny); z = clamp_index(z, a.nz);
    return __half2float(a.vox[((size_t)z * a.ny + y) * a.nx + x]);
}

// V: the kernel variant (KV_*).  The specialised ones (no picks; no flags, or the lattice
// flag alone) run the stochastic steps in pairs, see below.
// Resident 128-thread blocks per SM the register budget is set for: 10 (<= 48 registers) for
// the specialised 1-tap marches, no bound for the others.
template <int MODE, int V>
constexpr int march_min_blocks() { return (MODE == M_STOCHASTIC && V != KV_GENERAL) ? 10 : 1; }

template <int FILTER, int MODE, int V>
__global__ void __launch_bounds__(128, march_min_blocks<MODE, V>()) k_march(MarchArgs a, RoundKeys K) {
    constexpr int NT = ntaps(FILTER), T0 = tap0(FILTER);
    const float res[3] = {(float)a.nx, (float)a.ny, (float)a.nz};
    const uint32_t flags = V == KV_GENERAL ? a.flags : variant_flags(V);
    uint32_t* const picks = V == KV_GENERAL ? a.picks : nullptr;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.pix_count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        // o: the pixel's slot in the output range.  Tiled, the 32 threads of a warp take an
        // 8 x 4 block of pixels, so their rays stay close and share the voxels' cache lines.
        uint64_t o = i;
        if (a.tiled) {
            const uint64_t tile = i >> 5;
            const uint32_t lane = (uint32_t)i & 31u, tpr = a.width >> 3;
            o = (tile / tpr * 4u + (lane >> 3)) * (uint64_t)a.width + (tile % tpr) * 8u + (lane & 7u);
        }
        const uint64_t pix = a.pix_begin + o;
        const uint32_t px = (uint32_t)(pix % a.width), py = (uint32_t)(pix / a.width);
        const uint32_t id_lo = (uint32_t)pix, id_hi = (uint32_t)(pix >> 32);
        float acc = 0.0f;
        for (uint32_t s = 0; s < a.spp; ++s) {
            uint32_t* pk = picks ? picks + (o * a.spp + s) * a.steps : nullptr;
            float jx, jy;
            if (flags & FLAG_STRATIFIED) {
                jx = __fdiv_rn(__fadd_rn((float)(s % a.kside), 0.5f), (float)a.kside);
                jy = __fdiv_rn(__fadd_rn((float)(s / a.kside), 0.5f), (float)a.kside);
            } else {
                const uint4 r = philox(id_lo, id_hi, s, 0u, K);
                jx = unif(r.x); jy = unif(r.y);
            }
            const float sx = __fmaf_rn(__fadd_rn((float)px, jx), __fdiv_rn(2.0f, (float)a.width), -1.0f);
            const float sy = __fmaf_rn(-__fadd_rn((float)py, jy), __fdiv_rn(2.0f, (float)a.height), 1.0f);
            float d[3], e[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                e[c] = a.cam[c];
                d[c] = __fmaf_rn(sy, a.cam[9 + c], __fmaf_rn(sx, a.cam[6 + c], a.cam[3 + c]));
            }
            const float l2 = __fmaf_rn(d[2], d[2], __fmaf_rn(d[1], d[1], __fmul_rn(d[0], d[0])));
            const float inv = __fdiv_rn(1.0f, __fsqrt_rn(l2));
#pragma unroll
            for (int c = 0; c < 3; ++c) d[c] = __fmul_rn(d[c], inv);
            float tmin = 0.0f, tmax = __int_as_float(0x7f800000);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (d[c] != 0.0f) {
                    const float id = __fdiv_rn(1.0f, d[c]);
                    const float t1 = __fmul_rn(__fsub_rn(0.0f, e[c]), id), t2 = __fmul_rn(__fsub_rn(1.0f, e[c]), id);
                    tmin = fmaxf(tmin, fminf(t1, t2));
                    tmax = fminf(tmax, fmaxf(t1, t2));
                } else if (e[c] < 0.0f || e[c] > 1.0f) {
                    tmax = -1.0f;
                }
            }
            if (!(tmin < tmax)) {
                acc += 1.0f;
                if (pk) for (uint32_t k = 0; k < a.steps; ++k) pk[k] = NO_PICK;
                continue;
            }
            const float dt = __fdiv_rn(__fsub_rn(tmax, tmin), (float)a.steps);
            uint64_t fixed_sum = 0;                 // stochastic: sum of d * 2^24 (exact)
            float Ssum = 0.0f, Scomp = 0.0f;        // before: compensated sum of filtered sigma/scale
            float P = 1.0f, Pe = 0.0f;              // after: compensated product
            const float sdt = a.sigma_scale * dt;
            uint4 rw = make_uint4(0u, 0u, 0u, 0u);
            const uint32_t lshift = (flags & FLAG_LATTICE) ? lattice_shift(s, a.spp, 21) : 0u;
            if constexpr (V != KV_GENERAL && MODE == M_STOCHASTIC) {
                // Steps 2p and 2p+1 take their uniforms from the same Philox call: both picks
                // are made and both voxel loads issued before either density is added, so
                // two gathers are in flight per thread.  LATTICE: the call is the per-pixel
                // offset (sample index 0xFFFFFFFF), shifted per sample.
                // kh = k + 1/2, the step's midpoint in steps, kept as an exact float; the pick
                // uniforms come pre-scaled for pick_positive_scaled
                auto voxel = [&](float kh, const float uk[3]) -> int {
                    const float tk = __fmaf_rn(kh, dt, tmin);
                    int idx[3];
                    {   // x and y in packed FP32 pairs (one rounding per lane, as axis_pos), z alone
                        const float2 p = upk2(vfma(vfma(f2(tk), f2(d[0], d[1]), f2(e[0], e[1])),
                                                   f2(res[0], res[1]), vconst<F2>(-0.5f)).v);
                        const float fx = floorf(p.x), fy = floorf(p.y);
                        const F2 t = vsub(f2(p.x, p.y), f2(fx, fy));
                        int kx, ky;
                        pick_positive2_scaled<FILTER>(t, uk[0], uk[1], &kx, &ky);
                        idx[0] = (int)fx + T0 + kx;
                        idx[1] = (int)fy + T0 + ky;
                        const AxisPos ap = axis_pos(__fmaf_rn(tk, d[2], e[2]), res[2]);
                        idx[2] = ap.i0 + T0 + pick_positive_scaled<FILTER>(ap.t, uk[2]);
                    }
                    // A sample point lies inside the box, so a picked index is in [-2, n + 1] and
                    // the bordered copy holds its clamped voxel: no clamping here.  At most
                    // 1028^2 x 1032 voxels: the offset fits 32 bits.
                    return idx[2] * a.pxy + idx[1] * a.px + idx[0];
                };
                constexpr float US = pick_scale<FILTER>();
                auto step_uniforms = [&](const uint4& rw, int odd, float u[3]) {
                    if constexpr (V == KV_LATTICE) {
                        uint32_t f[3];
                        ints3_of6(rw, odd, f);
#pragma unroll
                        for (int c = 0; c < 3; ++c) u[c] = lattice(f[c], lshift, 21, US);
                    } else {
                        uniforms3_of6(rw, odd, u, US);
                    }
                };
                const PhiloxT R(id_lo, id_hi, V == KV_LATTICE ? 0xFFFFFFFFu : s, K);
                // The sum in an accumulator of type Acc.  32 bits hold it exactly when steps x
                // (largest density) < 256, each term d 2^24 then below 2^32 / steps (a.fixed32).
                auto march = [&](auto zero) -> uint64_t {
                    using Acc = decltype(zero);
                    Acc sum = zero;
                    uint32_t k = 0;
                    float kh = 0.5f;
                    for (; k + 1 < a.steps; k += 2, kh = __fadd_rn(kh, 2.0f)) {
                        const uint4 rw = R((k >> 1) + 1u, K);
                        float u0[3], u1[3];
                        step_uniforms(rw, 0, u0);
                        step_uniforms(rw, 1, u1);
                        const int v0 = voxel(kh, u0), v1 = voxel(__fadd_rn(kh, 1.0f), u1);
                        const float d0 = __half2float(a.vpad[v0]), d1 = __half2float(a.vpad[v1]);
                        sum += (Acc)(d0 * 16777216.0f) + (Acc)(d1 * 16777216.0f);
                    }
                    if (k < a.steps) {
                        float u0[3];
                        step_uniforms(R((k >> 1) + 1u, K), 0, u0);
                        sum += (Acc)(__half2float(a.vpad[voxel(kh, u0)]) * 16777216.0f);
                    }
                    return (uint64_t)sum;
                };
                fixed_sum = a.fixed32 ? march(uint32_t{0}) : march(uint64_t{0});
            } else
            for (uint32_t k = 0; k < a.steps; ++k) {
                const float tk = __fmaf_rn(__fadd_rn((float)k, 0.5f), dt, tmin);
                AxisPos ap[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) ap[c] = axis_pos(__fmaf_rn(tk, d[c], e[c]), res[c]);
                float w[3][4];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if constexpr (MODE == M_STOCHASTIC) axis_pick_weights<FILTER>(ap[c].t, w[c]);
                    else axis_weights<FILTER>(ap[c].t, w[c]);
                }
                if (MODE == M_STOCHASTIC) {
                    // steps 2p and 2p+1 share stream p+1 (six 21-bit uniforms)
                    float uk[3];
                    if (flags & FLAG_LATTICE) {   // per-pixel offsets, shifted lattice over samples
                        if ((k & 1u) == 0u) rw = philox(id_lo, id_hi, 0xFFFFFFFFu, (k >> 1) + 1u, K);
                        uint32_t f[3];
                        ints3_of6(rw, (int)(k & 1u), f);
#pragma unroll
                        for (int c = 0; c < 3; ++c) uk[c] = lattice(f[c], lshift, 21);
                    } else {
                        if ((k & 1u) == 0u) rw = philox(id_lo, id_hi, s, (k >> 1) + 1u, K);
                        uniforms3_of6(rw, (int)(k & 1u), uk);
                    }
                    int kx, ky, kz;
                    if (flags & FLAG_REUSE) {      // x, y, z from one uniform, remapped
                        float r1, r2, r3;
                        kx = cdf_pick_reuse<NT>(w[0], uk[0], &r1);
                        ky = cdf_pick_reuse<NT>(w[1], r1, &r2);
                        kz = cdf_pick_reuse<NT>(w[2], r2, &r3);
                    } else {
                        kx = pick_positive<FILTER>(ap[0].t, uk[0]);
                        ky = pick_positive<FILTER>(ap[1].t, uk[1]);
                        kz = pick_positive<FILTER>(ap[2].t, uk[2]);
                    }
                    const int ix = clamp_index(ap[0].i0 + T0 + kx, a.nx);
                    const int iy = clamp_index(ap[1].i0 + T0 + ky, a.ny);
                    const int iz = clamp_index(ap[2].i0 + T0 + kz, a.nz);
                    const float dv = __half2float(a.vox[((size_t)iz * a.ny + iy) * a.nx + ix]);
                    fixed_sum += (uint64_t)(dv * 16777216.0f);
                    if (pk) pk[k] = ((uint32_t)iz << 20) | ((uint32_t)iy << 10) | (uint32_t)ix;
                } else {
                    float fsig = 0.0f, fab = 0.0f;   // sum w d, sum w (1 - exp(-sigma dt))
                    auto tap = [&](float ww, float dv) {
                        if (MODE == M_NTAP_BEFORE) {
                            fsig = fmaf(ww, dv, fsig);
                        } else if (dv != 0.0f) {
                            fab = fmaf(ww, -expm1f(-sdt * dv), fab);
                        }
                    };
                    const int x0 = ap[0].i0 + T0, y0 = ap[1].i0 + T0, z0 = ap[2].i0 + T0;
                    const int xa = x0 & ~3;   // 8-byte aligned start of the row segment
                    // Tricubic rows inside the volume: each row's 4 voxels come from two aligned
                    // 8-byte loads (half the load requests of 4 scalar ones; the L1 request rate
                    // bounds this kernel), realigned with funnel shifts.  Rows that need clamping
                    // take the per-voxel path.  Same voxels, same summation order.
                    const bool rows = NT == 4 && (a.nx & 3) == 0 && x0 >= 0 && xa + 8 <= a.nx && y0 >= 0 &&
                                      y0 + NT <= a.ny && z0 >= 0 && z0 + NT <= a.nz;
                    if (rows) {
                        const int o = x0 - xa;          // 0..3
                        const bool hi_pair = (o & 2) != 0, odd = (o & 1) != 0;
#pragma unroll
                        for (int cz = 0; cz < NT; ++cz) {
#pragma unroll
                            for (int cy = 0; cy < NT; ++cy) {
                                const float wyz = w[2][cz] * w[1][cy];
                                const uint2* row = reinterpret_cast<const uint2*>(
                                    a.vox + ((size_t)(z0 + cz) * a.ny + (size_t)(y0 + cy)) * a.nx + xa);
                                const uint2 lo = __ldg(row), hi = __ldg(row + 1);
                                const uint32_t q0 = hi_pair ? lo.y : lo.x, q1 = hi_pair ? hi.x : lo.y,
                                               q2 = hi_pair ? hi.y : hi.x;
                                const uint32_t p0 = odd ? __funnelshift_r(q0, q1, 16) : q0;
                                const uint32_t p1 = odd ? __funnelshift_r(q1, q2, 16) : q1;
                                const float2 f01 = __half22float2(*reinterpret_cast<const __half2*>(&p0));
                                const float2 f23 = __half22float2(*reinterpret_cast<const __half2*>(&p1));
                                tap(wyz * w[0][0], f01.x);
                                tap(wyz * w[0][1], f01.y);
                                tap(wyz * w[0][2], f23.x);
                                tap(wyz * w[0][3], f23.y);
                            }
                        }
                    } else {
#pragma unroll
                        for (int cz = 0; cz < NT; ++cz) {
#pragma unroll
                            for (int cy = 0; cy < NT; ++cy) {
                                const float wyz = w[2][cz] * w[1][cy];
#pragma unroll
                                for (int cx = 0; cx < NT; ++cx)
                                    tap(wyz * w[0][cx], vox(a, x0 + cx, y0 + cy, z0 + cz));
                            }
                        }
                    }
                    if (MODE == M_NTAP_BEFORE) {
                        const float t = Ssum + fsig;   // Neumaier compensated summation
                        Scomp += (fabsf(Ssum) >= fabsf(fsig)) ? (Ssum - t) + fsig : (fsig - t) + Ssum;
                        Ssum = t;
                    } else if (fab != 0.0f) {
                        const float f = 1.0f - fab;
                        const float p = P * f;
                        Pe = fmaf(Pe, f, fmaf(P, f, -p));   // exact error of P*f, carried
                        P = p;
                    }
                    if (pk) pk[k] = NO_PICK;
                }
            }
            float T;
            if (MODE == M_STOCHASTIC) T = expf(-sdt * ((float)fixed_sum * 5.9604644775390625e-8f));
            else if (MODE == M_NTAP_BEFORE) T = expf(-sdt * (Ssum + Scomp));
            else T = P + Pe;
            acc += T;
        }
        a.T[o] = acc / (float)a.spp;
    }
}

// ---------------------------------------------------------------- TMA-staged tricubic N-tap
// The 64-tap comparators (tricubic filter-before / filter-after) with no flags: at every
// march step the 32 rays of a warp (an 8 x 4 pixel tile) read 4 x 4 x 4 voxel windows that
// mostly overlap.  One lane copies the box that holds all of them into the warp's shared
// memory with one 3-D TMA copy (cp.async.bulk.tensor, completion on an mbarrier); the lanes
// then read their windows from there, in the same order and with the same arithmetic as
// k_march, so the results are identical.  The box is 24 x 8 x 8 voxels and starts at an x that
// is a multiple of 8 (a 16-byte boundary); a step whose windows do not fit in it, or that
// needs clamping at a face of the volume, reads from global memory as k_march does.
// Every lane of a warp runs every (sample, step) in lockstep (rays that miss the volume sit
// idle), so the box and the copy are the warp's; waits are bounded, and a copy that times out
// sets DEV_TIMEOUT and sends the rest of the warp's steps to global memory.
constexpr int SB_X = 24, SB_Y = 8, SB_Z = 8, SB_ELEMS = SB_X * SB_Y * SB_Z;
constexpr long long SB_WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* tmap, int x, int y, int z, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"((uint32_t)(SB_ELEMS * 2))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool sb_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > SB_WAIT_CYCLES) return false;
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(128) k_march_staged(MarchArgs a, const __grid_constant__ CUtensorMap tmap, RoundKeys K) {
    constexpr int NT = 4, T0 = -1;
    __shared__ __align__(128) __half box[4][SB_ELEMS];
    __shared__ __align__(8) uint64_t bar[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) mbar_init(&bar[warp], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    uint32_t phase = 0;
    bool staging = true;            // false after a copy timed out (this warp's steps then read global memory)
    const float res[3] = {(float)a.nx, (float)a.ny, (float)a.nz};
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < a.pix_count;
    uint64_t o = i;
    if (a.tiled) {
        const uint64_t tile = i >> 5;
        const uint32_t ln = (uint32_t)i & 31u, tpr = a.width >> 3;
        o = (tile / tpr * 4u + (ln >> 3)) * (uint64_t)a.width + (tile % tpr) * 8u + (ln & 7u);
    }
    const uint64_t pix = a.pix_begin + o;
    const uint32_t px = (uint32_t)(pix % a.width), py = (uint32_t)(pix / a.width);
    const uint32_t id_lo = (uint32_t)pix, id_hi = (uint32_t)(pix >> 32);
    const __half* bx = box[warp];
    float acc = 0.0f;
    for (uint32_t s = 0; s < a.spp; ++s) {
        float d[3] = {0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f};
        float tmin = 0.0f, tmax = -1.0f;
        if (valid) {
            const uint4 r = philox(id_lo, id_hi, s, 0u, K);
            const float jx = unif(r.x), jy = unif(r.y);
            const float sx = __fmaf_rn(__fadd_rn((float)px, jx), __fdiv_rn(2.0f, (float)a.width), -1.0f);
            const float sy = __fmaf_rn(-__fadd_rn((float)py, jy), __fdiv_rn(2.0f, (float)a.height), 1.0f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                e[c] = a.cam[c];
                d[c] = __fmaf_rn(sy, a.cam[9 + c], __fmaf_rn(sx, a.cam[6 + c], a.cam[3 + c]));
            }
            const float l2 = __fmaf_rn(d[2], d[2], __fmaf_rn(d[1], d[1], __fmul_rn(d[0], d[0])));
            const float inv = __fdiv_rn(1.0f, __fsqrt_rn(l2));
#pragma unroll
            for (int c = 0; c < 3; ++c) d[c] = __fmul_rn(d[c], inv);
            tmax = __int_as_float(0x7f800000);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (d[c] != 0.0f) {
                    const float id = __fdiv_rn(1.0f, d[c]);
                    const float t1 = __fmul_rn(__fsub_rn(0.0f, e[c]), id), t2 = __fmul_rn(__fsub_rn(1.0f, e[c]), id);
                    tmin = fmaxf(tmin, fminf(t1, t2));
                    tmax = fminf(tmax, fmaxf(t1, t2));
                } else if (e[c] < 0.0f || e[c] > 1.0f) {
                    tmax = -1.0f;
                }
            }
        }
        const bool hit = valid && tmin < tmax;
        if (!__any_sync(0xFFFFFFFFu, hit)) {       // the whole warp misses the volume
            if (valid) acc += 1.0f;
            continue;
        }
        const float dt = hit ? __fdiv_rn(__fsub_rn(tmax, tmin), (float)a.steps) : 0.0f;
        const float sdt = a.sigma_scale * dt;
        float Ssum = 0.0f, Scomp = 0.0f;   // before: compensated sum of filtered sigma / scale
        float P = 1.0f, Pe = 0.0f;         // after: compensated product
        for (uint32_t k = 0; k < a.steps; ++k) {
            AxisPos ap[3] = {{0, 0.0f}, {0, 0.0f}, {0, 0.0f}};
            float w[3][4];
            if (hit) {
                const float tk = __fmaf_rn(__fadd_rn((float)k, 0.5f), dt, tmin);
#pragma unroll
                for (int c = 0; c < 3; ++c) ap[c] = axis_pos(__fmaf_rn(tk, d[c], e[c]), res[c]);
#pragma unroll
                for (int c = 0; c < 3; ++c) axis_weights<F_BSPLINE>(ap[c].t, w[c]);
            }
            const int x0 = ap[0].i0 + T0, y0 = ap[1].i0 + T0, z0 = ap[2].i0 + T0;
            // the box of the warp's windows (rays that miss take no part)
            const int BIG = 1 << 30;
            const int xmn = __reduce_min_sync(0xFFFFFFFFu, hit ? x0 : BIG), xmx = __reduce_max_sync(0xFFFFFFFFu, hit ? x0 : -BIG);
            const int ymn = __reduce_min_sync(0xFFFFFFFFu, hit ? y0 : BIG), ymx = __reduce_max_sync(0xFFFFFFFFu, hit ? y0 : -BIG);
            const int zmn = __reduce_min_sync(0xFFFFFFFFu, hit ? z0 : BIG), zmx = __reduce_max_sync(0xFFFFFFFFu, hit ? z0 : -BIG);
            const int xs = xmn & ~7;
            // staged: every window inside the volume (no clamping) and inside the box, with 4
            // voxels of slack after the last window in x for the 8-byte row reads below
            bool staged = staging && xmn >= 0 && ymn >= 0 && zmn >= 0 && xmx + 8 <= a.nx && ymx + NT <= a.ny &&
                          zmx + NT <= a.nz && xmx + 8 - xs <= SB_X && ymx + NT - ymn <= SB_Y && zmx + NT - zmn <= SB_Z;
            if (staged) {
                if (lane == 0) tma_load_box(box[warp], &tmap, xs, ymn, zmn, &bar[warp]);
                const bool ok = __all_sync(0xFFFFFFFFu, sb_wait(&bar[warp], phase));
                phase ^= 1u;
                if (!ok) {
                    staging = staged = false;
                    if (lane == 0) atomicOr(a.status, DEV_TIMEOUT);
                }
            }
            if (hit) {
                float fsig = 0.0f, fab = 0.0f;   // sum w d, sum w (1 - exp(-sigma dt))
                auto tap = [&](float ww, float dv) {
                    if (MODE == M_NTAP_BEFORE) {
                        fsig = fmaf(ww, dv, fsig);
                    } else if (dv != 0.0f) {
                        fab = fmaf(ww, -expm1f(-sdt * dv), fab);
                    }
                };
                const int xa = x0 & ~3;   // 8-byte aligned start of the row segment
                const bool rows = staged || ((a.nx & 3) == 0 && x0 >= 0 && xa + 8 <= a.nx && y0 >= 0 && y0 + NT <= a.ny &&
                                             z0 >= 0 && z0 + NT <= a.nz);
                if (rows) {
                    // each row's 4 voxels from two aligned 8-byte reads, realigned with funnel shifts
                    const int off = x0 - xa;          // 0..3
                    const bool hi_pair = (off & 2) != 0, odd = (off & 1) != 0;
#pragma unroll
                    for (int cz = 0; cz < NT; ++cz) {
#pragma unroll
                        for (int cy = 0; cy < NT; ++cy) {
                            const float wyz = w[2][cz] * w[1][cy];
                            uint2 lo2, hi2;
                            if (staged) {
                                const uint2* row = reinterpret_cast<const uint2*>(
                                    bx + ((z0 + cz - zmn) * SB_Y + (y0 + cy - ymn)) * SB_X + (xa - xs));
                                lo2 = row[0]; hi2 = row[1];
                            } else {
                                const uint2* row = reinterpret_cast<const uint2*>(
                                    a.vox + ((size_t)(z0 + cz) * a.ny + (size_t)(y0 + cy)) * a.nx + xa);
                                lo2 = __ldg(row); hi2 = __ldg(row + 1);
                            }
                            const uint32_t q0 = hi_pair ? lo2.y : lo2.x, q1 = hi_pair ? hi2.x : lo2.y,
                                           q2 = hi_pair ? hi2.y : hi2.x;
                            const uint32_t p0 = odd ? __funnelshift_r(q0, q1, 16) : q0;
                            const uint32_t p1 = odd ? __funnelshift_r(q1, q2, 16) : q1;
                            const float2 f01 = __half22float2(*reinterpret_cast<const __half2*>(&p0));
                            const float2 f23 = __half22float2(*reinterpret_cast<const __half2*>(&p1));
                            tap(wyz * w[0][0], f01.x);
                            tap(wyz * w[0][1], f01.y);
                            tap(wyz * w[0][2], f23.x);
                            tap(wyz * w[0][3], f23.y);
                        }
                    }
                } else {
#pragma unroll
                    for (int cz = 0; cz < NT; ++cz) {
#pragma unroll
                        for (int cy = 0; cy < NT; ++cy) {
                            const float wyz = w[2][cz] * w[1][cy];
#pragma unroll
                            for (int cx = 0; cx < NT; ++cx) tap(wyz * w[0][cx], vox(a, x0 + cx, y0 + cy, z0 + cz));
                        }
                    }
                }
                if (MODE == M_NTAP_BEFORE) {
                    const float t = Ssum + fsig;   // Neumaier compensated summation
                    Scomp += (fabsf(Ssum) >= fabsf(fsig)) ? (Ssum - t) + fsig : (fsig - t) + Ssum;
                    Ssum = t;
                } else if (fab != 0.0f) {
                    const float f = 1.0f - fab;
                    const float p = P * f;
                    Pe = fmaf(Pe, f, fmaf(P, f, -p));   // exact error of P*f, carried
                    P = p;
                }
            }
            __syncwarp();   // every lane has read the box before the next copy overwrites it
        }
        if (hit) acc += (MODE == M_NTAP_BEFORE) ? expf(-sdt * (Ssum + Scomp)) : P + Pe;
        else if (valid) acc += 1.0f;
    }
    if (valid) a.T[o] = acc / (float)a.spp;
    if (!staging && lane == 0) {
        // a copy that timed out may still be in flight: give it one more bounded wait before the
        // block's shared memory is released
        sb_wait(&bar[warp], phase ^ 1u);
    }
}

// The volume as a 3-D FP16 tensor for the staged march: dims (nx, ny, nz), x fastest, box
// 24 x 8 x 8.  Needs 16-byte row and slice strides (nx a multiple of 8); false otherwise or if
// the driver cannot encode it.
// Largest density of a volume as FP16 bits (non-negative FP16 values order like their bit
// patterns; negative densities count as 0, NaN and infinity above every finite value).
__global__ void k_vol_max_bits(const uint16_t* __restrict__ v, uint64_t n, unsigned int* out) {
    unsigned int m = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned int b = v[i];
        m = max(m, (b & 0x8000u) ? 0u : b);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
cudaError_t launch_vol_max_bits(const void* vox, uint64_t n, unsigned int* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const uint64_t g = (n + 255) / 256;
    k_vol_max_bits<<<(int)(g < 2048 ? (g ? g : 1) : 2048), 256, 0, st>>>((const uint16_t*)vox, n, out);
    return cudaGetLastError();
}

// The clamped border copy of a volume (clamp-to-edge addressing written out): every voxel of
// the padded grid takes the voxel at its coordinates clamped to the volume.
__global__ void k_pad_volume(const __half* __restrict__ src, int nx, int ny, int nz, __half* __restrict__ dst,
                             int px, int py, int pz) {
    const uint64_t n = (uint64_t)px * py * pz;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % (uint64_t)px), y = (int)(i / (uint64_t)px % (uint64_t)py), z = (int)(i / ((uint64_t)px * py));
        const int sx = clamp_index(x - VOL_PAD, nx), sy = clamp_index(y - VOL_PAD, ny), sz = clamp_index(z - VOL_PAD, nz);
        dst[i] = src[((size_t)sz * ny + sy) * nx + sx];
    }
}
cudaError_t launch_pad_volume(const void* src, int nx, int ny, int nz, void* dst, cudaStream_t st) {
    const int px = (int)vol_pad_pitch((uint32_t)nx), py = ny + 2 * VOL_PAD, pz = nz + 2 * VOL_PAD;
    const uint64_t g = ((uint64_t)px * py * pz + 255) / 256;
    k_pad_volume<<<(int)(g < 8192 ? (g ? g : 1) : 8192), 256, 0, st>>>((const __half*)src, nx, ny, nz, (__half*)dst,
                                                                       px, py, pz);
    return cudaGetLastError();
}

bool encode_volume_tmap(CUtensorMap* out, const void* vox, int nx, int ny, int nz) {
    if (nx % 8 != 0 || nx < SB_X || ny < SB_Y || nz < SB_Z) return false;
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = reinterpret_cast<Encode>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 2, (cuuint64_t)nx * ny * 2};
    const cuuint32_t boxd[3] = {SB_X, SB_Y, SB_Z}, estr[3] = {1, 1, 1};
    return encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(vox), dims, strides, boxd, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One block per 128 pixels: rays cost very different amounts (a ray that misses the
// volume takes no steps), and the hardware block scheduler balances them as blocks retire.
// Measured at 1920x1080 x 8 spp, this beats a one-wave grid-stride launch by 17-24 % for
// every filter and mode.
template <int FILTER, int MODE, int V>
static cudaError_t launch_one(const MarchArgs& a, cudaStream_t st) {
    const uint64_t need = (a.pix_count + 127) / 128;
    if (need > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    k_march<FILTER, MODE, V><<<(int)(need ? need : 1), 128, 0, st>>>(a, expand_key(a.seed));
    return cudaGetLastError();
}

template <int FILTER>
static cudaError_t launch_f(const MarchArgs& a, cudaStream_t st) {
    const bool plain = a.flags == 0 && a.picks == nullptr;
    switch (a.mode) {
        case M_NTAP_BEFORE:
            return plain ? launch_one<FILTER, M_NTAP_BEFORE, KV_PLAIN>(a, st) : launch_one<FILTER, M_NTAP_BEFORE, KV_GENERAL>(a, st);
        case M_NTAP_AFTER:
            return plain ? launch_one<FILTER, M_NTAP_AFTER, KV_PLAIN>(a, st) : launch_one<FILTER, M_NTAP_AFTER, KV_GENERAL>(a, st);
        case M_STOCHASTIC:
            switch (kernel_variant(a.flags, a.picks)) {
                case KV_PLAIN: return launch_one<FILTER, M_STOCHASTIC, KV_PLAIN>(a, st);
                case KV_LATTICE: return launch_one<FILTER, M_STOCHASTIC, KV_LATTICE>(a, st);
                default: return launch_one<FILTER, M_STOCHASTIC, KV_GENERAL>(a, st);
            }
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_march(const MarchArgs& a, const CUtensorMap* tmap, int num_sms, cudaStream_t st) {
    (void)num_sms;
    if (tmap && a.filter == F_BSPLINE && (a.mode == M_NTAP_BEFORE || a.mode == M_NTAP_AFTER) && a.flags == 0 &&
        a.picks == nullptr) {
        // staged: 8 x 4 pixel tiles per warp where the range allows, so a warp's windows share a box
        MarchArgs b = a;
        const uint64_t band = 4ull * a.width;
        b.tiled = (a.width % 8 == 0 && a.pix_begin % band == 0 && a.pix_count % band == 0) ? 1 : 0;
        const uint64_t need = (a.pix_count + 127) / 128;
        if (need > 0x7FFFFFFFull) return cudaErrorInvalidValue;
        if (a.mode == M_NTAP_BEFORE)
            k_march_staged<M_NTAP_BEFORE><<<(int)(need ? need : 1), 128, 0, st>>>(b, *tmap, expand_key(a.seed));
        else
            k_march_staged<M_NTAP_AFTER><<<(int)(need ? need : 1), 128, 0, st>>>(b, *tmap, expand_key(a.seed));
        return cudaGetLastError();
    }
    if (a.filter == F_LINEAR) return launch_f<F_LINEAR>(a, st);
    if (a.filter == F_BSPLINE) return launch_f<F_BSPLINE>(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace stf
