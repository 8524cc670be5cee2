// C-ABI layer of the learned form (neural texture): creation, training, quantisation,
// checkpoints, tensor-core decode and filter + shade.  Contract: include/stf.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "stf_ctx.h"

using stfi::CurrentDevice;
using stfi::cuda_fail;
using stfi::dev_alloc;
using stfi::fail;

namespace {

constexpr uint64_t MLP_N = 6792;              // W1 2048 + b1 64 + W2 4096 + b2 64 + W3 512 + b3 8
constexpr uint64_t WBF_N = 2048 + 4096 + 1024;
constexpr uint64_t BIAS_N = 144;
constexpr uint64_t WEXT_N = 64 * 48 + 64 * 80 + 16 * 80;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

NeuralRec* find(stf_ctx c, stf_neural h) {
    auto it = c->neural.find(h);
    return it == c->neural.end() ? nullptr : &it->second;
}

size_t block_bytes(const NeuralRec& r, int what) {
    switch (what) {
        case STF_NEURAL_LATENTS: case STF_NEURAL_GRAD_LATENTS: return r.lat_total * 4;
        case STF_NEURAL_MLP: case STF_NEURAL_GRAD_MLP: return MLP_N * 4;
        case STF_NEURAL_ADAM: return (2 * r.lat_total + 2 * MLP_N) * 4;
        case STF_NEURAL_SCALES: return 16;
        case STF_NEURAL_STEP: return 4;
    }
    return 0;
}

stf_status quantize(stf_ctx c, NeuralRec& r, int fmt) {
    cudaError_t e = stf::launch_ntc_quantize(r.view, r.lat_total, fmt, r.amax, c->stream);
    if (e == cudaSuccess && fmt == 1) {
        e = cudaMemcpyAsync(r.view.scale, r.view.scale_dev, 16, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "neural quantize");
    r.latent_fmt = fmt;
    r.view.latent_fmt = fmt;
    return STF_OK;
}

stf_status check_adam(stf_ctx c, const stf_adam_params* ap) {
    if (!ap) return fail(c, STF_ERR_INVALID_ARG, "adam parameters are required");
    if (!(ap->lr_min_frac >= 0.0f && ap->lr_min_frac <= 1.0f))
        return fail(c, STF_ERR_INVALID_ARG, "lr_min_frac must lie in [0, 1]");
    return STF_OK;
}

// Optimiser step k of a run of `steps`: Adam on the latents and on the MLP with the
// half-cosine learning-rate factor (1 when lr_min_frac = 1); consumes the gradients.
cudaError_t adam_update(stf_ctx c, NeuralRec& r, const stf_adam_params& ap, uint32_t k, uint32_t steps) {
    const int t = (int)r.step + 1;
    const double f = ap.lr_min_frac, fk = f + (1.0 - f) * 0.5 * (1.0 + std::cos(M_PI * (double)k / (double)steps));
    cudaError_t e = stf::launch_adam(r.view.lat32, r.view.dlat, r.m_lat, r.v_lat, r.lat_total,
                                     (float)(ap.lr_latent * fk), ap.beta1, ap.beta2, ap.eps, t, c->num_sms, c->stream);
    if (e == cudaSuccess)
        e = stf::launch_adam(r.view.mlp32, r.view.grad32, r.m_mlp, r.v_mlp, MLP_N, (float)(ap.lr_mlp * fk), ap.beta1,
                             ap.beta2, ap.eps, t, c->num_sms, c->stream);
    r.step++;
    return e;
}

}  // namespace

extern "C" {

stf_status stf_neural_create(stf_ctx c, const stf_neural_desc* d, stf_neural* out) {
    stfi::NvtxRange nvtx_range("stf_neural_create");
    if (!c || !d || !out) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    *out = 0;
    if (d->tex_res < 1 || d->tex_res > 16384) return fail(c, STF_ERR_INVALID_ARG, "tex_res must be 1..16384");
    if (!d->latent_init || !d->mlp_init) return fail(c, STF_ERR_INVALID_ARG, "latent_init and mlp_init are required");
    for (int g = 0; g < 4; ++g) {
        if (d->grid_res[g] < 1 || d->grid_res[g] > 4096) return fail(c, STF_ERR_INVALID_ARG, "grid_res must be 1..4096");
        if (!d->latent_init[g]) return fail(c, STF_ERR_INVALID_ARG, "null latent_init grid");
    }
    CurrentDevice cd(c->device);
    NeuralRec r;
    r.view.tex_res = (int)d->tex_res;
    uint64_t T = 0;
    for (int g = 0; g < 4; ++g) {
        r.view.res[g] = (int)d->grid_res[g];
        r.view.gscale[g] = (float)d->grid_res[g] / (float)d->tex_res;   // correctly rounded, as on the device
        r.view.lat_off[g] = T;
        T += (uint64_t)d->grid_res[g] * d->grid_res[g] * 8;
        r.view.scale[g] = 1.0f;
    }
    r.lat_total = T;
    const size_t tgt = d->targets ? (size_t)d->tex_res * d->tex_res * 8 : 0;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    // the latent and MLP gradients are adjacent (the MLP's start at the next 256-byte boundary;
    // the gap stays zero), so data-parallel training sums both with one all-reduce
    const size_t o_lat32 = take(T * 4), o_dlat = take(T * 4), o_grad = take(MLP_N * 4);
    const size_t o_mlat = take(T * 4), o_vlat = take(T * 4);
    const size_t o_lat16 = take(T * 2), o_lat8 = take(T);
    const size_t o_mlp = take(MLP_N * 4), o_mm = take(MLP_N * 4), o_vm = take(MLP_N * 4);
    const size_t o_wbf = take(WBF_N * 2), o_bias = take(BIAS_N * 4), o_scale = take(16), o_amax = take(16);
    const size_t o_wext = take(WEXT_N * 2);
    const size_t o_tgt = take(tgt);
    stf_status s = dev_alloc(c, &r.mem, off);
    if (s != STF_OK) return s;
    char* b = (char*)r.mem;
    r.view.lat32 = (float*)(b + o_lat32);
    r.view.dlat = (float*)(b + o_dlat);
    r.m_lat = (float*)(b + o_mlat); r.v_lat = (float*)(b + o_vlat);
    r.view.lat16 = (const __half*)(b + o_lat16);
    r.view.lat8 = (const uint8_t*)(b + o_lat8);
    r.view.mlp32 = (float*)(b + o_mlp); r.view.grad32 = (float*)(b + o_grad);
    r.m_mlp = (float*)(b + o_mm); r.v_mlp = (float*)(b + o_vm);
    r.view.wbf = (__nv_bfloat16*)(b + o_wbf); r.view.bias = (float*)(b + o_bias);
    r.view.wext = (__nv_bfloat16*)(b + o_wext);
    r.view.scale_dev = (float*)(b + o_scale); r.amax = (unsigned int*)(b + o_amax);
    r.view.targets = tgt ? (const uint8_t*)(b + o_tgt) : nullptr;
    r.trainable = tgt != 0;
    cudaError_t e = cudaMemsetAsync(r.mem, 0, off, c->stream);
    for (int g = 0; g < 4 && e == cudaSuccess; ++g)
        e = cudaMemcpyAsync(r.view.lat32 + r.view.lat_off[g], d->latent_init[g],
                            (size_t)d->grid_res[g] * d->grid_res[g] * 8 * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.view.mlp32, d->mlp_init, MLP_N * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && tgt)
        e = cudaMemcpyAsync((void*)r.view.targets, d->targets, tgt, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) { cudaFree(r.mem); return cuda_fail(c, e, "neural upload"); }
    s = quantize(c, r, 0);
    if (s == STF_OK) {
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(c, e, "neural create");
    }
    if (s != STF_OK) { cudaFree(r.mem); return s; }
    const uint64_t h = c->next_handle++;
    c->neural[h] = r;
    *out = h;
    return STF_OK;
}

stf_status stf_neural_destroy(stf_ctx c, stf_neural h) {
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->neural.find(h);
    if (it == c->neural.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    CurrentDevice cd(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(it->second.mem);
    if (it->second.loss) cudaFree(it->second.loss);
    c->neural.erase(it);
    return STF_OK;
}

stf_status stf_neural_train(stf_ctx c, stf_neural h, uint32_t steps, uint32_t batch, const stf_adam_params* ap,
                            uint64_t seed, float* losses) {
    stfi::NvtxRange nvtx_range("stf_neural_train");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (stf_status s = check_adam(c, ap); s != STF_OK) return s;
    if (!r->trainable) return fail(c, STF_ERR_UNSUPPORTED, "created without targets");
    if (batch < 1 || batch > (1u << 24)) return fail(c, STF_ERR_INVALID_ARG, "batch must be 1..2^24");
    if (steps == 0) return STF_OK;
    CurrentDevice cd(c->device);
    if (r->loss_cap < steps) {
        if (r->loss) { cudaStreamSynchronize(c->stream); cudaFree(r->loss); r->loss = nullptr; r->loss_cap = 0; }
        stf_status s = dev_alloc(c, (void**)&r->loss, steps * 4);
        if (s != STF_OK) return s;
        r->loss_cap = steps;
    }
    cudaError_t e = cudaMemsetAsync(r->loss, 0, steps * 4, c->stream);
    e = e == cudaSuccess ? cudaMemsetAsync(r->view.grad32, 0, MLP_N * 4, c->stream) : e;
    e = e == cudaSuccess ? cudaMemsetAsync(r->view.dlat, 0, r->lat_total * 4, c->stream) : e;
    for (uint32_t k = 0; k < steps && e == cudaSuccess; ++k) {
        e = stf::launch_ntc_train(r->view, r->step, batch, 0, batch, seed, r->loss + k, nullptr, nullptr, c->num_sms,
                                  c->d_status, c->stream);
        if (e == cudaSuccess) e = adam_update(c, *r, *ap, k, steps);
    }
    if (e == cudaSuccess && losses) e = cudaMemcpyAsync(losses, r->loss, steps * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "neural train");
    stf_status s = quantize(c, *r, r->latent_fmt);
    if (s != STF_OK) return s;
    e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "neural train");
}

stf_status stf_neural_grad(stf_ctx c, stf_neural h, uint32_t step, uint32_t batch, uint64_t seed,
                           const int32_t* ex_ix, const int32_t* ex_iy, float* loss) {
    stfi::NvtxRange nvtx_range("stf_neural_grad");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (!r->trainable) return fail(c, STF_ERR_UNSUPPORTED, "created without targets");
    if (batch < 1 || batch > (1u << 24) || (!ex_ix) != (!ex_iy)) return fail(c, STF_ERR_INVALID_ARG, "bad batch or texel list");
    CurrentDevice cd(c->device);
    if (r->loss_cap < 1) {
        stf_status s = dev_alloc(c, (void**)&r->loss, 4);
        if (s != STF_OK) return s;
        r->loss_cap = 1;
    }
    cudaError_t e = cudaMemsetAsync(r->loss, 0, 4, c->stream);
    e = e == cudaSuccess ? cudaMemsetAsync(r->view.grad32, 0, MLP_N * 4, c->stream) : e;
    e = e == cudaSuccess ? cudaMemsetAsync(r->view.dlat, 0, r->lat_total * 4, c->stream) : e;
    if (e == cudaSuccess)
        e = stf::launch_ntc_train(r->view, step, batch, 0, batch, seed, r->loss, ex_ix, ex_iy, c->num_sms, c->d_status,
                                  c->stream);
    float l = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, r->loss, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "neural grad");
    if (loss) *loss = l;
    return STF_OK;
}

stf_status stf_neural_grad_range(stf_ctx c, stf_neural h, uint32_t step, uint32_t batch, uint32_t first,
                                 uint32_t count, uint64_t seed, float* loss) {
    stfi::NvtxRange nvtx_range("stf_neural_grad_range");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (!r->trainable) return fail(c, STF_ERR_UNSUPPORTED, "created without targets");
    if (batch < 1 || batch > (1u << 24) || (uint64_t)first + count > batch)
        return fail(c, STF_ERR_INVALID_ARG, "batch must be 1..2^24 and [first, first + count) inside it");
    if (loss && ((uintptr_t)loss & 3u)) return fail(c, STF_ERR_INVALID_ARG, "loss must be 4-byte aligned");
    CurrentDevice cd(c->device);
    if (!loss && r->loss_cap < 1) {
        stf_status s = dev_alloc(c, (void**)&r->loss, 4);
        if (s != STF_OK) return s;
        r->loss_cap = 1;
    }
    cudaError_t e = cudaMemsetAsync(r->view.grad32, 0, MLP_N * 4, c->stream);
    e = e == cudaSuccess ? cudaMemsetAsync(r->view.dlat, 0, r->lat_total * 4, c->stream) : e;
    if (e == cudaSuccess)
        e = stf::launch_ntc_train(r->view, step, batch, first, count, seed, loss ? loss : r->loss, nullptr, nullptr,
                                  c->num_sms, c->d_status, c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "neural grad range");
}

stf_status stf_neural_grad_buffers(stf_ctx c, stf_neural h, float** grad_latents, uint64_t* n_latents,
                                   float** grad_mlp, uint64_t* n_mlp) {
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (!grad_latents || !n_latents || !grad_mlp || !n_mlp) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    *grad_latents = r->view.dlat;
    *n_latents = r->lat_total;
    *grad_mlp = r->view.grad32;
    *n_mlp = MLP_N;
    return STF_OK;
}

stf_status stf_neural_adam_step(stf_ctx c, stf_neural h, const stf_adam_params* ap, uint32_t k, uint32_t steps) {
    stfi::NvtxRange nvtx_range("stf_neural_adam_step");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (stf_status s = check_adam(c, ap); s != STF_OK) return s;
    if (!r->trainable) return fail(c, STF_ERR_UNSUPPORTED, "created without targets");
    if (k >= steps) return fail(c, STF_ERR_INVALID_ARG, "k must lie in [0, steps)");
    CurrentDevice cd(c->device);
    const cudaError_t e = adam_update(c, *r, *ap, k, steps);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "neural adam step");
}

stf_status stf_neural_quantize(stf_ctx c, stf_neural h, stf_latent_format fmt) {
    stfi::NvtxRange nvtx_range("stf_neural_quantize");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (fmt != STF_LATENT_FP16 && fmt != STF_LATENT_FP8_E4M3 && fmt != STF_LATENT_KEEP)
        return fail(c, STF_ERR_INVALID_ARG, "unknown latent format");
    CurrentDevice cd(c->device);
    stf_status s = quantize(c, *r, fmt == STF_LATENT_KEEP ? r->latent_fmt : (int)fmt);
    if (s != STF_OK) return s;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "neural quantize");
}

static stf_status neural_copy(stf_ctx c, stf_neural h, int what, void* host, size_t bytes, bool to_host) {
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    const size_t need = block_bytes(*r, what);
    if (!host || need == 0 || bytes != need) return fail(c, STF_ERR_INVALID_ARG, "unknown block or wrong byte count");
    CurrentDevice cd(c->device);
    if (what == STF_NEURAL_STEP) {
        if (to_host) std::memcpy(host, &r->step, 4); else std::memcpy(&r->step, host, 4);
        return STF_OK;
    }
    if (what == STF_NEURAL_SCALES) {
        if (to_host) { std::memcpy(host, r->view.scale, 16); return STF_OK; }
        return fail(c, STF_ERR_UNSUPPORTED, "scales are derived by stf_neural_quantize");
    }
    struct Part { void* dev; size_t bytes; };
    Part parts[4] = {};
    int np = 1;
    switch (what) {
        case STF_NEURAL_LATENTS: parts[0] = {r->view.lat32, r->lat_total * 4}; break;
        case STF_NEURAL_GRAD_LATENTS: parts[0] = {r->view.dlat, r->lat_total * 4}; break;
        case STF_NEURAL_MLP: parts[0] = {r->view.mlp32, MLP_N * 4}; break;
        case STF_NEURAL_GRAD_MLP: parts[0] = {r->view.grad32, MLP_N * 4}; break;
        case STF_NEURAL_ADAM:
            parts[0] = {r->m_lat, r->lat_total * 4}; parts[1] = {r->v_lat, r->lat_total * 4};
            parts[2] = {r->m_mlp, MLP_N * 4}; parts[3] = {r->v_mlp, MLP_N * 4};
            np = 4;
            break;
    }
    char* hp = (char*)host;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
        const Part& p = parts[i];
        e = to_host ? cudaMemcpyAsync(hp, p.dev, p.bytes, cudaMemcpyDeviceToHost, c->stream)
                    : cudaMemcpyAsync(p.dev, hp, p.bytes, cudaMemcpyHostToDevice, c->stream);
        hp += p.bytes;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "neural block copy");
    if (!to_host && (what == STF_NEURAL_LATENTS || what == STF_NEURAL_MLP)) return quantize(c, *r, r->latent_fmt);
    return STF_OK;
}

stf_status stf_neural_get(stf_ctx c, stf_neural h, stf_neural_block what, void* host, size_t bytes) {
    return neural_copy(c, h, (int)what, host, bytes, true);
}
stf_status stf_neural_set(stf_ctx c, stf_neural h, stf_neural_block what, const void* host, size_t bytes) {
    return neural_copy(c, h, (int)what, const_cast<void*>(host), bytes, false);
}

// checkpoint file: "STFN" | u32 version=1 | u32 tex_res | u32 grid_res[4] | u32 step |
//                  FP32 latents | FP32 MLP | FP32 Adam moments
stf_status stf_neural_save(stf_ctx c, stf_neural h, const char* path) {
    if (!c || !path) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    std::vector<char> lat(block_bytes(*r, STF_NEURAL_LATENTS)), mlp(MLP_N * 4), adam(block_bytes(*r, STF_NEURAL_ADAM));
    stf_status s = neural_copy(c, h, STF_NEURAL_LATENTS, lat.data(), lat.size(), true);
    if (s == STF_OK) s = neural_copy(c, h, STF_NEURAL_MLP, mlp.data(), mlp.size(), true);
    if (s == STF_OK) s = neural_copy(c, h, STF_NEURAL_ADAM, adam.data(), adam.size(), true);
    if (s != STF_OK) return s;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c, STF_ERR_INVALID_ARG, "cannot open checkpoint for writing");
    uint32_t hdr[8] = {0x4E465453u, 1u, (uint32_t)r->view.tex_res, (uint32_t)r->view.res[0], (uint32_t)r->view.res[1],
                       (uint32_t)r->view.res[2], (uint32_t)r->view.res[3], r->step};
    bool ok = std::fwrite(hdr, 4, 8, f) == 8 && std::fwrite(lat.data(), 1, lat.size(), f) == lat.size() &&
              std::fwrite(mlp.data(), 1, mlp.size(), f) == mlp.size() &&
              std::fwrite(adam.data(), 1, adam.size(), f) == adam.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? STF_OK : fail(c, STF_ERR_INVALID_ARG, "checkpoint write failed");
}

stf_status stf_neural_load(stf_ctx c, stf_neural h, const char* path) {
    if (!c || !path) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, STF_ERR_INVALID_ARG, "cannot open checkpoint");
    uint32_t hdr[8];
    std::vector<char> lat(block_bytes(*r, STF_NEURAL_LATENTS)), mlp(MLP_N * 4), adam(block_bytes(*r, STF_NEURAL_ADAM));
    bool ok = std::fread(hdr, 4, 8, f) == 8 && hdr[0] == 0x4E465453u && hdr[1] == 1u &&
              hdr[2] == (uint32_t)r->view.tex_res && hdr[3] == (uint32_t)r->view.res[0] &&
              hdr[4] == (uint32_t)r->view.res[1] && hdr[5] == (uint32_t)r->view.res[2] &&
              hdr[6] == (uint32_t)r->view.res[3] && std::fread(lat.data(), 1, lat.size(), f) == lat.size() &&
              std::fread(mlp.data(), 1, mlp.size(), f) == mlp.size() &&
              std::fread(adam.data(), 1, adam.size(), f) == adam.size();
    std::fclose(f);
    if (!ok) return fail(c, STF_ERR_INVALID_ARG, "checkpoint does not match this network");
    stf_status s = neural_copy(c, h, STF_NEURAL_LATENTS, lat.data(), lat.size(), false);
    if (s == STF_OK) s = neural_copy(c, h, STF_NEURAL_MLP, mlp.data(), mlp.size(), false);
    if (s == STF_OK) s = neural_copy(c, h, STF_NEURAL_ADAM, adam.data(), adam.size(), false);
    if (s == STF_OK) r->step = hdr[7];
    return s;
}

stf_status stf_neural_decode(stf_ctx c, stf_neural h, uint64_t n, const int32_t* ix, const int32_t* iy, float* y) {
    stfi::NvtxRange nvtx_range("stf_neural_decode");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (n == 0) return STF_OK;
    if (!ix || !iy || !y || n > (1ull << 34)) return fail(c, STF_ERR_INVALID_ARG, "bad decode arguments");
    if (c->fault == stfi::FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    CurrentDevice cd(c->device);
    stf::NeuralDecodeArgs a{};
    a.n = n; a.mode = -1; a.filter = 0; a.spp = 1; a.nrows = n; a.tex_res = r->view.tex_res;
    a.ex_ix = ix; a.ex_iy = iy; a.y_out = y; a.status = c->d_status;
    a.inject_timeout = c->fault == stfi::FAULT_MMA_TIMEOUT;
    cudaError_t e = stf::launch_ntc_decode(r->view, a, c->num_sms, c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "neural decode launch");
}

stf_status stf_neural_filter_shade(stf_ctx c, stf_neural h, const stf_queries* q, const stf_derivs* d,
                                   stf_filter f, stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed,
                                   uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_neural_filter_shade");
    if (!c) return STF_ERR_INVALID_ARG;
    NeuralRec* r = find(c, h);
    if (!r) return fail(c, STF_ERR_BAD_HANDLE, "unknown neural handle");
    if (!q || !out) return fail(c, STF_ERR_INVALID_ARG, "queries and output must be non-null");
    if (f < 0 || f > 3 || m < 0 || m > 3 || (sh != STF_SHADE_GGX_LAMBERT && sh != STF_SHADE_LINEAR))
        return fail(c, STF_ERR_INVALID_ARG, "filter, mode or shade out of range");
    if (m == STF_MODE_STOCHASTIC_POSITIVIZED && f != STF_FILTER_MITCHELL && f != STF_FILTER_CATMULL_ROM)
        return fail(c, STF_ERR_UNSUPPORTED, "positivization needs a filter with negative lobes");
    if (spp == 0) return fail(c, STF_ERR_INVALID_ARG, "spp must be >= 1");
    if (flags != 0) return fail(c, STF_ERR_INVALID_ARG, "flags must be 0");
    if (q->n == 0) return STF_OK;
    if (!q->u || !q->v || !out->r || !out->g || !out->b) return fail(c, STF_ERR_INVALID_ARG, "null query/output pointer");
    if (q->order) return fail(c, STF_ERR_UNSUPPORTED, "the neural path takes no execution order");
    if (d && (!d->dudx || !d->dvdx || !d->dudy || !d->dvdy)) return fail(c, STF_ERR_INVALID_ARG, "null derivative pointer");
    const int nt = f == STF_FILTER_LINEAR ? 2 : 4;
    const uint64_t nr = m == STF_MODE_STOCHASTIC ? 1 : (m == STF_MODE_STOCHASTIC_POSITIVIZED ? 2 : (uint64_t)nt * nt);
    const uint64_t rows = q->n * (uint64_t)spp * nr;
    if (q->n > (1ull << 40) || rows > (1ull << 42)) return fail(c, STF_ERR_INVALID_ARG, "too many decodes");
    if (c->fault == stfi::FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    CurrentDevice cd(c->device);
    cudaError_t e = cudaMemsetAsync(out->r, 0, q->n * 4, c->stream);
    e = e == cudaSuccess ? cudaMemsetAsync(out->g, 0, q->n * 4, c->stream) : e;
    e = e == cudaSuccess ? cudaMemsetAsync(out->b, 0, q->n * 4, c->stream) : e;
    if (e != cudaSuccess) return cuda_fail(c, e, "neural filter output clear");
    stf::NeuralDecodeArgs a{};
    a.n = q->n; a.id_base = q->id_base; a.u = q->u; a.v = q->v;
    a.has_derivs = d ? 1 : 0;
    if (d) { a.dudx = d->dudx; a.dvdx = d->dvdx; a.dudy = d->dudy; a.dvdy = d->dvdy; }
    a.filter = f; a.mode = m; a.shade = sh; a.spp = spp; a.seed = seed; a.tex_res = r->view.tex_res;
    a.nrows = rows; a.r = out->r; a.g = out->g; a.b = out->b; a.status = c->d_status;
    a.inject_timeout = c->fault == stfi::FAULT_MMA_TIMEOUT;
    e = stf::launch_ntc_decode(r->view, a, c->num_sms, c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "neural filter_shade launch");
}

}  // extern "C"
