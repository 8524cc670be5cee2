// C-ABI layer of libstf: contexts, handles, argument validation, uploads and launches.
// See include/stf.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "stf_ctx.h"

using stfi::CurrentDevice;

namespace stfi {
stf_status fail(stf_ctx c, stf_status s, const char* msg) {
    if (c) c->last_error = msg;
    return s;
}
stf_status cuda_fail(stf_ctx c, cudaError_t e, const char* where) {
    if (c) c->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STF_ERR_OOM : STF_ERR_CUDA;
}
stf_status dev_alloc(stf_ctx c, void** p, size_t bytes) {
    if (c->fault == FAULT_ALLOC) return fail(c, STF_ERR_OOM, "injected allocation failure (STF_FAULT=alloc)");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(c, e, "cudaMalloc"); }
    return STF_OK;
}
}  // namespace stfi

namespace {
using stfi::fail;
using stfi::cuda_fail;
using stfi::dev_alloc;

bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }
bool bad_enum_filter(int f) { return f < 0 || f > 3; }
bool bad_enum_mode(int m) { return m < 0 || m > 3; }
bool signed_filter(int f) { return f == STF_FILTER_CATMULL_ROM || f == STF_FILTER_MITCHELL; }
int square_side(uint32_t spp) {
    int k = (int)std::lround(std::sqrt((double)spp));
    return (uint32_t)(k * k) == spp ? k : -1;
}
uint32_t level_dim(uint32_t d, uint32_t l) { uint32_t x = d >> l; return x ? x : 1u; }


// Waits for the copy-pipeline lanes (asynchronous host-buffer calls may still use them).
void drain_lanes(stf_ctx c) {
    for (int i = 0; i < STF_LANES; ++i)
        if (c->lane[i]) cudaStreamSynchronize(c->lane[i]);
}

// Staging of the host-buffer pipeline; only the lanes touch it.
stf_status ensure_stage(stf_ctx c, size_t bytes) {
    if (c->stage_bytes >= bytes) return STF_OK;
    if (c->stage) {
        drain_lanes(c);
        cudaFree(c->stage); c->stage = nullptr; c->stage_bytes = 0; c->lane_bytes = 0;
    }
    stf_status s = dev_alloc(c, &c->stage, bytes);
    if (s == STF_OK) c->stage_bytes = bytes;
    return s;
}

// Histogram scratch of the binning call; only the context stream touches it.
stf_status ensure_bin_scratch(stf_ctx c, size_t bytes) {
    if (c->bin_scratch_bytes >= bytes) return STF_OK;
    if (c->bin_scratch) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->bin_scratch); c->bin_scratch = nullptr; c->bin_scratch_bytes = 0;
    }
    stf_status s = dev_alloc(c, &c->bin_scratch, bytes);
    if (s == STF_OK) c->bin_scratch_bytes = bytes;
    return s;
}

stf_status validate_filter_call(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d,
                                stf_filter f, stf_mode m, stf_shade sh, uint32_t spp, uint32_t flags,
                                const stf_output* out, TexRec** rec) {
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->tex.find(t);
    if (it == c->tex.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown texture handle");
    *rec = &it->second;
    if (!q || !out) return fail(c, STF_ERR_INVALID_ARG, "queries and output must be non-null");
    if ((bad_enum_filter(f) && f != STF_FILTER_EWA) || bad_enum_mode(m) ||
        (sh != STF_SHADE_GGX_LAMBERT && sh != STF_SHADE_LINEAR))
        return fail(c, STF_ERR_INVALID_ARG, "filter, mode or shade out of range");
    if (m == STF_MODE_STOCHASTIC_POSITIVIZED && !signed_filter(f))
        return fail(c, STF_ERR_UNSUPPORTED, "positivization needs a filter with negative lobes");
    if (spp == 0) return fail(c, STF_ERR_INVALID_ARG, "spp must be >= 1");
    if ((flags & STF_FLAG_REUSE) && m == STF_MODE_STOCHASTIC_POSITIVIZED)
        return fail(c, STF_ERR_UNSUPPORTED, "sample reuse is defined for the 1-tap estimator");
    if (flags & ~(uint32_t)(STF_FLAG_STRATIFIED | STF_FLAG_LATTICE | STF_FLAG_REUSE | STF_FLAG_LOD0))
        return fail(c, STF_ERR_INVALID_ARG, "unknown flag bits");
    if (f == STF_FILTER_EWA && (flags & ~(uint32_t)STF_FLAG_LOD0))
        return fail(c, STF_ERR_UNSUPPORTED, "EWA takes no jitter, lattice or reuse flags");
    if ((flags & STF_FLAG_STRATIFIED) && square_side(spp) < 0)
        return fail(c, STF_ERR_INVALID_ARG, "stratified jitter needs a square spp");
    if (q->n == 0) return STF_OK;
    if (q->n > (1ull << 40)) return fail(c, STF_ERR_INVALID_ARG, "too many queries");
    if (out->picks && q->n * (uint64_t)spp > (1ull << 40)) return fail(c, STF_ERR_INVALID_ARG, "pick buffer too large");
    const void* ptrs[5] = {q->u, q->v, out->r, out->g, out->b};
    for (const void* p : ptrs)
        if (!p || !aligned4(p)) return fail(c, STF_ERR_INVALID_ARG, "query/output pointers must be non-null and 4-byte aligned");
    if (d) {
        const void* dp[4] = {d->dudx, d->dvdx, d->dudy, d->dvdy};
        for (const void* p : dp)
            if (!p || !aligned4(p)) return fail(c, STF_ERR_INVALID_ARG, "derivative pointers must be all non-null and 4-byte aligned");
    }
    if (out->picks && !aligned4(out->picks)) return fail(c, STF_ERR_INVALID_ARG, "picks must be 4-byte aligned");
    return STF_OK;
}

}  // namespace

namespace stfi {
stf_status validate_filter_args(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d, stf_filter f,
                                stf_mode m, stf_shade sh, uint32_t spp, uint32_t flags, const stf_output* out,
                                TexRec** rec, int* kside) {
    const stf_status s = validate_filter_call(c, t, q, d, f, m, sh, spp, flags, out, rec);
    if (s == STF_OK && kside) *kside = (flags & STF_FLAG_STRATIFIED) ? square_side(spp) : 1;
    return s;
}
}  // namespace stfi

using stfi::fail;
using stfi::cuda_fail;
using stfi::dev_alloc;
using stfi::FAULT_ALLOC;
using stfi::FAULT_LAUNCH;

extern "C" {

const char* stf_status_string(stf_status s) {
    switch (s) {
        case STF_OK: return "STF_OK";
        case STF_ERR_INVALID_ARG: return "STF_ERR_INVALID_ARG";
        case STF_ERR_BAD_HANDLE: return "STF_ERR_BAD_HANDLE";
        case STF_ERR_OOM: return "STF_ERR_OOM";
        case STF_ERR_CUDA: return "STF_ERR_CUDA";
        case STF_ERR_UNSUPPORTED: return "STF_ERR_UNSUPPORTED";
        case STF_ERR_DEVICE_STATUS: return "STF_ERR_DEVICE_STATUS";
        case STF_ERR_TIMEOUT: return "STF_ERR_TIMEOUT";
    }
    return "STF_ERR_UNKNOWN";
}

const char* stf_last_error(stf_ctx c) { return c ? c->last_error.c_str() : "null context"; }

stf_status stf_create(int device, void* cuda_stream, stf_ctx* out) {
    if (!out) return STF_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) { cudaGetLastError(); return STF_ERR_CUDA; }
    if (device < 0 || device >= ndev) return STF_ERR_INVALID_ARG;
    stf_ctx c = new stf_ctx_s();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (const char* f = std::getenv("STF_FAULT")) {
        if (!std::strcmp(f, "alloc")) c->fault = FAULT_ALLOC;
        else if (!std::strcmp(f, "launch")) c->fault = FAULT_LAUNCH;
        else if (!std::strcmp(f, "mma_timeout")) c->fault = stfi::FAULT_MMA_TIMEOUT;
    }
    CurrentDevice cd(device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    stf_status s = dev_alloc(c, (void**)&c->d_status, sizeof(uint32_t));
    if (s != STF_OK) { delete c; return s; }
    cudaMemset(c->d_status, 0, sizeof(uint32_t));
    // EWA weights exp(-2 r^2) - exp(-2) at r^2 = i/127, rounded once to FP32
    float lut[stf::EWA_LUT_N];
    for (int i = 0; i < stf::EWA_LUT_N; ++i) {
        const double r2 = (double)i / (double)(stf::EWA_LUT_N - 1);
        lut[i] = (float)(std::exp(-2.0 * r2) - std::exp(-2.0));
    }
    s = dev_alloc(c, (void**)&c->d_ewa_lut, sizeof(lut));
    if (s == STF_OK && cudaMemcpy(c->d_ewa_lut, lut, sizeof(lut), cudaMemcpyHostToDevice) != cudaSuccess)
        s = STF_ERR_CUDA;
    if (s != STF_OK) { cudaFree(c->d_status); if (c->d_ewa_lut) cudaFree(c->d_ewa_lut); delete c; return s; }
    *out = c;
    return STF_OK;
}

stf_status stf_destroy(stf_ctx c) {
    if (!c) return STF_ERR_INVALID_ARG;
    CurrentDevice cd(c->device);
    cudaStreamSynchronize(c->stream);
    drain_lanes(c);
    for (auto& kv : c->tex) cudaFree(kv.second.mem);
    for (auto& kv : c->vol) { cudaFree(kv.second.mem); cudaFree(kv.second.pad); }
    for (auto& kv : c->tables) cudaFree(kv.second.mem);
    for (auto& kv : c->neural) { cudaFree(kv.second.mem); if (kv.second.loss) cudaFree(kv.second.loss); }
    for (int i = 0; i < STF_LANES; ++i) {
        if (c->lane[i]) { cudaStreamSynchronize(c->lane[i]); cudaStreamDestroy(c->lane[i]); }
    }
    for (int i = 0; i < STF_LANES; ++i)
        if (c->lane_ev[i]) cudaEventDestroy(c->lane_ev[i]);
    if (c->entry_ev) cudaEventDestroy(c->entry_ev);
    if (c->stage) cudaFree(c->stage);
    if (c->bin_scratch) cudaFree(c->bin_scratch);
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_ewa_lut) cudaFree(c->d_ewa_lut);
    delete c;
    return STF_OK;
}

stf_status stf_set_stream(stf_ctx c, void* stream) {
    if (!c) return STF_ERR_INVALID_ARG;
    // the binning scratch and the status word are context-owned: work queued on the old
    // stream finishes before work on the new one can reuse them
    CurrentDevice cd(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    c->stream = (cudaStream_t)stream;
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "cudaStreamSynchronize");
}

stf_status stf_synchronize(stf_ctx c) {
    if (!c) return STF_ERR_INVALID_ARG;
    CurrentDevice cd(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    for (int i = 0; i < STF_LANES && e == cudaSuccess; ++i)
        if (c->lane[i]) e = cudaStreamSynchronize(c->lane[i]);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "cudaStreamSynchronize");
}

stf_status stf_get_device_status(stf_ctx c, uint32_t* flags) {
    if (!c || !flags) return STF_ERR_INVALID_ARG;
    CurrentDevice cd(c->device);
    drain_lanes(c);      // kernels of asynchronous host-buffer calls report here too
    uint32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_status, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device status read");
    *flags = h;
    return h ? STF_ERR_DEVICE_STATUS : STF_OK;
}

// ------------------------------------------------------------------------------ textures
// DCT-compressed levels are stored as given: ceil(H/8) x ceil(W/8) blocks of 32 bytes each.
static stf_status create_dct_texture(stf_ctx c, const stf_texture_desc* d, stf_tex* out) {
    if (d->normal_data) return fail(c, STF_ERR_INVALID_ARG, "DCT6 textures carry their normals in the blocks");
    TexRec rec;
    rec.view.fmt = stf::FMT_DCT;
    rec.view.levels = (int)d->num_levels;
    rec.view.has_normal = 1;
    rec.view.address = 0;
    size_t total = 0;
    size_t bytes[STF_MAX_LEVELS] = {};
    for (uint32_t l = 0; l < d->num_levels; ++l) {
        const uint32_t w = level_dim(d->width, l), h = level_dim(d->height, l);
        if (d->data_on_device && ((uintptr_t)d->level_data[l] & 15u))
            return fail(c, STF_ERR_INVALID_ARG, "device DCT6 levels must be 16-byte aligned");
        rec.view.w[l] = (int)w; rec.view.h[l] = (int)h;
        rec.view.off[l] = total;
        bytes[l] = (size_t)((w + 7) / 8) * ((h + 7) / 8) * 32;
        total += (bytes[l] + 255) & ~(size_t)255;
    }
    for (uint32_t l = d->num_levels; l < STF_MAX_LEVELS; ++l) { rec.view.w[l] = rec.view.h[l] = 1; rec.view.off[l] = 0; }
    stf_status s = dev_alloc(c, &rec.mem, total);
    if (s != STF_OK) return s;
    rec.view.base = rec.mem;
    const cudaMemcpyKind kind = d->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaSuccess;
    for (uint32_t l = 0; l < d->num_levels && e == cudaSuccess; ++l)
        e = cudaMemcpyAsync((char*)rec.mem + rec.view.off[l], d->level_data[l], bytes[l], kind, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { cudaFree(rec.mem); return cuda_fail(c, e, "DCT texture upload"); }
    const uint64_t h = c->next_handle++;
    c->tex[h] = rec;
    *out = h;
    return STF_OK;
}

stf_status stf_create_texture(stf_ctx c, const stf_texture_desc* d, stf_tex* out) {
    stfi::NvtxRange nvtx_range("stf_create_texture");
    if (!c || !d || !out) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    *out = 0;
    if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384)
        return fail(c, STF_ERR_INVALID_ARG, "texture size must be 1..16384");
    if (d->num_levels < 1 || d->num_levels > STF_MAX_LEVELS) return fail(c, STF_ERR_INVALID_ARG, "num_levels must be 1..16");
    if (d->format != STF_FMT_RGBA32F && d->format != STF_FMT_RGBA8 && d->format != STF_FMT_DCT6)
        return fail(c, STF_ERR_INVALID_ARG, "2-D textures are RGBA32F, RGBA8 or DCT6");
    if (d->address != STF_ADDRESS_WRAP) return fail(c, STF_ERR_UNSUPPORTED, "2-D textures use wrap addressing");
    if (!d->level_data) return fail(c, STF_ERR_INVALID_ARG, "level_data is null");
    if (d->normal_data && d->format != STF_FMT_RGBA8) return fail(c, STF_ERR_INVALID_ARG, "normal maps accompany RGBA8 textures");
    for (uint32_t l = 0; l < d->num_levels; ++l) {
        if (!d->level_data[l]) return fail(c, STF_ERR_INVALID_ARG, "null level pointer");
        if (d->normal_data && !d->normal_data[l]) return fail(c, STF_ERR_INVALID_ARG, "null normal level pointer");
        if (d->data_on_device && d->format == STF_FMT_RGBA8 &&
            (((uintptr_t)d->level_data[l] & 3u) || (d->normal_data && ((uintptr_t)d->normal_data[l] & 1u))))
            return fail(c, STF_ERR_INVALID_ARG, "device RGBA8 levels must be 4-byte and RG8 levels 2-byte aligned");
    }
    CurrentDevice cd(c->device);
    if (d->format == STF_FMT_DCT6) return create_dct_texture(c, d, out);
    const size_t texel = d->format == STF_FMT_RGBA32F ? 16 : 8;
    TexRec rec;
    rec.view.fmt = d->format == STF_FMT_RGBA32F ? 0 : 1;
    rec.view.levels = (int)d->num_levels;
    rec.view.has_normal = d->normal_data ? 1 : 0;
    rec.view.address = 0;
    size_t total = 0, max_level = 0;
    for (uint32_t l = 0; l < d->num_levels; ++l) {
        const uint32_t w = level_dim(d->width, l), h = level_dim(d->height, l);
        rec.view.w[l] = (int)w; rec.view.h[l] = (int)h;
        rec.view.off[l] = total;
        const size_t b = (size_t)w * h * texel;
        total += (b + 255) & ~(size_t)255;
        max_level = std::max(max_level, (size_t)w * h);
    }
    for (uint32_t l = d->num_levels; l < STF_MAX_LEVELS; ++l) { rec.view.w[l] = rec.view.h[l] = 1; rec.view.off[l] = 0; }
    stf_status s = dev_alloc(c, &rec.mem, total);
    if (s != STF_OK) return s;
    rec.view.base = rec.mem;
    const cudaMemcpyKind kind = d->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaSuccess;
    void* tmp = nullptr;
    if (rec.view.fmt == 1 && !d->data_on_device) {
        s = dev_alloc(c, &tmp, max_level * 6);
        if (s != STF_OK) { cudaFree(rec.mem); return s; }
    }
    for (uint32_t l = 0; l < d->num_levels && e == cudaSuccess; ++l) {
        const size_t n = (size_t)rec.view.w[l] * rec.view.h[l];
        char* dst = (char*)rec.mem + rec.view.off[l];
        if (rec.view.fmt == 0) {
            e = cudaMemcpyAsync(dst, d->level_data[l], n * 16, kind, c->stream);
        } else {
            const void* rgba = d->level_data[l];
            const void* rg = d->normal_data ? d->normal_data[l] : nullptr;
            if (!d->data_on_device) {
                e = cudaMemcpyAsync(tmp, rgba, n * 4, cudaMemcpyHostToDevice, c->stream);
                if (e == cudaSuccess && rg) e = cudaMemcpyAsync((char*)tmp + n * 4, rg, n * 2, cudaMemcpyHostToDevice, c->stream);
                rgba = tmp;
                rg = rg ? (const char*)tmp + n * 4 : nullptr;
            }
            if (e == cudaSuccess) e = stf::launch_pack_rgba8(rgba, rg, dst, n, c->stream);
            if (e == cudaSuccess && !d->data_on_device) e = cudaStreamSynchronize(c->stream);   // tmp reuse
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) { cudaFree(rec.mem); return cuda_fail(c, e, "texture upload"); }
    const uint64_t h = c->next_handle++;
    c->tex[h] = rec;
    *out = h;
    return STF_OK;
}

stf_status stf_destroy_texture(stf_ctx c, stf_tex t) {
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->tex.find(t);
    if (it == c->tex.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown texture handle");
    for (auto& kv : c->tables)
        for (uint64_t m : kv.second.members)
            if (m == t) return fail(c, STF_ERR_INVALID_ARG, "texture is referenced by a texture table");
    CurrentDevice cd(c->device);
    cudaStreamSynchronize(c->stream);
    drain_lanes(c);
    cudaFree(it->second.mem);
    c->tex.erase(it);
    return STF_OK;
}

// ------------------------------------------------------------------------- filter + shade
static stf_status enqueue_filter(stf_ctx c, const TexRec& rec, const stf_queries* q, const stf_derivs* d,
                                 int f, stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed,
                                 uint32_t flags, const stf_output* out, cudaStream_t stream, float sigma = 0.0f) {
    if (c->fault == FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    stf::FilterShadeArgs a{};
    a.n = q->n; a.id_base = q->id_base; a.u = q->u; a.v = q->v; a.order = q->order;
    a.has_derivs = d ? 1 : 0;
    if (d) { a.dudx = d->dudx; a.dvdx = d->dvdx; a.dudy = d->dudy; a.dvdy = d->dvdy; }
    a.filter = f; a.mode = m; a.shade = sh; a.spp = spp; a.flags = flags;
    a.kside = (flags & STF_FLAG_STRATIFIED) ? square_side(spp) : 1;
    a.seed = seed; a.r = out->r; a.g = out->g; a.b = out->b; a.picks = out->picks;
    a.status = c->d_status;
    a.ewa_lut = c->d_ewa_lut;
    a.sigma = sigma;
    a.inv_s2 = sigma > 0.0f ? 1.0f / (sigma * sigma) : 0.0f;
    cudaError_t e = stf::launch_filter_shade(a, rec.view, c->num_sms, stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "filter_shade launch");
}

stf_status stf_filter_shade(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d,
                            stf_filter f, stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed,
                            uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_filter_shade");
    TexRec* rec = nullptr;
    stf_status s = validate_filter_call(c, t, q, d, f, m, sh, spp, flags, out, &rec);
    if (s != STF_OK || q->n == 0) return s;
    CurrentDevice cd(c->device);
    return enqueue_filter(c, *rec, q, d, f, m, sh, spp, seed, flags, out, c->stream);
}

stf_status stf_filter_shade_ex(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d,
                               const stf_filter_desc* fd, stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed,
                               uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_filter_shade_ex");
    if (!c) return STF_ERR_INVALID_ARG;
    if (!fd) return fail(c, STF_ERR_INVALID_ARG, "null filter descriptor");
    if (fd->sampler != STF_SAMPLER_FRS && fd->sampler != STF_SAMPLER_FIS)
        return fail(c, STF_ERR_INVALID_ARG, "sampler out of range");
    const bool gauss = fd->filter == STF_FILTER_GAUSSIAN, fis = fd->sampler == STF_SAMPLER_FIS;
    if (!gauss && !fis) return stf_filter_shade(c, t, q, d, fd->filter, m, sh, spp, seed, flags, out);
    if (fis && fd->filter != STF_FILTER_LINEAR && fd->filter != STF_FILTER_BSPLINE && !gauss)
        return fail(c, STF_ERR_UNSUPPORTED, "FIS samples the tent, the cubic B-spline and the Gaussian");
    if (gauss && !(fd->sigma > 0.0f && fd->sigma <= 8.0f))
        return fail(c, STF_ERR_INVALID_ARG, "sigma must lie in (0, 8]");
    if (m == STF_MODE_STOCHASTIC_POSITIVIZED) return fail(c, STF_ERR_UNSUPPORTED, "no positivization for these filters");
    if (flags & ~(uint32_t)(STF_FLAG_STRATIFIED | STF_FLAG_LOD0))
        return fail(c, STF_ERR_UNSUPPORTED, "Gaussian and FIS lookups take the STRATIFIED and LOD0 flags only");
    // internal filter id: FIS picks are their own kernels; an N-tap FIS call evaluates the
    // filter that FIS converges to
    int fi;
    if (!fis) fi = stf::F_GAUSS;
    else if (m == STF_MODE_STOCHASTIC) fi = fd->filter == STF_FILTER_LINEAR ? stf::F_FIS_LINEAR
                                          : fd->filter == STF_FILTER_BSPLINE ? stf::F_FIS_BSPLINE : stf::F_FIS_GAUSS;
    else fi = fd->filter == STF_FILTER_LINEAR ? stf::F_LINEAR : fd->filter == STF_FILTER_BSPLINE ? stf::F_BSPLINE
                                                                                                : stf::F_GAUSS_BOX;
    TexRec* rec = nullptr;
    stf_status s = validate_filter_call(c, t, q, d, STF_FILTER_LINEAR, m, sh, spp, flags, out, &rec);
    if (s != STF_OK || q->n == 0) return s;
    CurrentDevice cd(c->device);
    return enqueue_filter(c, *rec, q, d, fi, m, sh, spp, seed, flags, out, c->stream, gauss ? fd->sigma : 0.0f);
}

// ------------------------------------------------------------------------- triplanar
stf_status stf_triplanar_shade(stf_ctx c, const stf_tex tex[3], float scale, const stf_tri_queries* q,
                               const stf_tri_derivs* d, stf_filter f, stf_mode m, stf_blend blend, stf_shade sh,
                               uint32_t spp, uint64_t seed, uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_triplanar_shade");
    if (!c) return STF_ERR_INVALID_ARG;
    if (!tex || !q || !out) return fail(c, STF_ERR_INVALID_ARG, "textures, queries and output must be non-null");
    TexRec* rec[3];
    for (int i = 0; i < 3; ++i) {
        auto it = c->tex.find(tex[i]);
        if (it == c->tex.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown texture handle");
        rec[i] = &it->second;
    }
    const bool dct0 = rec[0]->view.fmt == stf::FMT_DCT;
    if ((rec[1]->view.fmt == stf::FMT_DCT) != dct0 || (rec[2]->view.fmt == stf::FMT_DCT) != dct0)
        return fail(c, STF_ERR_INVALID_ARG, "the three textures must all be DCT6 or all be uncompressed");
    if (bad_enum_filter(f) || bad_enum_mode(m) || (sh != STF_SHADE_GGX_LAMBERT && sh != STF_SHADE_LINEAR) ||
        (blend != STF_BLEND_FULL && blend != STF_BLEND_STOCHASTIC))
        return fail(c, STF_ERR_INVALID_ARG, "filter, mode, blend or shade out of range");
    if (m == STF_MODE_STOCHASTIC_POSITIVIZED && !signed_filter(f))
        return fail(c, STF_ERR_UNSUPPORTED, "positivization needs a filter with negative lobes");
    if (spp == 0) return fail(c, STF_ERR_INVALID_ARG, "spp must be >= 1");
    if (flags & ~(uint32_t)(STF_FLAG_STRATIFIED | STF_FLAG_LATTICE | STF_FLAG_REUSE | STF_FLAG_LOD0))
        return fail(c, STF_ERR_INVALID_ARG, "unknown flag bits");
    if (flags & STF_FLAG_REUSE) return fail(c, STF_ERR_UNSUPPORTED, "triplanar lookups take no sample reuse");
    if ((flags & STF_FLAG_STRATIFIED) && square_side(spp) < 0)
        return fail(c, STF_ERR_INVALID_ARG, "stratified jitter needs a square spp");
    if (!std::isfinite(scale) || scale == 0.0f) return fail(c, STF_ERR_INVALID_ARG, "scale must be finite and non-zero");
    if (q->n == 0) return STF_OK;
    if (q->n > (1ull << 40)) return fail(c, STF_ERR_INVALID_ARG, "too many queries");
    if (out->picks && q->n * (uint64_t)spp > (1ull << 38)) return fail(c, STF_ERR_INVALID_ARG, "pick buffer too large");
    const void* ptrs[9] = {q->px, q->py, q->pz, q->nx, q->ny, q->nz, out->r, out->g, out->b};
    for (const void* p : ptrs)
        if (!p || !aligned4(p)) return fail(c, STF_ERR_INVALID_ARG, "query/output pointers must be non-null and 4-byte aligned");
    if (d) {
        const void* dp[6] = {d->dpdx_x, d->dpdx_y, d->dpdx_z, d->dpdy_x, d->dpdy_y, d->dpdy_z};
        for (const void* p : dp)
            if (!p || !aligned4(p)) return fail(c, STF_ERR_INVALID_ARG, "derivative pointers must be all non-null and 4-byte aligned");
    }
    if (out->picks && !aligned4(out->picks)) return fail(c, STF_ERR_INVALID_ARG, "picks must be 4-byte aligned");
    if (c->fault == FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    CurrentDevice cd(c->device);
    stf::TriplanarArgs a{};
    a.n = q->n; a.id_base = q->id_base; a.order = q->order;
    a.px = q->px; a.py = q->py; a.pz = q->pz; a.nx = q->nx; a.ny = q->ny; a.nz = q->nz;
    a.has_derivs = d ? 1 : 0;
    if (d) {
        a.dxx = d->dpdx_x; a.dxy = d->dpdx_y; a.dxz = d->dpdx_z;
        a.dyx = d->dpdy_x; a.dyy = d->dpdy_y; a.dyz = d->dpdy_z;
    }
    a.scale = scale;
    a.filter = f; a.mode = m; a.blend = blend; a.shade = sh; a.spp = spp; a.flags = flags;
    a.kside = (flags & STF_FLAG_STRATIFIED) ? square_side(spp) : 1;
    a.seed = seed; a.r = out->r; a.g = out->g; a.b = out->b; a.picks = out->picks;
    a.status = c->d_status;
    const stf::TexView tv[3] = {rec[0]->view, rec[1]->view, rec[2]->view};
    cudaError_t e = stf::launch_triplanar(a, tv, c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "triplanar launch");
}

// The host-buffer path is a copy pipeline: the queries are cut into chunks, and chunk k
// goes to lane k mod STF_LANES (its own stream and staging buffers), so that one chunk's
// host->device copy, another's kernel and a third's device->host copy run at once on the
// two copy engines and the SMs.  Each chunk keeps its global query ids (id_base + offset),
// so the random numbers, and therefore the results, do not depend on the chunking.
static stf_status ensure_lanes(stf_ctx c) {
    for (int i = 0; i < STF_LANES; ++i) {
        if (c->lane[i]) continue;
        cudaError_t e = cudaStreamCreateWithFlags(&c->lane[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "lane stream creation");
    }
    cudaEvent_t* evs[STF_LANES + 1] = {&c->entry_ev};
    for (int i = 0; i < STF_LANES; ++i) evs[i + 1] = &c->lane_ev[i];
    for (cudaEvent_t* ev : evs) {
        if (*ev) continue;
        cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(c, e, "event creation");
    }
    return STF_OK;
}

static stf_status host_pipeline(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d, stf_filter f,
                                stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed, uint32_t flags,
                                const stf_output* out, bool async) {
    TexRec* rec = nullptr;
    stf_status s = validate_filter_call(c, t, q, d, f, m, sh, spp, flags, out, &rec);
    if (s != STF_OK || q->n == 0) return s;
    if (q->order) return fail(c, STF_ERR_UNSUPPORTED, "the host-buffer entry point takes no execution order");
    CurrentDevice cd(c->device);
    const uint64_t n = q->n;
    const int nin = d ? 6 : 2;
    // chunk: 2^16 .. 2^21 queries (at most ~256 MB of staging per lane), a multiple of 256.
    // Each call drains its pipeline before returning, so smaller chunks fill and drain it
    // faster, while larger ones move each array in fewer, larger copies.  Measured on the
    // bench's 2^24-query calls (8 spp), 2^21 was best: 13.8 G lookups/s end to end, against
    // 12.1 / 13.2 / 13.6 / 13.5 at 2^18 / 2^19 / 2^20 / 2^22.
    const uint64_t per_q = (uint64_t)(nin + 3) * 4 + (out->picks ? (uint64_t)spp * 8 : 0);
    uint64_t chunk = std::min<uint64_t>(1ull << 21, std::max<uint64_t>(1ull << 16, (256ull << 20) / per_q)) & ~255ull;
    chunk = std::min(chunk, n);
    const uint64_t nchunks = (n + chunk - 1) / chunk;
    const int lanes = (int)std::min<uint64_t>(STF_LANES, nchunks);
    const size_t fb = ((chunk * 4 + 255) / 256) * 256;
    const size_t pick_b = out->picks ? ((chunk * spp * 8 + 255) / 256) * 256 : 0;
    const size_t lane_b = fb * (nin + 3) + pick_b;
    s = ensure_lanes(c);
    if (s == STF_OK) s = ensure_stage(c, lane_b * lanes);
    if (s != STF_OK) return s;
    cudaError_t e = cudaEventRecord(c->entry_ev, c->stream);   // earlier work on the caller's stream
    for (int i = 0; i < lanes && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->lane[i], c->entry_ev, 0);
    // Lane i stages in [i * lane_b, (i + 1) * lane_b).  Calls with the same layout reuse each
    // region on the same lane, so stream order protects it.  A new layout moves the regions
    // across the old ones: every lane (used by this call or not, so that later calls with
    // this layout inherit the order) then also waits for the other lanes' earlier work.
    if (c->lane_bytes != 0 && c->lane_bytes != lane_b)
        for (int i = 0; i < STF_LANES && e == cudaSuccess; ++i)
            for (int j = 0; j < STF_LANES && e == cudaSuccess; ++j)
                if (j != i) e = cudaStreamWaitEvent(c->lane[i], c->lane_ev[j], 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream ordering");
    c->lane_bytes = lane_b;
    const float* hv[6] = {q->u, q->v, d ? d->dudx : nullptr, d ? d->dvdx : nullptr, d ? d->dudy : nullptr, d ? d->dvdy : nullptr};
    float* ho[3] = {out->r, out->g, out->b};
    stf_status first = STF_OK;
    for (uint64_t k = 0; k < nchunks && first == STF_OK; ++k) {
        const int li = (int)(k % lanes);
        cudaStream_t st = c->lane[li];
        char* base = (char*)c->stage + lane_b * li;
        const uint64_t off = k * chunk, cn = std::min(chunk, n - off);
        float* dv[6] = {};
        for (int i = 0; i < nin && e == cudaSuccess; ++i) {
            dv[i] = (float*)(base + fb * i);
            e = cudaMemcpyAsync(dv[i], hv[i] + off, cn * 4, cudaMemcpyHostToDevice, st);
        }
        if (e != cudaSuccess) { first = cuda_fail(c, e, "host->device copy"); break; }
        stf_queries dq{cn, q->id_base + off, dv[0], dv[1], nullptr};
        stf_derivs dd{};
        if (d) dd = stf_derivs{dv[2], dv[3], dv[4], dv[5]};
        float* dout3[3] = {(float*)(base + fb * nin), (float*)(base + fb * (nin + 1)), (float*)(base + fb * (nin + 2))};
        uint32_t* dpk = out->picks ? (uint32_t*)(base + fb * (nin + 3)) : nullptr;
        stf_output dout{dout3[0], dout3[1], dout3[2], dpk};
        first = enqueue_filter(c, *rec, &dq, d ? &dd : nullptr, f, m, sh, spp, seed, flags, &dout, st);
        if (first != STF_OK) break;
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(ho[i] + off, dout3[i], cn * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && dpk)
            e = cudaMemcpyAsync(out->picks + off * spp * 2, dpk, cn * spp * 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) first = cuda_fail(c, e, "device->host copy");
    }
    // every lane drains before returning (also after an error: staging stays in use until
    // then); an asynchronous call leaves them running, and the next call's chunks queue behind
    for (int i = 0; i < lanes && e == cudaSuccess && first == STF_OK; ++i) {
        e = cudaEventRecord(c->lane_ev[i], c->lane[i]);
        if (e != cudaSuccess) first = cuda_fail(c, e, "lane event");
    }
    if (async && first == STF_OK) return STF_OK;
    for (int i = 0; i < lanes; ++i) {
        cudaError_t ei = cudaStreamSynchronize(c->lane[i]);
        if (ei != cudaSuccess && first == STF_OK) first = cuda_fail(c, ei, "lane synchronise");
    }
    return first;
}

stf_status stf_filter_shade_host(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d,
                                 stf_filter f, stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed,
                                 uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_filter_shade_host");
    return host_pipeline(c, t, q, d, f, m, sh, spp, seed, flags, out, false);
}

stf_status stf_filter_shade_host_async(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d,
                                       stf_filter f, stf_mode m, stf_shade sh, uint32_t spp, uint64_t seed,
                                       uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_filter_shade_host_async");
    return host_pipeline(c, t, q, d, f, m, sh, spp, seed, flags, out, true);
}

// ---------------------------------------------------------------------------- texture table
stf_status stf_create_texture_table(stf_ctx c, uint32_t n, const stf_tex* textures, stf_table* out) {
    if (!c || !textures || !out) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    *out = 0;
    if (n < 1 || n > (1u << 20)) return fail(c, STF_ERR_INVALID_ARG, "table size must be 1..2^20");
    std::vector<stf::FetchCtx> host(n);
    for (uint32_t i = 0; i < n; ++i) {
        auto it = c->tex.find(textures[i]);
        if (it == c->tex.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown texture handle in table");
        if (it->second.view.fmt == stf::FMT_DCT)
            return fail(c, STF_ERR_UNSUPPORTED, "texture tables take RGBA32F and RGBA8 textures");
        host[i] = stf::make_fetch_ctx(it->second.view);
    }
    CurrentDevice cd(c->device);
    TableRec rec;
    rec.n = n;
    rec.members.assign(textures, textures + n);
    const size_t bytes = (size_t)n * sizeof(stf::FetchCtx);
    const size_t cnt_off = (bytes + 255) & ~(size_t)255;
    stf_status s = dev_alloc(c, &rec.mem, cnt_off + 256);
    if (s != STF_OK) return s;
    rec.counter = (unsigned long long*)((char*)rec.mem + cnt_off);
    cudaError_t e = cudaMemcpyAsync(rec.mem, host.data(), bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { cudaFree(rec.mem); return cuda_fail(c, e, "table upload"); }
    const uint64_t h = c->next_handle++;
    c->tables[h] = std::move(rec);
    *out = h;
    return STF_OK;
}

stf_status stf_destroy_texture_table(stf_ctx c, stf_table t) {
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->tables.find(t);
    if (it == c->tables.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown table handle");
    CurrentDevice cd(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(it->second.mem);
    c->tables.erase(it);
    return STF_OK;
}

stf_status stf_filter_shade_table(stf_ctx c, stf_table t, const stf_queries* q, const uint32_t* tex_id,
                                  const stf_derivs* d, stf_filter f, stf_mode m, stf_shade sh, uint32_t spp,
                                  uint64_t seed, uint32_t flags, const stf_output* out) {
    stfi::NvtxRange nvtx_range("stf_filter_shade_table");
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->tables.find(t);
    if (it == c->tables.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown table handle");
    if (c->tex.empty()) return fail(c, STF_ERR_BAD_HANDLE, "no textures");
    if (f == STF_FILTER_EWA || (flags & STF_FLAG_LOD0))
        return fail(c, STF_ERR_UNSUPPORTED, "the texture table takes the separable filters and no LOD0 flag");
    // validate everything but the texture handle with the regular checks
    TexRec* any = nullptr;
    stf_status s = validate_filter_call(c, c->tex.begin()->first, q, d, f, m, sh, spp, flags, out, &any);
    if (s != STF_OK || q->n == 0) return s;
    if (!tex_id || !aligned4(tex_id)) return fail(c, STF_ERR_INVALID_ARG, "tex_id must be non-null and 4-byte aligned");
    if (c->fault == FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    CurrentDevice cd(c->device);
    stf::FilterShadeArgs a{};
    a.n = q->n; a.id_base = q->id_base; a.u = q->u; a.v = q->v; a.order = q->order;
    a.has_derivs = d ? 1 : 0;
    if (d) { a.dudx = d->dudx; a.dvdx = d->dvdx; a.dudy = d->dudy; a.dvdy = d->dvdy; }
    a.filter = f; a.mode = m; a.shade = sh; a.spp = spp; a.flags = flags;
    a.kside = (flags & STF_FLAG_STRATIFIED) ? square_side(spp) : 1;
    a.seed = seed; a.r = out->r; a.g = out->g; a.b = out->b; a.picks = out->picks;
    a.status = c->d_status;
    cudaError_t e = cudaMemsetAsync(it->second.counter, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess)
        e = stf::launch_filter_shade_table(a, (const stf::FetchCtx*)it->second.mem, it->second.n, tex_id,
                                           it->second.counter, c->num_sms, c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "filter_shade_table launch");
}

// ----------------------------------------------------------------------------- binning
stf_status stf_bin_queries(stf_ctx c, uint64_t n, const float* u, const float* v, const uint32_t* tex_id,
                           uint32_t ntex, uint32_t tile_log2, uint32_t* order_out) {
    stfi::NvtxRange nvtx_range("stf_bin_queries");
    if (!c) return STF_ERR_INVALID_ARG;
    if (n == 0) return STF_OK;
    if (!u || !v || !order_out || !aligned4(u) || !aligned4(v) || !aligned4(order_out))
        return fail(c, STF_ERR_INVALID_ARG, "u, v and order must be non-null and 4-byte aligned");
    if (n >= (1ull << 32)) return fail(c, STF_ERR_INVALID_ARG, "at most 2^32 - 1 queries");
    if (!tex_id) ntex = 1;
    if (ntex < 1 || tile_log2 > 12 || (uint64_t)ntex << (2 * tile_log2) > (1ull << 26))
        return fail(c, STF_ERR_INVALID_ARG, "ntex * 4^tile_log2 must be in 1..2^26");
    if (c->fault == FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    CurrentDevice cd(c->device);
    const uint64_t nbins = (uint64_t)ntex << (2 * tile_log2);
    const uint64_t nblk = (nbins + 1023) / 1024;
    stf_status s = ensure_bin_scratch(c, (nblk * 1024 + nblk) * 4);
    if (s != STF_OK) return s;
    cudaError_t e = stf::launch_bin_queries(n, u, v, tex_id, ntex, tile_log2, order_out, (uint32_t*)c->bin_scratch, nbins,
                                            c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "bin launch");
}

// --------------------------------------------------------------------------------- volume
stf_status stf_create_volume(stf_ctx c, uint32_t nx, uint32_t ny, uint32_t nz, stf_format fmt,
                             float sigma_scale, const void* data, int on_device, stf_vol* out) {
    stfi::NvtxRange nvtx_range("stf_create_volume");
    if (!c || !data || !out) return fail(c, STF_ERR_INVALID_ARG, "null argument");
    *out = 0;
    if (fmt != STF_FMT_R16F) return fail(c, STF_ERR_INVALID_ARG, "volumes are R16F");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024)
        return fail(c, STF_ERR_INVALID_ARG, "volume size must be 1..1024 per axis");
    if (!(sigma_scale >= 0.0f) || std::isinf(sigma_scale)) return fail(c, STF_ERR_INVALID_ARG, "sigma_scale must be finite and >= 0");
    CurrentDevice cd(c->device);
    VolRec rec;
    rec.nx = nx; rec.ny = ny; rec.nz = nz; rec.sigma_scale = sigma_scale;
    const size_t bytes = (size_t)nx * ny * nz * 2;
    stf_status s = dev_alloc(c, &rec.mem, bytes);
    if (s != STF_OK) return s;
    const size_t pbytes = (size_t)stf::vol_pad_pitch(nx) * (ny + 2 * stf::VOL_PAD) * (nz + 2 * stf::VOL_PAD) * 2;
    s = dev_alloc(c, &rec.pad, pbytes);
    if (s != STF_OK) { cudaFree(rec.mem); return s; }
    unsigned int* d_max = nullptr;
    s = dev_alloc(c, (void**)&d_max, sizeof(unsigned int));
    if (s != STF_OK) { cudaFree(rec.mem); cudaFree(rec.pad); return s; }
    unsigned int max_bits = 0x7C00u;
    cudaError_t e = cudaMemcpyAsync(rec.mem, data, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = stf::launch_pad_volume(rec.mem, (int)nx, (int)ny, (int)nz, rec.pad, c->stream);
    if (e == cudaSuccess) e = stf::launch_vol_max_bits(rec.mem, bytes / 2, d_max, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&max_bits, d_max, sizeof(max_bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_max);
    if (e != cudaSuccess) { cudaFree(rec.mem); cudaFree(rec.pad); return cuda_fail(c, e, "volume upload"); }
    __half_raw hr;
    hr.x = (unsigned short)max_bits;
    rec.dmax = max_bits >= 0x7C00u ? INFINITY : __half2float(__half(hr));
    rec.tmap_ok = stf::encode_volume_tmap(&rec.tmap, rec.mem, (int)nx, (int)ny, (int)nz);
    const uint64_t h = c->next_handle++;
    c->vol[h] = rec;
    *out = h;
    return STF_OK;
}

stf_status stf_destroy_volume(stf_ctx c, stf_vol v) {
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->vol.find(v);
    if (it == c->vol.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown volume handle");
    CurrentDevice cd(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(it->second.mem);
    cudaFree(it->second.pad);
    c->vol.erase(it);
    return STF_OK;
}

stf_status stf_march_volume(stf_ctx c, stf_vol v, const float* cam, uint32_t width, uint32_t height,
                            uint32_t steps, stf_filter f, stf_mode m, uint32_t spp, uint64_t seed,
                            uint32_t flags, uint64_t pix_begin, uint64_t pix_count, float* out_T,
                            uint32_t* out_picks) {
    stfi::NvtxRange nvtx_range("stf_march_volume");
    if (!c) return STF_ERR_INVALID_ARG;
    auto it = c->vol.find(v);
    if (it == c->vol.end()) return fail(c, STF_ERR_BAD_HANDLE, "unknown volume handle");
    if (!cam) return fail(c, STF_ERR_INVALID_ARG, "camera is null");
    if (f != STF_FILTER_LINEAR && f != STF_FILTER_BSPLINE) return fail(c, STF_ERR_UNSUPPORTED, "volumes use LINEAR or BSPLINE");
    if (m != STF_MODE_NTAP_BEFORE && m != STF_MODE_NTAP_AFTER && m != STF_MODE_STOCHASTIC)
        return fail(c, STF_ERR_UNSUPPORTED, "volume mode must be NTAP_BEFORE, NTAP_AFTER or STOCHASTIC");
    if (width < 1 || height < 1 || steps < 1 || steps > 65535 || spp < 1) return fail(c, STF_ERR_INVALID_ARG, "bad image size, steps or spp");
    if (flags & ~(uint32_t)(STF_FLAG_STRATIFIED | STF_FLAG_LATTICE | STF_FLAG_REUSE)) return fail(c, STF_ERR_INVALID_ARG, "unknown flag bits");
    if ((flags & STF_FLAG_STRATIFIED) && square_side(spp) < 0) return fail(c, STF_ERR_INVALID_ARG, "stratified jitter needs a square spp");
    if (pix_begin + pix_count > (uint64_t)width * height) return fail(c, STF_ERR_INVALID_ARG, "pixel range outside the image");
    if (pix_count == 0) return STF_OK;
    if (!out_T || !aligned4(out_T) || (out_picks && !aligned4(out_picks))) return fail(c, STF_ERR_INVALID_ARG, "bad output pointer");
    if (c->fault == FAULT_LAUNCH) return fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");
    CurrentDevice cd(c->device);
    stf::MarchArgs a{};
    a.vox = (const __half*)it->second.mem;
    a.nx = (int)it->second.nx; a.ny = (int)it->second.ny; a.nz = (int)it->second.nz;
    a.px = (int)stf::vol_pad_pitch(it->second.nx);
    a.pxy = a.px * (a.ny + 2 * stf::VOL_PAD);
    a.vpad = (const __half*)it->second.pad + (size_t)stf::VOL_PAD * ((size_t)a.pxy + a.px + 1);
    a.fixed32 = (double)steps * it->second.dmax < 256.0 ? 1 : 0;
    a.sigma_scale = it->second.sigma_scale;
    for (int i = 0; i < 12; ++i) a.cam[i] = cam[i];
    a.width = width; a.height = height; a.steps = steps; a.spp = spp; a.flags = flags;
    a.kside = (flags & STF_FLAG_STRATIFIED) ? square_side(spp) : 1;
    a.filter = f; a.mode = m; a.seed = seed; a.pix_begin = pix_begin; a.pix_count = pix_count;
    // 8 x 4 pixel tiles per warp where they measured faster at 1920x1080 x 8 spp (1-tap: 2-5 %,
    // tricubic filter-after: 17 %); filter-before keeps row order (tiles: tricubic +-0 %,
    // trilinear 15 % slower)
    const uint64_t band = 4ull * width;
    a.tiled = (m != STF_MODE_NTAP_BEFORE && width % 8 == 0 && pix_begin % band == 0 && pix_count % band == 0) ? 1 : 0;
    a.T = out_T; a.picks = out_picks; a.status = c->d_status;
    cudaError_t e = stf::launch_march(a, it->second.tmap_ok ? &it->second.tmap : nullptr, c->num_sms, c->stream);
    return e == cudaSuccess ? STF_OK : cuda_fail(c, e, "march launch");
}

}  // extern "C"

// ------------------------------------------------------------------------ upload packing
namespace stf {
// RGBA8 albedo+roughness and RG8 normal -> one 8-byte texel, so that a stochastic lookup
// touches a single 32-byte sector.
__global__ void k_pack_rgba8(const uint32_t* rgba, const uint16_t* rg, uint2* out, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = make_uint2(rgba[i], rg ? (uint32_t)rg[i] : 0x8080u);
}
cudaError_t launch_pack_rgba8(const void* rgba, const void* rg, void* out, uint64_t n, cudaStream_t st) {
    const uint64_t g = (n + 255) / 256;
    k_pack_rgba8<<<(int)(g < 4096 ? (g ? g : 1) : 4096), 256, 0, st>>>((const uint32_t*)rgba, (const uint16_t*)rg, (uint2*)out, n);
    return cudaGetLastError();
}
}  // namespace stf
