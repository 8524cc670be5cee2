// Host-buffer filter + shade that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they need a lookup: a renderer's frame loop
// whose device memory is budgeted up front (cudaMalloc may synchronise the device or fail
// under memory pressure), or a plug-in running inside a host application that owns every
// device allocation.  stf_filter_shade_host grows a context-owned staging buffer with
// cudaMalloc on demand; this entry point instead stages queries, results and the device
// status word in one fixed, file-scope device array, so a call never allocates.
//
// The array is a static __device__ object: every GPU that loads the library holds it (a
// little over 9 MiB) until the process exits.  In host code its name is only a host-side
// stand-in, so its device address is looked up once per device with cudaGetSymbolAddress.
#include <cstring>
#include <mutex>

#include "stf_ctx.h"

namespace {

constexpr uint64_t NOALLOC_MAX_QUERIES = 1ull << 18;              // queries per call
constexpr size_t NOALLOC_HEADER = 256;                            // status word, padded
constexpr size_t NOALLOC_ARRAY = NOALLOC_MAX_QUERIES * 4;         // one float per query
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + 9 * NOALLOC_ARRAY;   // u v 4 derivs r g b

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on `device` (which must be current); looked up on
// the first call per device.
stf_status scratch_address(stf_ctx c, unsigned char** out) {
    if (c->device < 0 || c->device >= MAX_DEVICES) return stfi::fail(c, STF_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[c->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return stfi::cuda_fail(c, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
        }
        g_scratch_addr[c->device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[c->device];
    return STF_OK;
}

}  // namespace

extern "C" stf_status stf_filter_shade_host_noalloc(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d,
                                                    stf_filter f, stf_mode m, stf_shade sh, uint32_t spp,
                                                    uint64_t seed, uint32_t flags, const stf_output* out) {
    // the same argument checks as stf_filter_shade_host (every filter, mode and flag it takes)
    TexRec* rec = nullptr;
    int kside = 1;
    stf_status vs = stfi::validate_filter_args(c, t, q, d, f, m, sh, spp, flags, out, &rec, &kside);
    if (vs != STF_OK) return vs;
    if (out->picks) return stfi::fail(c, STF_ERR_UNSUPPORTED, "the no-allocation entry point does not report picks");
    if (q->n > NOALLOC_MAX_QUERIES)
        return stfi::fail(c, STF_ERR_INVALID_ARG,
                          "stf_filter_shade_host_noalloc: at most 262144 queries per call (split larger batches)");
    if (q->n == 0) return STF_OK;
    if (q->order) return stfi::fail(c, STF_ERR_UNSUPPORTED, "the host-buffer entry points take no execution order");
    if (c->fault == stfi::FAULT_LAUNCH) return stfi::fail(c, STF_ERR_CUDA, "injected launch failure (STF_FAULT=launch)");

    stfi::CurrentDevice cd(c->device);
    unsigned char* base = nullptr;
    stf_status s = scratch_address(c, &base);
    if (s != STF_OK) return s;
    const uint64_t n = q->n;
    uint32_t* status = reinterpret_cast<uint32_t*>(base);
    float* arr[9];
    for (int i = 0; i < 9; ++i) arr[i] = reinterpret_cast<float*>(base + NOALLOC_HEADER + i * NOALLOC_ARRAY);
    const float* hin[6] = {q->u, q->v, d ? d->dudx : nullptr, d ? d->dvdx : nullptr, d ? d->dudy : nullptr,
                           d ? d->dvdy : nullptr};
    // the status word must start at zero; the staged arrays are fully overwritten
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(uint32_t), c->stream);
    for (int i = 0; i < (d ? 6 : 2) && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(arr[i], hin[i], n * 4, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return stfi::cuda_fail(c, e, "host->device copy");

    stf::FilterShadeArgs a{};
    a.n = n; a.id_base = q->id_base; a.u = arr[0]; a.v = arr[1];
    a.has_derivs = d ? 1 : 0;
    if (d) { a.dudx = arr[2]; a.dvdx = arr[3]; a.dudy = arr[4]; a.dvdy = arr[5]; }
    a.filter = f; a.mode = m; a.shade = sh; a.spp = spp; a.flags = flags; a.kside = kside;
    a.seed = seed; a.r = arr[6]; a.g = arr[7]; a.b = arr[8]; a.picks = nullptr;
    a.status = status;
    a.ewa_lut = c->d_ewa_lut;       // allocated with the context: the call still allocates nothing
    e = stf::launch_filter_shade(a, rec->view, c->num_sms, c->stream);
    if (e != cudaSuccess) return stfi::cuda_fail(c, e, "filter_shade launch");
    uint32_t st = 0;
    e = cudaMemcpyAsync(out->r, arr[6], n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->g, arr[7], n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->b, arr[8], n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return stfi::cuda_fail(c, e, "device->host copy");
    if (st) return stfi::fail(c, STF_ERR_DEVICE_STATUS, "device status bits set (e.g. NaN input)");
    return STF_OK;
}
