// Internal: the context object and helpers shared by the C-ABI translation units.
#pragma once
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/stf.h"
#include "stf_kernels.h"

enum { STF_LANES = 3 };

struct TexRec {
    void* mem = nullptr;
    stf::TexView view{};
};
struct VolRec {
    void* mem = nullptr;
    void* pad = nullptr;            // the voxels with a clamped two-voxel border (launch_pad_volume)
    uint32_t nx = 0, ny = 0, nz = 0;
    float sigma_scale = 1.0f;
    float dmax = 0.0f;              // largest density (0 for none; infinite for inf or NaN voxels)
    CUtensorMap tmap{};             // the voxels as a TMA tensor (valid when tmap_ok)
    bool tmap_ok = false;
};
struct NeuralRec {
    void* mem = nullptr;           // one allocation for every array below
    stf::NeuralView view{};
    uint64_t lat_total = 0;        // latent elements over all grids
    float *m_lat = nullptr, *v_lat = nullptr, *m_mlp = nullptr, *v_mlp = nullptr;
    unsigned int* amax = nullptr;  // FP8 scale reduction
    float* loss = nullptr;         // per-step losses (grown on demand)
    uint32_t loss_cap = 0;
    uint32_t step = 0;             // optimiser steps taken
    int latent_fmt = 0;
    bool trainable = false;
};

struct TableRec {
    void* mem = nullptr;              // FetchCtx[n] followed by the 8-byte work counter
    uint32_t n = 0;
    std::vector<uint64_t> members;    // texture handles (they must outlive the table)
    unsigned long long* counter = nullptr;
};

struct stf_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 148;
    uint32_t* d_status = nullptr;
    float* d_ewa_lut = nullptr;     // EWA Gaussian weight table (128 floats)
    std::string last_error;
    uint64_t next_handle = 1;
    std::unordered_map<uint64_t, TexRec> tex;
    std::unordered_map<uint64_t, VolRec> vol;
    std::unordered_map<uint64_t, NeuralRec> neural;
    std::unordered_map<uint64_t, TableRec> tables;
    void* stage = nullptr;          // device staging for the host-buffer entry points (lanes only)
    size_t stage_bytes = 0;
    void* bin_scratch = nullptr;    // histogram scratch of stf_bin_queries (context stream only)
    size_t bin_scratch_bytes = 0;
    cudaStream_t lane[STF_LANES] = {};   // copy-pipeline streams of the host-buffer path
    cudaEvent_t entry_ev = nullptr;      // orders the lanes after the caller's stream
    cudaEvent_t lane_ev[STF_LANES] = {}; // end of each lane's work in the latest host-buffer call
    size_t lane_bytes = 0;               // staging bytes per lane in the latest host-buffer call
    int fault = 0;                  // host-side fault injection (STF_FAULT), 0 = off
};

namespace stfi {
enum { FAULT_NONE = 0, FAULT_ALLOC = 1, FAULT_LAUNCH = 2, FAULT_MMA_TIMEOUT = 3 };
stf_status fail(stf_ctx c, stf_status s, const char* msg);
stf_status cuda_fail(stf_ctx c, cudaError_t e, const char* where);
stf_status dev_alloc(stf_ctx c, void** p, size_t bytes);
// The argument checks of stf_filter_shade and the host-buffer entry points (handles, enums,
// flags, spp, pointer alignment); *kside = the side of the stratified jitter grid (1 without
// STF_FLAG_STRATIFIED).  q->n == 0 passes without checking the pointers.
stf_status validate_filter_args(stf_ctx c, stf_tex t, const stf_queries* q, const stf_derivs* d, stf_filter f,
                                stf_mode m, stf_shade sh, uint32_t spp, uint32_t flags, const stf_output* out,
                                TexRec** rec, int* kside);
// Names an entry point's host-side span in a profiler's timeline (NVTX ranges; no cost
// beyond a function-pointer test unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev) { cudaGetDevice(&prev); if (prev != dev) cudaSetDevice(dev); }
    ~CurrentDevice() { int now = -1; cudaGetDevice(&now); if (prev >= 0 && now != prev) cudaSetDevice(prev); }
};
}  // namespace stfi
