// bp_internal.h -- declarations shared between libbp's translation units
// (host-side launchers and parameter structs).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bp.h"

#include <nvtx3/nvToolsExt.h>

namespace bp {

// Host-side NVTX range around an entry point (a no-op unless a tool such as
// a profiler is attached; ncu --nvtx can filter kernels by these ranges).
// Raises a kernel's dynamic shared-memory limit to `bytes` (once per kernel,
// device and size; defined in lib.cu).
bp_status ensure_smem_attr(const void* kernel, int bytes);

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


// Post neurons per shared-memory tile: 54 944 4-byte accumulators (214.6 KiB)
// fit one CTA per SM under the 227 KiB opt-in limit together with the event
// product's per-warp segment tables (12.3 KiB: 32 row segments per warp of a
// 1024-thread CTA).
constexpr int32_t kTileCols = 54944;
constexpr int kMaxSmemPerCta = 232448;  // 227 KiB opt-in limit of sm_100-class GPUs
constexpr int kTileThreads = 1024;

// FP32 constants of one COBA/LIF step; decay factors from FP64 exp().
struct LifConst {
    float a_m, a_e, a_i;
    float V_rest, V_th, V_reset, E_e, E_i, R, I_ext, w_e, w_i;
    int32_t ref_steps;
};

LifConst make_lif_const(const bp_coba_params& p);
bp_status check_coba(const bp_coba_params* p);

// Per-step control of a network simulation kept in device memory: kernels of
// a captured CUDA graph read the record pointer and the step number from it.
struct NetCtrl {
    int64_t step;          // steps completed since the last reset
    int64_t record_base;   // value of `step` when the current record began
    int32_t* record;       // [T][2] or NULL
    int64_t record_len;    // T
    uint32_t done_ctas;    // CTAs of the current step launch that have finished (the last advances `step`)
    uint32_t pad;
};

// Stored CSR operand of the event products.
struct CsrArgs {
    int64_t n_pre, n_post;
    const int64_t* indptr;
    const int32_t* indices;
    const void* data;
    int32_t wkind;
    float w_homo;
    const int32_t* tile_ptr;
    int32_t tile_cols;
    // the two bound slots at the end of the tile index (fixed-point tile
    // sums, BP_ACC_FIXED): [0] the weight bound b as FP32 bits, [1] the most
    // rows with an entry in one column (0: not recorded); NULL without a
    // tile index
    const int32_t* w_bound = nullptr;
};

// Accumulation mode of the event CSR product (launch_event_csrmv): 0 auto,
// 1 direct (global atomics), 2 shared tiles; kModeFixed or-ed in asks for
// fixed-point tile sums of float products.
constexpr int kModeFixed = 16;

// JIT operand (Appendix C): key, gap range, weight law.
struct JitArgs {
    uint64_t seed;
    uint32_t K;
    int32_t wkind;
    float w0, w1;
};

// One fused network step: neuron pass over [0, n) reading half `parity` of
// the double-buffered accumulators ye2 / yi2 ([2n] each) and delivering the
// step's spikes into the other half.
struct NetStepLaunch {
    LifConst c;
    int64_t n, n_e;
    float* V;
    float* ge;
    float* gi;
    uint8_t* ref;
    void* ye2;
    void* yi2;
    uint8_t* spk;
    int32_t* spike_list;   // nullable
    int32_t* n_spikes;     // [2], used with spike_list
    int64_t* totals;
    NetCtrl* ctrl;
    bool counts;
    bool jit;
    CsrArgs csr;
    int32_t group;         // lanes per CSR row in the delivery (4, 8, 16 or 32)
    JitArgs je, ji;
    // delay ring (a projection with delay > 0): ring_slots = max delay + 2
    // spike lists of n ids after ring_slots counts; 0 = no delayed projection
    int32_t* ring;
    int32_t ring_slots, delay_e, delay_i;
    // AlignPre form: presynaptic traces (NULL: AlignPost)
    float* trace;
};

// ---- lif.cu
bp_status launch_lif_step(const LifConst& c, int64_t n, int64_t n_e, float* V, float* ge, float* gi,
                          uint8_t* ref, void* ye, void* yi, bool counts, const float* I_vec, uint8_t* spk,
                          int32_t* spike_list, int32_t* n_spikes, int32_t* clear_counter,
                          int64_t* totals, const NetCtrl* ctrl, int32_t t_local, cudaStream_t s);
// advance > 0: the launch's last CTA to finish adds `advance` to the device
// step counter and to totals[3] (the last step of a captured chunk, or an
// eager step), so no separate kernel is needed for it.
bp_status launch_network_step(const NetStepLaunch& L, int parity, int32_t t_local, cudaStream_t s,
                              int32_t advance = 0);
bp_status launch_spike_compact(int64_t n, const uint8_t* events, int32_t* spike_list, int32_t* n_spikes,
                               cudaStream_t s);

// ---- csrmv.cu
// Scatter of the spiking rows' entries into y.  events_total (nullable) +=
// sum of spiking rows' lengths.  mode: 0 auto, 1 direct (global atomics),
// 2 shared tiles.
bp_status launch_event_csrmv(const CsrArgs& a, const int32_t* spike_list, const int32_t* n_spikes,
                             int64_t max_spikes, void* y, bool counts, int64_t* events_total, int mode,
                             cudaStream_t s);

// ---- tcgemm.cu
// G[s][a] (+)= sum_{b < B, t < T} X_bt[s] D_bt[a] on the tensor cores: D float
// [B][T][na]; X_bt[s] = x_dense[b][t][s] != 0 for s < n_dense, bit s - n_dense
// of z_bits[b][t - 1] (zw words per step, zero at t = 0) for the next n_bits
// features.  G row stride ldg.  work >= tc_spike_gemm_workspace(B, T, na,
// n_dense + n_bits) bytes, 1024-byte aligned.
size_t tc_spike_gemm_workspace(int32_t B, int32_t T, int32_t na, int32_t ns);
bp_status launch_tc_spike_gemm(int32_t B, int32_t T, const float* d, int32_t na, const uint8_t* x_dense,
                               int32_t n_dense, const uint32_t* z_bits, int32_t n_bits, int32_t zw, float* g,
                               int64_t ldg, bool accumulate, void* work, size_t work_bytes, cudaStream_t st);

// ---- jitconn.cu
// Scatter of JIT rows (row id = spike id) into y.
bp_status launch_jit_event_mv(const JitArgs& d, int64_t n_post, const int32_t* spike_list, const int32_t* n_spikes,
                              int64_t max_spikes, void* y, bool counts, int64_t* events_total, int mode,
                              cudaStream_t s);

}  // namespace bp
