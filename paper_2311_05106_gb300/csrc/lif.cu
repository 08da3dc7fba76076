// lif.cu -- fused COBA / exponential-synapse / LIF step with spike-list
// compaction (a1-a4), and dense-event compaction.
//
// One pass over the neuron state (structure of arrays, FP32): decay and event
// add of both conductances (Appendix E), COBA current with the pre-update
// potential (Appendix F), exponential-Euler membrane update with refractory
// clamp, threshold and reset.  Spiking neurons are compacted per CTA into a
// shared-memory buffer (warp ballot + popcount, block prefix) and appended to
// the global spike list with one atomic per CTA flush, so the list costs a
// handful of L2 atomics per step instead of one per warp.
#include "bp_common.cuh"
#include "bp_internal.h"

namespace bp {
namespace {

constexpr int kLifThreads = 256;
constexpr int kLifWarps = kLifThreads / 32;
constexpr int kSpikeBuf = 2048;

struct SpikeStage {
    int32_t ids[kSpikeBuf];
    int32_t warp_cnt[kLifWarps];
    int32_t base;
    int32_t red[2][kLifWarps];
};

// Adds this iteration's spikes (flag s, id i) to the CTA buffer; `count` is
// the buffer fill, identical in every thread.  Ends with a barrier.
__device__ __forceinline__ void stage_spikes(SpikeStage& st, bool s, int64_t i, int& count) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(FULL_MASK, s);
    if (lane == 0) st.warp_cnt[warp] = __popc(m);
    __syncthreads();
    int off = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kLifWarps; ++w) {
        const int c = st.warp_cnt[w];
        off += (w < warp) ? c : 0;
        total += c;
    }
    if (s) st.ids[count + off + __popc(m & lanemask_lt())] = static_cast<int32_t>(i);
    count += total;
    __syncthreads();
}

// Appends the CTA buffer to the global list (one atomic) and empties it.
// Positions at or beyond `cap` (a counter that was not zeroed) are dropped.
__device__ __forceinline__ void flush_spikes(SpikeStage& st, int& count, int32_t* spike_list, int32_t* n_spikes,
                                             int64_t cap) {
    if (count == 0) return;  // uniform across the CTA
    if (threadIdx.x == 0) st.base = atomicAdd(n_spikes, count);
    __syncthreads();
    const int64_t base = st.base;
    for (int k = threadIdx.x; k < count; k += kLifThreads)
        if (base + k >= 0 && base + k < cap) spike_list[base + k] = st.ids[k];
    count = 0;
    __syncthreads();
}

template <bool COUNTS>
__global__ void __launch_bounds__(kLifThreads) k_lif_step(
    LifConst c, int64_t n, int64_t n_e, float* __restrict__ V, float* __restrict__ ge,
    float* __restrict__ gi, int32_t* __restrict__ ref, void* __restrict__ ye_, void* __restrict__ yi_,
    const float* __restrict__ I_vec, uint8_t* __restrict__ spk, int32_t* __restrict__ spike_list,
    int32_t* __restrict__ n_spikes, int32_t* __restrict__ clear_counter, int64_t* __restrict__ totals,
    const NetCtrl* __restrict__ ctrl, int32_t t_local) {
    __shared__ SpikeStage st;
    using Y = typename std::conditional<COUNTS, int32_t, float>::type;
    Y* __restrict__ ye = static_cast<Y*>(ye_);
    Y* __restrict__ yi = static_cast<Y*>(yi_);
    if (clear_counter && blockIdx.x == 0 && threadIdx.x == 0) *clear_counter = 0;

    int count = 0;
    int cnt_e = 0, cnt_i = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kLifThreads;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kLifThreads; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool s = false;
        if (i < n) {
            const Y ce = ye[i], ci = yi[i];
            float add_e, add_i;
            if constexpr (COUNTS) {
                add_e = c.w_e * static_cast<float>(ce);
                add_i = c.w_i * static_cast<float>(ci);
            } else {
                add_e = ce;
                add_i = ci;
            }
            if (ce != Y(0)) ye[i] = Y(0);
            if (ci != Y(0)) yi[i] = Y(0);
            const float g_e = ge[i] * c.a_e + add_e;
            const float g_i = gi[i] * c.a_i + add_i;
            ge[i] = g_e;
            gi[i] = g_i;
            float v = V[i];
            float I = g_e * (c.E_e - v) + g_i * (c.E_i - v) + c.I_ext;
            if (I_vec) I += I_vec[i];
            const int32_t r = ref[i];
            if (r > 0) {
                ref[i] = r - 1;
            } else {
                const float v_inf = c.V_rest + c.R * I;
                v = v_inf + (v - v_inf) * c.a_m;
                if (v > c.V_th) {
                    s = true;
                    v = c.V_reset;
                    ref[i] = c.ref_steps;
                }
                V[i] = v;
            }
            if (spk) spk[i] = s ? 1 : 0;
            if (s) {
                if (i < n_e) ++cnt_e; else ++cnt_i;
            }
        }
        if (count + kLifThreads > kSpikeBuf) flush_spikes(st, count, spike_list, n_spikes, n);
        stage_spikes(st, s, i, count);
    }
    flush_spikes(st, count, spike_list, n_spikes, n);

    if (totals || ctrl) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        cnt_e = group_reduce_sum(cnt_e, 32);
        cnt_i = group_reduce_sum(cnt_i, 32);
        if (lane == 0) {
            st.red[0][warp] = cnt_e;
            st.red[1][warp] = cnt_i;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int se = 0, si = 0;
            for (int w = 0; w < kLifWarps; ++w) {
                se += st.red[0][w];
                si += st.red[1][w];
            }
            if (totals && (se | si)) {
                atomicAdd(reinterpret_cast<unsigned long long*>(totals + 0), static_cast<unsigned long long>(se));
                atomicAdd(reinterpret_cast<unsigned long long*>(totals + 1), static_cast<unsigned long long>(si));
            }
            if (ctrl && ctrl->record && (se | si)) {
                const int64_t idx = ctrl->step + t_local - ctrl->record_base;
                if (idx >= 0 && idx < ctrl->record_len) {
                    atomicAdd(ctrl->record + 2 * idx, se);
                    atomicAdd(ctrl->record + 2 * idx + 1, si);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kLifThreads) k_spike_compact(int64_t n, const uint8_t* __restrict__ events,
                                                              int32_t* __restrict__ spike_list,
                                                              int32_t* __restrict__ n_spikes) {
    __shared__ SpikeStage st;
    int count = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kLifThreads;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kLifThreads; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool s = (i < n) && events[i] != 0;
        if (count + kLifThreads > kSpikeBuf) flush_spikes(st, count, spike_list, n_spikes, n);
        stage_spikes(st, s, i, count);
    }
    flush_spikes(st, count, spike_list, n_spikes, n);
}

int lif_grid(int64_t n) {
    const int64_t need = (n + kLifThreads - 1) / kLifThreads;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    const int64_t g = need < cap ? need : cap;
    return static_cast<int>(g > 0 ? g : 1);
}

}  // namespace

bp_status launch_lif_step(const LifConst& c, int64_t n, int64_t n_e, float* V, float* ge, float* gi,
                          int32_t* ref, void* ye, void* yi, bool counts, const float* I_vec, uint8_t* spk,
                          int32_t* spike_list, int32_t* n_spikes, int32_t* clear_counter, int64_t* totals,
                          const NetCtrl* ctrl, int32_t t_local, cudaStream_t s) {
    if (n == 0) {
        if (clear_counter) BP_CUDA(cudaMemsetAsync(clear_counter, 0, sizeof(int32_t), s));
        return BP_OK;
    }
    const int grid = lif_grid(n);
    if (counts)
        k_lif_step<true><<<grid, kLifThreads, 0, s>>>(c, n, n_e, V, ge, gi, ref, ye, yi, I_vec, spk, spike_list,
                                                      n_spikes, clear_counter, totals, ctrl, t_local);
    else
        k_lif_step<false><<<grid, kLifThreads, 0, s>>>(c, n, n_e, V, ge, gi, ref, ye, yi, I_vec, spk, spike_list,
                                                       n_spikes, clear_counter, totals, ctrl, t_local);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status launch_spike_compact(int64_t n, const uint8_t* events, int32_t* spike_list, int32_t* n_spikes,
                               cudaStream_t s) {
    if (n == 0) return BP_OK;
    k_spike_compact<<<lif_grid(n), kLifThreads, 0, s>>>(n, events, spike_list, n_spikes);
    BP_LAUNCHED();
    return BP_OK;
}

}  // namespace bp

extern "C" {

bp_status bp_lif_step(const bp_coba_params* p, int64_t n, int64_t n_e, float* V, float* ge, float* gi,
                      int32_t* ref, void* ye, void* yi, int32_t y_is_count, const float* I_vec, uint8_t* spk,
                      int32_t* spike_list, int32_t* n_spikes, int64_t* spike_totals, bp_stream_t stream) {
    bp::clear_error();
    BP_TRY(bp::check_coba(p));
    BP_REQUIRE(n >= 0 && n <= INT32_MAX, "n = %lld out of range", (long long)n);
    BP_REQUIRE(n_e >= 0 && n_e <= n, "n_e = %lld not in [0, n]", (long long)n_e);
    BP_REQUIRE(n == 0 || (V && ge && gi && ref && ye && yi && spike_list && n_spikes),
               "a required state pointer is NULL");
    const bp::LifConst c = bp::make_lif_const(*p);
    return bp::launch_lif_step(c, n, n_e, V, ge, gi, ref, ye, yi, y_is_count != 0, I_vec, spk, spike_list,
                               n_spikes, nullptr, spike_totals, nullptr, 0, stream);
}

bp_status bp_spike_compact(int64_t n, const uint8_t* events, int32_t* spike_list, int32_t* n_spikes,
                           bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n >= 0 && n <= INT32_MAX, "n = %lld out of range", (long long)n);
    BP_REQUIRE(n == 0 || (events && spike_list && n_spikes), "a required pointer is NULL");
    return bp::launch_spike_compact(n, events, spike_list, n_spikes, stream);
}

}  // extern "C"
