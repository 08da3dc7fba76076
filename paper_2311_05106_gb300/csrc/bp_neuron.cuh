// bp_neuron.cuh -- the per-neuron COBA / exponential-synapse / LIF update
// shared by the single-network and the batched kernels, so that both paths
// perform the identical FP32 arithmetic.
#pragma once

#include "bp_common.cuh"
#include "bp_internal.h"

namespace bp {

// One neuron and one step; returns true if it spikes.
//   g_e <- g_e a_e + add_e, g_i <- g_i a_i + add_i       (Appendix E)
//   I = g_e (E_e - V) + g_i (E_i - V) + I_ext + I_add    (Appendix F, pre-update V)
//   refractory: counter down, V held; otherwise exponential Euler
//   V <- V_inf + (V - V_inf) a_m, V_inf = V_rest + R I; spike if V > V_th.
__device__ __forceinline__ bool neuron_update(const LifConst& c, float& v, float& g_e, float& g_i, int32_t& r,
                                              float add_e, float add_i, float I_add) {
    g_e = g_e * c.a_e + add_e;
    g_i = g_i * c.a_i + add_i;
    const float I = g_e * (c.E_e - v) + g_i * (c.E_i - v) + c.I_ext + I_add;
    if (r > 0) {
        r -= 1;
        return false;
    }
    const float v_inf = c.V_rest + c.R * I;
    v = v_inf + (v - v_inf) * c.a_m;
    if (v > c.V_th) {
        v = c.V_reset;
        r = c.ref_steps;
        return true;
    }
    return false;
}

// Conductance increment from an accumulator entry: w * count for integer
// event counts, the weighted sum itself otherwise.
template <bool COUNTS>
__device__ __forceinline__ float event_add(typename std::conditional<COUNTS, int32_t, float>::type y, float w) {
    if constexpr (COUNTS) {
        return w * static_cast<float>(y);
    } else {
        return y;
    }
}

}  // namespace bp
