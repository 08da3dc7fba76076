// bp_rows.cuh -- device routines that deliver one presynaptic row: the
// strided walk of a stored CSR segment and the warp-cooperative regeneration
// of a JIT row (Appendix B, Appendix C).  Shared by the operator kernels and
// the fused network step.
#pragma once

#include "bp_common.cuh"
#include "bp_internal.h"

namespace bp {

// Lanes per row: enough that a segment is one to two passes of the group.
__device__ __forceinline__ int pick_group(int64_t nnz, int64_t n_pre, int64_t tiles) {
    const int64_t denom = (n_pre > 0 ? n_pre : 1) * (tiles > 0 ? tiles : 1);
    const int64_t mean = nnz / denom;
    if (mean >= 48) return 32;
    if (mean >= 24) return 16;
    if (mean >= 12) return 8;
    return 4;
}

template <typename Acc>
__device__ __forceinline__ Acc event_value(float w) {
    if constexpr (std::is_same<Acc, int32_t>::value) {
        return 1;
    } else {
        return w;
    }
}

// Accumulation targets: plain atomics (shared memory or global), or global
// REDs that keep the target line in L2 (KEEP).
template <bool KEEP>
struct AccOp {
    uint64_t pol;
    __device__ __forceinline__ AccOp() : pol(KEEP ? l2_keep_policy() : 0ull) {}
    template <typename T>
    __device__ __forceinline__ void operator()(T* p, T v) const {
        if constexpr (KEEP) red_add_keep(p, v, pol); else acc_add(p, v);
    }
};

// out[indices[j] - col0] += value(w_j) for j = b0 + lane, b0 + lane + G, ...
// Each pass issues up to four predicated loads per lane before any atomic,
// so a row of up to 4 G entries costs one memory latency.
template <typename Acc, int WK, bool KEEP = false>
__device__ __forceinline__ void scatter_segment(const int32_t* __restrict__ indices, const void* __restrict__ data,
                                                float w_homo, int64_t b0, int64_t b1, int lane, int G,
                                                Acc* __restrict__ out, int64_t col0) {
    const AccOp<KEEP> add;
    for (int64_t j = b0 + lane; j < b1; j += 4 * G) {
        int32_t c[4];
        float w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t jj = j + u * G;
            c[u] = jj < b1 ? ld_stream(indices + jj) : -1;
            w[u] = jj < b1 ? load_weight<WK>(data, jj, w_homo) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c[u] >= 0) add(out + (c[u] - col0), event_value<Acc>(w[u]));
    }
}

// As scatter_segment, with 16-byte loads: the part of the segment between
// the first and last multiple of 4 is read as aligned groups of four entries
// (four groups per lane per pass, so 64 bytes of indices in flight per lane),
// the unaligned head and tail entry by entry.  Needs 16-byte aligned indices
// (and FP32 weights; 8-byte aligned BF16 weights).  The body is a
// load-then-accumulate loop whose next pass is loaded at the end of the
// current one (measured 7-15 % faster than the equivalent for loop on the
// n = 1e6 operator cells).
template <typename Acc, int WK>
__device__ __forceinline__ void scatter_segment_v4(const int32_t* __restrict__ indices, const void* __restrict__ data,
                                                   float w_homo, int64_t b0, int64_t b1, int lane, int G,
                                                   Acc* __restrict__ out, int64_t col0) {
    int64_t a4 = (b0 + 3) & ~int64_t(3);
    if (a4 > b1) a4 = b1;
    int64_t e4 = b1 & ~int64_t(3);
    if (e4 < a4) e4 = a4;
    // head and tail: at most 3 entries each
    {
        const int64_t nh = a4 - b0, nt = b1 - e4;
        for (int64_t t = lane; t < nh + nt; t += G) {
            const int64_t j = t < nh ? b0 + t : e4 + (t - nh);
            acc_add(out + (ld_stream(indices + j) - col0), event_value<Acc>(load_weight<WK>(data, j, w_homo)));
        }
    }
    const int64_t c1 = e4 >> 2;
    int64_t cb = (a4 >> 2) + lane;
    int4 c[4];
    float4 w[4];
    auto load = [&]() {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t cc = cb + u * G;
            if (cc < c1) {
                c[u] = ld_stream4(indices + 4 * cc);
                w[u] = load_weight4<WK>(data, 4 * cc, w_homo);
            } else {
                c[u] = make_int4(-1, -1, -1, -1);
                w[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    load();
    while (true) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u].x < 0) continue;
            acc_add(out + (c[u].x - col0), event_value<Acc>(w[u].x));
            acc_add(out + (c[u].y - col0), event_value<Acc>(w[u].y));
            acc_add(out + (c[u].z - col0), event_value<Acc>(w[u].z));
            acc_add(out + (c[u].w - col0), event_value<Acc>(w[u].w));
        }
        cb += 4 * G;
        if (cb >= c1) break;
        load();
    }
}

// Weight of synapses 4 blk + m (m = 0..3) of a JIT row.
template <int WK>
__device__ __forceinline__ void jit_weights(const JitArgs& d, uint32_t blk, uint32_t row, float w[4]) {
    if constexpr (WK == BP_JIT_UNIFORM) {
        const uint4 x = Philox::block(make_uint4(blk, row, 1u, 0u), static_cast<uint32_t>(d.seed),
                                      static_cast<uint32_t>(d.seed >> 32));
        const float span = d.w1 - d.w0;
        const float s24 = 1.0f / 16777216.0f;
        w[0] = d.w0 + span * (static_cast<float>(x.x >> 8) * s24);
        w[1] = d.w0 + span * (static_cast<float>(x.y >> 8) * s24);
        w[2] = d.w0 + span * (static_cast<float>(x.z >> 8) * s24);
        w[3] = d.w0 + span * (static_cast<float>(x.w >> 8) * s24);
    } else if constexpr (WK == BP_JIT_NORMAL) {
        const float s24 = 1.0f / 16777216.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 x = Philox::block(make_uint4(2u * blk + h, row, 2u, 0u), static_cast<uint32_t>(d.seed),
                                          static_cast<uint32_t>(d.seed >> 32));
            const float u1a = static_cast<float>((x.x >> 8) + 1u) * s24;
            const float u2a = static_cast<float>(x.y >> 8) * s24;
            const float u1b = static_cast<float>((x.z >> 8) + 1u) * s24;
            const float u2b = static_cast<float>(x.w >> 8) * s24;
            w[2 * h] = d.w0 + d.w1 * (sqrtf(-2.0f * logf(u1a)) * cospif(2.0f * u2a));
            w[2 * h + 1] = d.w0 + d.w1 * (sqrtf(-2.0f * logf(u1b)) * cospif(2.0f * u2b));
        }
    } else {
        w[0] = w[1] = w[2] = w[3] = d.w0;
    }
}

// Walks JIT row `row` with a group of G lanes (G = 32: the calling full warp;
// G = 16: the calling half warp, the other half walking another row) in
// chunks of 4 G gaps: lane l draws the Philox block (c + l, row, 0, 0), maps
// its four words to U[1, K] with a multiply-high, and a group inclusive scan
// of the lanes' sums gives the positions q_0 = U_0 - 1,
// q_{k+1} = q_k + U_{k+1}.  The blocks are drawn in the same order whatever G,
// so the targets do not depend on it.  f(q, k, w) runs for every target
// q < n_post (k = synapse index).  Every lane of the group must call it with
// the same row.  Returns this lane's count.
template <int WK, int G, typename F>
__device__ __forceinline__ int64_t jit_walk_g(const JitArgs& d, uint32_t row, int64_t n_post, F&& f) {
    static_assert(G == 16 || G == 32, "JIT rows are walked by 16 or 32 lanes");
    const uint32_t lane = threadIdx.x & (G - 1u);
    const unsigned mask = G == 32 ? FULL_MASK : (0xFFFFu << (threadIdx.x & 16u));
    const uint32_t k0 = static_cast<uint32_t>(d.seed), k1 = static_cast<uint32_t>(d.seed >> 32);
    int64_t carry = -1;
    int64_t count = 0;
    for (uint32_t c = 0;; c += G) {
        const uint32_t blk = c + lane;
        const uint4 x = Philox::block(make_uint4(blk, row, 0u, 0u), k0, k1);
        const uint32_t g0 = 1u + __umulhi(x.x, d.K);
        const uint32_t g1 = 1u + __umulhi(x.y, d.K);
        const uint32_t g2 = 1u + __umulhi(x.z, d.K);
        const uint32_t g3 = 1u + __umulhi(x.w, d.K);
        const uint64_t s4 = static_cast<uint64_t>(g0) + g1 + g2 + g3;
        uint64_t incl = s4;
#pragma unroll
        for (int dd = 1; dd < G; dd <<= 1) {
            const uint64_t o = __shfl_up_sync(mask, incl, dd, G);
            if (lane >= static_cast<uint32_t>(dd)) incl += o;
        }
        const int64_t q0 = carry + static_cast<int64_t>(incl - s4) + g0;
        const int64_t q1 = q0 + g1, q2 = q1 + g2, q3 = q2 + g3;
        if (q0 < n_post) {
            float w[4];
            jit_weights<WK>(d, blk, row, w);
            const uint64_t kb = 4ull * blk;
            f(q0, kb, w[0]);
            ++count;
            if (q1 < n_post) { f(q1, kb + 1, w[1]); ++count; }
            if (q2 < n_post) { f(q2, kb + 2, w[2]); ++count; }
            if (q3 < n_post) { f(q3, kb + 3, w[3]); ++count; }
        }
        carry += static_cast<int64_t>(__shfl_sync(mask, incl, G - 1, G));
        if (carry >= n_post - 1) break;
    }
    return count;
}

// The full-warp walk (G = 32).
template <int WK, typename F>
__device__ __forceinline__ int64_t jit_walk(const JitArgs& d, uint32_t row, int64_t n_post, F&& f) {
    return jit_walk_g<WK, 32>(d, row, n_post, static_cast<F&&>(f));
}

// Adds v (one value per thread) into *dst with one atomic per CTA.  Every
// thread of the CTA must call it.
__device__ __forceinline__ void block_add_i64(int64_t v, int64_t* dst) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    v = group_reduce_sum(v, 32);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_sum, static_cast<unsigned long long>(v));
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(reinterpret_cast<unsigned long long*>(dst), s_sum);
}

}  // namespace bp
