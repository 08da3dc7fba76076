// jitconn.cu -- just-in-time connectivity (a6, Section 4.2, Appendix C).
//
// A warp regenerates one presynaptic row in chunks of 128 gaps: lane l draws
// the Philox block with counter (c + l, row, 0, 0), i.e. gaps 4(c+l) ..
// 4(c+l)+3, maps each 32-bit word to U[1, K] with a multiply-high, and a warp
// inclusive scan of the lanes' 4-gap sums turns gaps into target positions
// (q_0 = U_0 - 1, q_{k+1} = q_k + U_{k+1}).  The chunk's last position is
// carried to the next chunk; the walk stops once it reaches n_post - 1.
// Weights come from their own counter streams (1: uniform, 2: normal) at the
// same synapse index, so any synapse can be regenerated independently.
// Accumulation: the whole postsynaptic vector in shared memory when it fits
// (flushed once per CTA, skipping zeros), otherwise atomics into L2.  Calls
// with few, long rows walk each row with a whole CTA (jit_walk_cta).
#include "bp_common.cuh"
#include "bp_internal.h"
#include "bp_rows.cuh"

namespace bp {
namespace {

constexpr int kJitThreads = 512;
constexpr int kJitWarps = kJitThreads / 32;

// The whole CTA walks row `row` together (for calls with few, long rows):
// per round, warp w draws the 32 Philox blocks c + 32 w + lane (128 gaps), a
// warp scan orders them within the warp, and a prefix over the warps' totals
// (shared memory) gives each warp its offset, so the positions are exactly
// those of jit_walk's chunk-by-chunk walk; rounds continue from the last
// position until it reaches n_post - 1.  Every thread of the CTA must call
// it with the same row.  Returns this lane's count.
template <int WK, typename F>
__device__ __forceinline__ int64_t jit_walk_cta(const JitArgs& d, uint32_t row, int64_t n_post, F&& f) {
    __shared__ uint64_t s_tot[kJitWarps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t k0 = static_cast<uint32_t>(d.seed), k1 = static_cast<uint32_t>(d.seed >> 32);
    int64_t carry = -1;
    int64_t count = 0;
    for (uint32_t c = 0;; c += 32u * kJitWarps) {
        const uint32_t blk = c + 32u * warp + lane;
        const uint4 x = Philox::block(make_uint4(blk, row, 0u, 0u), k0, k1);
        const uint32_t g0 = 1u + __umulhi(x.x, d.K);
        const uint32_t g1 = 1u + __umulhi(x.y, d.K);
        const uint32_t g2 = 1u + __umulhi(x.z, d.K);
        const uint32_t g3 = 1u + __umulhi(x.w, d.K);
        const uint64_t s4 = static_cast<uint64_t>(g0) + g1 + g2 + g3;
        const uint64_t incl = warp_inclusive_scan(s4);
        if (lane == 31u) s_tot[warp] = incl;
        __syncthreads();
        uint64_t off = 0, tot = 0;
#pragma unroll
        for (int v = 0; v < kJitWarps; ++v) {
            const uint64_t t = s_tot[v];
            off += v < static_cast<int>(warp) ? t : 0;
            tot += t;
        }
        const int64_t q0 = carry + static_cast<int64_t>(off + incl - s4) + g0;
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
        carry += static_cast<int64_t>(tot);
        __syncthreads();  // s_tot is rewritten next round
        if (carry >= n_post - 1) break;
    }
    return count;
}

// Event scatter of JIT rows.  SMEM: the CTA accumulates all n_post columns
// in shared memory of `wpad` entries.  With few rows compared with the warps
// and long rows (expected length 2 n_post / (K + 1) of 512 or more) each row
// is walked by a whole CTA (jit_walk_cta) instead of one warp.
template <typename Acc, int WK, bool SMEM>
__global__ void __launch_bounds__(kJitThreads) k_jit_scatter(JitArgs d, int64_t n_post,
                                                             const int32_t* __restrict__ spike_list,
                                                             const int32_t* __restrict__ n_spikes, int64_t max_spikes,
                                                             Acc* __restrict__ y, int32_t wpad,
                                                             int64_t* __restrict__ events_total) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* acc = reinterpret_cast<Acc*>(smem_raw);
    if constexpr (SMEM) {
        for (int t = threadIdx.x; t < wpad; t += blockDim.x) acc[t] = Acc(0);
        __syncthreads();
    }
    Acc* out = SMEM ? acc : y;
    int64_t ns = *n_spikes;
    ns = ns < max_spikes ? ns : max_spikes;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kJitWarps;
    int64_t ev = 0;
    const int64_t est_len = 2 * n_post / (static_cast<int64_t>(d.K) + 1);
    if (ns * 4 <= nwarps && est_len >= 512) {
        for (int64_t u = blockIdx.x; u < ns; u += gridDim.x) {
            const int32_t i = spike_list[u];
            if (i < 0) continue;
            ev += jit_walk_cta<WK>(d, static_cast<uint32_t>(i), n_post,
                                   [&](int64_t q, uint64_t, float w) { acc_add(out + q, event_value<Acc>(w)); });
        }
    } else {
        for (int64_t u = static_cast<int64_t>(blockIdx.x) * kJitWarps + (threadIdx.x >> 5); u < ns; u += nwarps) {
            const int32_t i = spike_list[u];
            if (i < 0) continue;
            ev += jit_walk<WK>(d, static_cast<uint32_t>(i), n_post,
                               [&](int64_t q, uint64_t, float w) { acc_add(out + q, event_value<Acc>(w)); });
        }
    }
    if constexpr (SMEM) {
        __syncthreads();
        for (int t = threadIdx.x; t < n_post; t += blockDim.x) {
            const Acc v = acc[t];
            if (v != Acc(0)) acc_add(y + t, v);
        }
    }
    if (events_total) block_add_i64(ev, events_total);
}

// Gather over all rows: y_pre[i] += sum over targets q of w x[q].
template <int WK>
__global__ void __launch_bounds__(kJitThreads) k_jit_gather(JitArgs d, int64_t n_pre, int64_t n_post,
                                                            const float* __restrict__ x, float* __restrict__ y_pre) {
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kJitWarps;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kJitWarps + (threadIdx.x >> 5); i < n_pre; i += nwarps) {
        float sum = 0.f;
        jit_walk<WK>(d, static_cast<uint32_t>(i), n_post, [&](int64_t q, uint64_t, float w) { sum += w * __ldg(x + q); });
        sum = group_reduce_sum(sum, 32);
        if ((threadIdx.x & 31) == 0) y_pre[i] += sum;
    }
}

// Dense-vector product: y[q] += w x[i] over all rows i.
template <int WK, bool SMEM>
__global__ void __launch_bounds__(kJitThreads) k_jit_mv(JitArgs d, int64_t n_pre, int64_t n_post,
                                                        const float* __restrict__ x, float* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* acc = reinterpret_cast<float*>(smem_raw);
    if constexpr (SMEM) {
        for (int t = threadIdx.x; t < n_post; t += blockDim.x) acc[t] = 0.f;
        __syncthreads();
    }
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kJitWarps;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kJitWarps + (threadIdx.x >> 5); i < n_pre; i += nwarps) {
        const float xi = __ldg(x + i);
        float* out = SMEM ? acc : y;
        jit_walk<WK>(d, static_cast<uint32_t>(i), n_post, [&](int64_t q, uint64_t, float w) { atomicAdd(out + q, w * xi); });
    }
    if constexpr (SMEM) {
        __syncthreads();
        for (int t = threadIdx.x; t < n_post; t += blockDim.x) {
            const float v = acc[t];
            if (v != 0.f) atomicAdd(y + t, v);
        }
    }
}

// Row lengths into indptr[i + 1]; indptr[0] = 0.
__global__ void __launch_bounds__(kJitThreads) k_jit_rowlen(JitArgs d, int64_t n_pre, int64_t n_post,
                                                            int64_t* __restrict__ indptr) {
    if (blockIdx.x == 0 && threadIdx.x == 0) indptr[0] = 0;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kJitWarps;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kJitWarps + (threadIdx.x >> 5); i < n_pre; i += nwarps) {
        int64_t c = jit_walk<BP_JIT_HOMO>(d, static_cast<uint32_t>(i), n_post, [](int64_t, uint64_t, float) {});
        c = group_reduce_sum(c, 32);
        if ((threadIdx.x & 31) == 0) indptr[i + 1] = c;
    }
}

// In-place inclusive prefix sum of v[0 .. n) by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_inplace(int64_t* __restrict__ v, int64_t n) {
    constexpr int kItems = 8;
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < n; base += 1024 * kItems) {
        int64_t x[kItems];
        const int64_t off = base + static_cast<int64_t>(threadIdx.x) * kItems;
        int64_t run = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            x[k] = (off + k < n) ? v[off + k] : 0;
            run += x[k];
            x[k] = run;
        }
        const uint64_t incl = warp_inclusive_scan(static_cast<uint64_t>(run));
        if (lane == 31) warp_tot[warp] = static_cast<int64_t>(incl);
        __syncthreads();
        if (warp == 0) {
            const uint64_t t = warp_inclusive_scan(static_cast<uint64_t>(warp_tot[lane]));
            warp_tot[lane] = static_cast<int64_t>(t);
        }
        __syncthreads();
        const int64_t prefix = s_carry + (warp > 0 ? warp_tot[warp - 1] : 0) + static_cast<int64_t>(incl) - run;
#pragma unroll
        for (int k = 0; k < kItems; ++k)
            if (off + k < n) v[off + k] = x[k] + prefix;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += warp_tot[31];
        __syncthreads();
    }
}

// Writes row i's targets (and weights) at indptr[i] + k.
template <int WK, int DK>
__global__ void __launch_bounds__(kJitThreads) k_jit_fill(JitArgs d, int64_t n_pre, int64_t n_post,
                                                          const int64_t* __restrict__ indptr,
                                                          int32_t* __restrict__ indices, void* __restrict__ data) {
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kJitWarps;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kJitWarps + (threadIdx.x >> 5); i < n_pre; i += nwarps) {
        const int64_t rs = indptr[i];
        jit_walk<WK>(d, static_cast<uint32_t>(i), n_post, [&](int64_t q, uint64_t k, float w) {
            indices[rs + static_cast<int64_t>(k)] = static_cast<int32_t>(q);
            if constexpr (DK == BP_W_F32) static_cast<float*>(data)[rs + k] = w;
            if constexpr (DK == BP_W_BF16) static_cast<__nv_bfloat16*>(data)[rs + k] = __float2bfloat16_rn(w);
        });
    }
}

int jit_grid(int64_t rows) {
    const int64_t need = (rows + kJitWarps - 1) / kJitWarps;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 4;
    const int64_t g = need < cap ? need : cap;
    return static_cast<int>(g > 0 ? g : 1);
}

template <typename Acc, int WK>
bp_status launch_jit_scatter_t(const JitArgs& d, int64_t n_post, const int32_t* sl, const int32_t* ns, int64_t mx,
                               void* y, int64_t* ev, int mode, cudaStream_t s) {
    const int32_t cap = kTileCols;
    const bool fits = n_post <= cap;
    const int grid_direct = sm_count() * 4;
    if (fits && mode != 1) {
        const int32_t wpad = static_cast<int32_t>((n_post + 31) & ~int64_t(31));
        const size_t smem = static_cast<size_t>(wpad) * sizeof(Acc);
        BP_TRY(ensure_smem_attr(reinterpret_cast<const void*>(k_jit_scatter<Acc, WK, true>),
                                static_cast<int>(cap * sizeof(Acc))));
        // one shared copy of y per CTA: use one CTA per SM
        k_jit_scatter<Acc, WK, true><<<sm_count(), kJitThreads, smem, s>>>(d, n_post, sl, ns, mx,
                                                                           static_cast<Acc*>(y), wpad, ev);
    } else {
        k_jit_scatter<Acc, WK, false><<<grid_direct, kJitThreads, 0, s>>>(d, n_post, sl, ns, mx,
                                                                          static_cast<Acc*>(y), 0, ev);
    }
    BP_LAUNCHED();
    return BP_OK;
}

template <typename Acc>
bp_status launch_jit_scatter_wk(const JitArgs& d, int64_t n_post, const int32_t* sl, const int32_t* ns, int64_t mx,
                                void* y, int64_t* ev, int mode, cudaStream_t s) {
    switch (d.wkind) {
        case BP_JIT_UNIFORM: return launch_jit_scatter_t<Acc, BP_JIT_UNIFORM>(d, n_post, sl, ns, mx, y, ev, mode, s);
        case BP_JIT_NORMAL: return launch_jit_scatter_t<Acc, BP_JIT_NORMAL>(d, n_post, sl, ns, mx, y, ev, mode, s);
        default: return launch_jit_scatter_t<Acc, BP_JIT_HOMO>(d, n_post, sl, ns, mx, y, ev, mode, s);
    }
}

JitArgs to_args(const bp_jit_desc& d) {
    JitArgs a;
    a.seed = d.seed;
    a.K = static_cast<uint32_t>(d.K);
    a.wkind = d.wkind;
    a.w0 = d.w0;
    a.w1 = d.w1;
    return a;
}

bp_status check_desc(const bp_jit_desc* d, int64_t n_pre, int64_t n_post) {
    BP_REQUIRE(d != nullptr, "descriptor is NULL");
    BP_REQUIRE(d->K >= 1 && d->K < (int64_t(1) << 32), "descriptor K = %lld invalid (call bp_jit_desc_init)",
               (long long)d->K);
    BP_REQUIRE(d->wkind >= BP_JIT_HOMO && d->wkind <= BP_JIT_NORMAL, "unknown weight kind %d", d->wkind);
    BP_REQUIRE(n_pre >= 0 && n_post >= 0 && n_pre <= INT32_MAX && n_post <= INT32_MAX, "bad sizes");
    return BP_OK;
}

}  // namespace

bp_status launch_jit_event_mv(const JitArgs& d, int64_t n_post, const int32_t* spike_list, const int32_t* n_spikes,
                              int64_t max_spikes, void* y, bool counts, int64_t* events_total, int mode,
                              cudaStream_t s) {
    if (max_spikes <= 0 || n_post == 0) return BP_OK;
    if (counts)
        return launch_jit_scatter_wk<int32_t>(d, n_post, spike_list, n_spikes, max_spikes, y, events_total, mode, s);
    return launch_jit_scatter_wk<float>(d, n_post, spike_list, n_spikes, max_spikes, y, events_total, mode, s);
}

}  // namespace bp

extern "C" {

bp_status bp_jitconn_event_mv(const bp_jit_desc* d, int64_t n_pre, int64_t n_post, const int32_t* spike_list,
                              const int32_t* n_spikes, int64_t max_spikes, void* y, int32_t y_is_count, uint32_t flags,
                              bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_jitconn_event_mv");
    BP_TRY(bp::check_desc(d, n_pre, n_post));
    BP_REQUIRE(!y_is_count || d->wkind == BP_JIT_HOMO, "integer counts need homogeneous weights");
    BP_REQUIRE(max_spikes >= 0 && max_spikes <= n_pre, "max_spikes out of range");
    BP_REQUIRE(n_post == 0 || y != nullptr, "y is NULL");
    BP_REQUIRE(max_spikes == 0 || (spike_list && n_spikes), "spike list or count is NULL");
    if (flags & BP_OVERWRITE) BP_CUDA(cudaMemsetAsync(y, 0, static_cast<size_t>(n_post) * 4, stream));
    const bp::JitArgs a = bp::to_args(*d);
    const int mode = (flags & BP_ACC_GLOBAL) ? 1 : ((flags & BP_ACC_SHARED) ? 2 : 0);
    return bp::launch_jit_event_mv(a, n_post, spike_list, n_spikes, max_spikes, y, y_is_count != 0, nullptr, mode,
                                   stream);
}

bp_status bp_jitconn_event_mv_bwd(const bp_jit_desc* d, int64_t n_pre, int64_t n_post, const float* dy, float* dx_pre,
                                  bp_stream_t stream) {
    bp::clear_error();
    BP_TRY(bp::check_desc(d, n_pre, n_post));
    BP_REQUIRE(n_pre == 0 || (dy && dx_pre), "dy or dx_pre is NULL");
    if (n_pre == 0 || n_post == 0) return BP_OK;
    const bp::JitArgs a = bp::to_args(*d);
    const int grid = bp::jit_grid(n_pre);
    switch (a.wkind) {
        case BP_JIT_UNIFORM: bp::k_jit_gather<BP_JIT_UNIFORM><<<grid, bp::kJitThreads, 0, stream>>>(a, n_pre, n_post, dy, dx_pre); break;
        case BP_JIT_NORMAL: bp::k_jit_gather<BP_JIT_NORMAL><<<grid, bp::kJitThreads, 0, stream>>>(a, n_pre, n_post, dy, dx_pre); break;
        default: bp::k_jit_gather<BP_JIT_HOMO><<<grid, bp::kJitThreads, 0, stream>>>(a, n_pre, n_post, dy, dx_pre); break;
    }
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_jitconn_mv(const bp_jit_desc* d, int64_t n_pre, int64_t n_post, const float* x_pre, float* y_post,
                        uint32_t flags, bp_stream_t stream) {
    bp::clear_error();
    BP_TRY(bp::check_desc(d, n_pre, n_post));
    BP_REQUIRE(n_post == 0 || y_post != nullptr, "y_post is NULL");
    BP_REQUIRE(n_pre == 0 || x_pre != nullptr, "x_pre is NULL");
    if (flags & BP_OVERWRITE) BP_CUDA(cudaMemsetAsync(y_post, 0, static_cast<size_t>(n_post) * 4, stream));
    if (n_pre == 0 || n_post == 0) return BP_OK;
    const bp::JitArgs a = bp::to_args(*d);
    const bool smem = n_post <= bp::kTileCols && !(flags & BP_ACC_GLOBAL);
    const int grid = smem ? bp::sm_count() : bp::jit_grid(n_pre);
    const size_t bytes = smem ? static_cast<size_t>((n_post + 31) & ~int64_t(31)) * 4 : 0;
#define BP_JIT_MV_LAUNCH(WKV)                                                                                     \
    do {                                                                                                        \
        if (smem) {                                                                                             \
            BP_TRY(bp::ensure_smem_attr(reinterpret_cast<const void*>(bp::k_jit_mv<WKV, true>), bp::kTileCols * 4)); \
            bp::k_jit_mv<WKV, true><<<grid, bp::kJitThreads, bytes, stream>>>(a, n_pre, n_post, x_pre, y_post);  \
        } else {                                                                                                \
            bp::k_jit_mv<WKV, false><<<grid, bp::kJitThreads, 0, stream>>>(a, n_pre, n_post, x_pre, y_post);    \
        }                                                                                                       \
    } while (0)
    switch (a.wkind) {
        case BP_JIT_UNIFORM: BP_JIT_MV_LAUNCH(BP_JIT_UNIFORM); break;
        case BP_JIT_NORMAL: BP_JIT_MV_LAUNCH(BP_JIT_NORMAL); break;
        default: BP_JIT_MV_LAUNCH(BP_JIT_HOMO); break;
    }
#undef BP_JIT_MV_LAUNCH
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_jit_materialize_csr(const bp_jit_desc* d, int64_t n_pre, int64_t n_post, int64_t* indptr,
                                 int32_t* indices, void* data, int32_t data_kind, bp_stream_t stream) {
    bp::clear_error();
    BP_TRY(bp::check_desc(d, n_pre, n_post));
    BP_REQUIRE(indptr != nullptr, "indptr is NULL");
    BP_REQUIRE(data_kind >= BP_W_HOMO && data_kind <= BP_W_BF16, "unknown data kind %d", data_kind);
    const bp::JitArgs a = bp::to_args(*d);
    const int grid = bp::jit_grid(n_pre);
    if (indices == nullptr) {
        if (n_pre == 0) {
            BP_CUDA(cudaMemsetAsync(indptr, 0, sizeof(int64_t), stream));
            return BP_OK;
        }
        bp::k_jit_rowlen<<<grid, bp::kJitThreads, 0, stream>>>(a, n_pre, n_post, indptr);
        BP_LAUNCHED();
        bp::k_scan_inplace<<<1, 1024, 0, stream>>>(indptr + 1, n_pre);
        BP_LAUNCHED();
        return BP_OK;
    }
    BP_REQUIRE(data_kind == BP_W_HOMO || data != nullptr, "data is NULL for a stored weight kind");
    if (n_pre == 0 || n_post == 0) return BP_OK;
#define BP_FILL(WKV, DKV) bp::k_jit_fill<WKV, DKV><<<grid, bp::kJitThreads, 0, stream>>>(a, n_pre, n_post, indptr, indices, data)
#define BP_FILL_DK(WKV)                                   \
    do {                                                  \
        if (data_kind == BP_W_F32) BP_FILL(WKV, BP_W_F32);  \
        else if (data_kind == BP_W_BF16) BP_FILL(WKV, BP_W_BF16); \
        else BP_FILL(WKV, BP_W_HOMO);                       \
    } while (0)
    switch (a.wkind) {
        case BP_JIT_UNIFORM: BP_FILL_DK(BP_JIT_UNIFORM); break;
        case BP_JIT_NORMAL: BP_FILL_DK(BP_JIT_NORMAL); break;
        default: BP_FILL_DK(BP_JIT_HOMO); break;
    }
#undef BP_FILL_DK
#undef BP_FILL
    BP_LAUNCHED();
    return BP_OK;
}

}  // extern "C"
