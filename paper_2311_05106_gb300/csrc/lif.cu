// lif.cu -- the fused neuron step (a1-a4) and, for the network, the delivery
// of the step's spikes in the same kernel (a5/a6).
//
// Neuron pass.  Structure-of-arrays FP32 state and one-byte refractory
// counters; each thread updates VEC = 4 consecutive neurons per grid-stride
// iteration with 16-byte loads and stores (one 4-byte word for the four
// counters): decay and event add of both conductances (Appendix E), COBA
// current with the pre-update potential (Appendix F), exponential-Euler
// membrane update with refractory clamp, threshold and reset.  Spike flags
// stay in a 32-bit register mask (bit = iteration * VEC + element), so the
// loop has no barrier; the grid is sized so that no thread runs more than
// 32 / VEC iterations.  One block-wide prefix over the masks then compacts
// the CTA's spikes into shared memory.
//
// Delivery.  In the network step each CTA then delivers its own spikes:
// groups of lanes walk the stored CSR rows, or whole warps regenerate the
// JIT rows, with atomics into the OTHER half of the double-buffered event
// accumulators (the half this step did not read), which the next step reads
// (zero delay).  The spike list and the per-step record are optional outputs.
#include <mutex>
#include <unordered_map>

#include "bp_common.cuh"
#include "bp_internal.h"
#include "bp_neuron.cuh"
#include "bp_rows.cuh"

namespace bp {
namespace {

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;
constexpr int kMaskBits = 32;

// CONN_PRE: the neuron pass of the AlignPre form (the conductances are
// recomputed each step, so they are not loaded; no delivery)
enum { CONN_NONE = 0, CONN_CSR = 1, CONN_JIT = 2, CONN_PRE = 3 };

struct StepArgs {
    LifConst c;
    int64_t n, n_e;
    float* V;
    float* ge;
    float* gi;
    uint8_t* ref;  // refractory steps left, one byte per neuron
    void* ye_in;   // read and zeroed this step
    void* yi_in;
    void* ye_out;  // receive this step's deliveries
    void* yi_out;
    const float* I_vec;
    uint8_t* spk;
    int32_t* spike_list;
    int32_t* n_spikes;
    int32_t* clear_counter;
    int64_t* totals;  // [0] E spikes, [1] I spikes, [2] events (nullable)
    const NetCtrl* ctrl;
    int32_t t_local;
    CsrArgs csr;
    int32_t group;  // lanes per CSR row in the delivery
    JitArgs je, ji;
    // delay ring: ring_slots counts, then ring_slots lists of n spike ids
    int32_t* ring;
    int32_t ring_slots, delay_e, delay_i;
    // the step counter advance done by the launch's last CTA (0: none)
    NetCtrl* adv_ctrl;
    int32_t advance;
};

struct StepSmem {
    int32_t ids[kStepThreads * kMaskBits];
    int32_t warp_sum[kStepWarps];
    int32_t total;
    int32_t base;
    int32_t ring_base;
    long long red[3][kStepWarps];
};

// The last CTA of the launch to finish advances the device step counter by
// a.advance (and the step total): every CTA has finished reading the counter
// when it counts itself done, so no CTA of this launch sees the new value.
__device__ __forceinline__ void advance_step_counter(const StepArgs& a) {
    if (a.advance == 0 || a.adv_ctrl == nullptr) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.adv_ctrl->done_ctas, 1u);
        if (prev == gridDim.x - 1) {
            a.adv_ctrl->done_ctas = 0;
            a.adv_ctrl->step += a.advance;
            if (a.totals) a.totals[3] += a.advance;
            __threadfence();
        }
    }
}

template <bool COUNTS, int VEC, int CONN, int WK, bool RING = false>
__global__ void __launch_bounds__(kStepThreads, 4) k_step(StepArgs a) {
    __shared__ StepSmem sm;
    using Y = typename std::conditional<COUNTS, int32_t, float>::type;
    using Y4 = typename std::conditional<COUNTS, int4, float4>::type;
    const LifConst& c = a.c;
    Y* __restrict__ ye = static_cast<Y*>(a.ye_in);
    Y* __restrict__ yi = static_cast<Y*>(a.yi_in);
    Y* out_e = static_cast<Y*>(a.ye_out);
    Y* out_i = static_cast<Y*>(a.yi_out);
    // programmatic dependent launch (network steps on a partial wave): wait
    // for the previous step's grid and its memory, then let the next step's
    // grid be scheduled; both return at once for an ordinary launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (a.clear_counter && blockIdx.x == 0 && threadIdx.x == 0) *a.clear_counter = 0;
    // RING (a delayed projection): step t appends its spikes to list
    // t mod S and delivers the lists of steps t - d; the count of list
    // (t + 1) mod S, which no one reads or writes in this step, is cleared
    // for the next step (S = max delay + 2).
    int64_t tt = 0;
    if constexpr (RING) {
        tt = a.ctrl->step + a.t_local;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ring[(tt + 1) % a.ring_slots] = 0;
    }

    uint32_t mask = 0;
    int cnt_e = 0, cnt_i = 0;
    const uint64_t keep = l2_keep_policy();
    const int64_t nq = (a.n + VEC - 1) / VEC;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kStepThreads;
    const int64_t q0 = static_cast<int64_t>(blockIdx.x) * kStepThreads + threadIdx.x;
    int it = 0;
    for (int64_t q = q0; q < nq; q += stride, ++it) {
        const int64_t i0 = q * VEC;
        uint32_t bits = 0;
        if (VEC == 4 && i0 + 4 <= a.n) {
            // the state streams through L2 (evict-first); the accumulators
            // are read with the keep policy since the next delivery targets them
            float4 v = __ldcs(reinterpret_cast<const float4*>(a.V + i0));
            float4 g_e = make_float4(0.f, 0.f, 0.f, 0.f), g_i = g_e;
            if constexpr (CONN != CONN_PRE) {
                g_e = __ldcs(reinterpret_cast<const float4*>(a.ge + i0));
                g_i = __ldcs(reinterpret_cast<const float4*>(a.gi + i0));
            }
            const uchar4 r8 = __ldcs(reinterpret_cast<const uchar4*>(a.ref + i0));
            int4 r = make_int4(r8.x, r8.y, r8.z, r8.w);
            const Y4 ce = ld_keep(reinterpret_cast<const Y4*>(ye + i0), keep);
            const Y4 ci = ld_keep(reinterpret_cast<const Y4*>(yi + i0), keep);
            float4 Iv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.I_vec) Iv = __ldcs(reinterpret_cast<const float4*>(a.I_vec + i0));
            const int4 r_old = r;
            bits |= neuron_update(c, v.x, g_e.x, g_i.x, r.x, event_add<COUNTS>(ce.x, c.w_e), event_add<COUNTS>(ci.x, c.w_i), Iv.x) ? 1u : 0u;
            bits |= neuron_update(c, v.y, g_e.y, g_i.y, r.y, event_add<COUNTS>(ce.y, c.w_e), event_add<COUNTS>(ci.y, c.w_i), Iv.y) ? 2u : 0u;
            bits |= neuron_update(c, v.z, g_e.z, g_i.z, r.z, event_add<COUNTS>(ce.z, c.w_e), event_add<COUNTS>(ci.z, c.w_i), Iv.z) ? 4u : 0u;
            bits |= neuron_update(c, v.w, g_e.w, g_i.w, r.w, event_add<COUNTS>(ce.w, c.w_e), event_add<COUNTS>(ci.w, c.w_i), Iv.w) ? 8u : 0u;
            __stcs(reinterpret_cast<float4*>(a.V + i0), v);
            __stcs(reinterpret_cast<float4*>(a.ge + i0), g_e);
            __stcs(reinterpret_cast<float4*>(a.gi + i0), g_i);
            if (r.x != r_old.x || r.y != r_old.y || r.z != r_old.z || r.w != r_old.w)
                __stcs(reinterpret_cast<uchar4*>(a.ref + i0),
                       make_uchar4(static_cast<unsigned char>(r.x), static_cast<unsigned char>(r.y),
                                   static_cast<unsigned char>(r.z), static_cast<unsigned char>(r.w)));
            if (ce.x != Y(0) || ce.y != Y(0) || ce.z != Y(0) || ce.w != Y(0))
                st_keep(reinterpret_cast<Y4*>(ye + i0), Y4{}, keep);
            if (ci.x != Y(0) || ci.y != Y(0) || ci.z != Y(0) || ci.w != Y(0))
                st_keep(reinterpret_cast<Y4*>(yi + i0), Y4{}, keep);
            if (a.spk) {
                const uint32_t packed = (bits & 1u) | ((bits & 2u) << 7) | ((bits & 4u) << 14) | ((bits & 8u) << 21);
                *reinterpret_cast<uint32_t*>(a.spk + i0) = packed;
            }
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                const int64_t i = i0 + k;
                if (i >= a.n) break;
                float v = a.V[i];
                float g_e = CONN == CONN_PRE ? 0.f : a.ge[i];
                float g_i = CONN == CONN_PRE ? 0.f : a.gi[i];
                int32_t r = a.ref[i];
                const int32_t r_old = r;
                const Y ce = ye[i], ci = yi[i];
                const float Iv = a.I_vec ? a.I_vec[i] : 0.f;
                const bool s = neuron_update(c, v, g_e, g_i, r, event_add<COUNTS>(ce, c.w_e),
                                             event_add<COUNTS>(ci, c.w_i), Iv);
                a.V[i] = v;
                a.ge[i] = g_e;
                a.gi[i] = g_i;
                if (r != r_old) a.ref[i] = static_cast<uint8_t>(r);
                if (ce != Y(0)) ye[i] = Y(0);
                if (ci != Y(0)) yi[i] = Y(0);
                if (a.spk) a.spk[i] = s ? 1 : 0;
                bits |= s ? (1u << k) : 0u;
            }
        }
        if (bits) {
            mask |= bits << (it * VEC);
#pragma unroll
            for (int k = 0; k < VEC; ++k)
                if (bits & (1u << k)) {
                    if (i0 + k < a.n_e) ++cnt_e; else ++cnt_i;
                    // the delivery below reads this row's extent: start the fetch now
                    if constexpr (CONN == CONN_CSR)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.csr.indptr + i0 + k));
                }
        }
    }

    // ---- start fetching the rows this CTA delivers right after the barrier
    // below: each spiking neuron's row extent was prefetched at detection, so
    // its index (and weight) lines can be requested into L2 now, while other
    // warps still stream (measured 24.7 -> 24.2 us per step at N = 4e6)
    if constexpr (CONN == CONN_CSR && !RING) {
        for (uint32_t m = mask; m; m &= m - 1) {
            const int b = __ffs(m) - 1;
            const int64_t i = (q0 + static_cast<int64_t>(b / VEC) * stride) * VEC + (b % VEC);
            const int64_t b0 = a.csr.indptr[i], b1 = a.csr.indptr[i + 1];
            for (int64_t j = b0 & ~int64_t(31); j < b1; j += 32) {  // 128-byte lines of 4-byte entries
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.csr.indices + j));
                if constexpr (WK == WK_F32)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const float*>(a.csr.data) + j));
                // BF16 weights: a 128-byte line holds 64 entries
                if constexpr (WK == WK_BF16)
                    if ((j & 63) == 0 || j == (b0 & ~int64_t(31)))
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const __nv_bfloat16*>(a.csr.data) + j));
            }
        }
    }

    // ---- compaction of the CTA's spikes into shared memory
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mine = __popc(mask);
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) sm.warp_sum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kStepWarps; ++w) {
            const int v = sm.warp_sum[w];
            sm.warp_sum[w] = run;
            run += v;
        }
        sm.total = run;
    }
    __syncthreads();
    int off = sm.warp_sum[warp] + incl - mine;
    for (uint32_t m = mask; m; m &= m - 1) {
        const int b = __ffs(m) - 1;
        const int64_t i = (q0 + static_cast<int64_t>(b / VEC) * stride) * VEC + (b % VEC);
        sm.ids[off++] = static_cast<int32_t>(i);
    }
    __syncthreads();
    const int total = sm.total;

    // ---- optional global spike list (one atomic per CTA)
    if (a.spike_list && total > 0) {
        if (threadIdx.x == 0) sm.base = atomicAdd(a.n_spikes, total);
        __syncthreads();
        const int64_t base = sm.base;
        for (int k = threadIdx.x; k < total; k += kStepThreads)
            if (base + k >= 0 && base + k < a.n) a.spike_list[base + k] = sm.ids[k];
    }

    // ---- delay ring: append this CTA's spikes to list t mod S (one atomic)
    if constexpr (RING) {
        if (total > 0) {
            const int64_t ws = tt % a.ring_slots;
            if (threadIdx.x == 0) sm.ring_base = atomicAdd(a.ring + ws, total);
            __syncthreads();
            const int64_t base = sm.ring_base;
            int32_t* list = a.ring + a.ring_slots + ws * a.n;
            for (int k = threadIdx.x; k < total; k += kStepThreads)
                if (base + k >= 0 && base + k < a.n) list[base + k] = sm.ids[k];
        }
    }

    // ---- delivery (network step): lanes in groups of G walk one row each
    int64_t ev = 0;
    if constexpr (CONN == CONN_CSR || CONN == CONN_JIT) {
        const int G = CONN == CONN_CSR ? a.group : 32;  // JIT rows: whole warps
        const int gl = threadIdx.x % G;
        const int ng = kStepThreads / G;
        // called by the G lanes of a group with the same row i
        auto deliver = [&](int32_t i) {
            if constexpr (CONN == CONN_CSR) {
                const CsrArgs& A = a.csr;
                const int64_t b0 = A.indptr[i], b1 = A.indptr[i + 1];
                if (gl == 0) ev += b1 - b0;
                scatter_segment<Y, WK, true>(A.indices, A.data, A.w_homo, b0, b1, gl, G, i < a.n_e ? out_e : out_i, 0);
            } else {
                const bool upper = i >= a.n_e;
                const JitArgs& d = upper ? a.ji : a.je;
                Y* out = upper ? out_i : out_e;
                ev += jit_walk<BP_JIT_HOMO>(d, static_cast<uint32_t>(upper ? i - a.n_e : i), a.n,
                                            [&](int64_t q, uint64_t, float w) { red_add_keep(out + q, event_value<Y>(w), keep); });
            }
        };
        // this CTA's own spikes (every projection without delay)
        for (int k = threadIdx.x / G; k < total; k += ng) {
            const int32_t i = sm.ids[k];
            if (RING && (i < a.n_e ? a.delay_e : a.delay_i) > 0) continue;
            deliver(i);
        }
        if constexpr (RING) {
            // the spikes of step t - d of each delayed projection, rows spread
            // over all CTAs (the lists were completed by earlier launches)
            const bool same = a.delay_e == a.delay_i;
            for (int proj = 0; proj < 2; ++proj) {
                const int d = proj ? a.delay_i : a.delay_e;
                if (d == 0 || (proj == 1 && same)) continue;
                const int64_t rs = (tt + a.ring_slots - d) % a.ring_slots;
                const int64_t c = min(static_cast<int64_t>(a.ring[rs]), a.n);
                const int32_t* list = a.ring + a.ring_slots + rs * a.n;
                for (int64_t k = static_cast<int64_t>(blockIdx.x) * ng + threadIdx.x / G; k < c;
                     k += static_cast<int64_t>(gridDim.x) * ng) {
                    const int32_t i = list[k];
                    if (i < 0 || i >= a.n) continue;
                    if (!same && ((i < a.n_e) != (proj == 0))) continue;
                    deliver(i);
                }
            }
        }
    }

    // ---- totals and the per-step record
    if (a.totals || a.ctrl) {
        long long v0 = group_reduce_sum(static_cast<long long>(cnt_e), 32);
        long long v1 = group_reduce_sum(static_cast<long long>(cnt_i), 32);
        long long v2 = group_reduce_sum(static_cast<long long>(ev), 32);
        if (lane == 0) {
            sm.red[0][warp] = v0;
            sm.red[1][warp] = v1;
            sm.red[2][warp] = v2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long se = 0, si = 0, sv = 0;
            for (int w = 0; w < kStepWarps; ++w) {
                se += sm.red[0][w];
                si += sm.red[1][w];
                sv += sm.red[2][w];
            }
            if (a.totals) {
                if (se) atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 0), static_cast<unsigned long long>(se));
                if (si) atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 1), static_cast<unsigned long long>(si));
                if (sv && CONN != CONN_NONE)
                    atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 2), static_cast<unsigned long long>(sv));
            }
            if (a.ctrl && a.ctrl->record && (se | si)) {
                const int64_t idx = a.ctrl->step + a.t_local - a.ctrl->record_base;
                if (idx >= 0 && idx < a.ctrl->record_len) {
                    atomicAdd(a.ctrl->record + 2 * idx, static_cast<int32_t>(se));
                    atomicAdd(a.ctrl->record + 2 * idx + 1, static_cast<int32_t>(si));
                }
            }
        }
    }
    advance_step_counter(a);
}

struct TraceArgs {
    int64_t n, n_e;
    float a_e, a_i, w_e, w_i;
    float* trace;
    const uint8_t* spk;
    float* acc_e;
    float* acc_i;
    int64_t* totals;
    CsrArgs csr;
    int32_t group;
    JitArgs je, ji;
};

// AlignPre (Appendix D): every presynaptic row i updates its trace,
// s_i <- s_i a + z_i (z_i the previous step's spike flag), and, when s_i is
// not zero, adds s_i w_ij to the conductance sum of each target j (stored
// CSR rows walked by G lanes, or JIT rows regenerated by a warp).  Lane 0 of
// a group owns the trace read-modify-write and broadcasts s_i.  totals[2] +=
// the out-degree of the rows with z_i = 1.
template <int CONN, int WK>
__global__ void __launch_bounds__(kStepThreads) k_trace_scatter(TraceArgs a) {
    const int G = CONN == CONN_CSR ? a.group : 32;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const unsigned gmask = G == 32 ? FULL_MASK : ((1u << G) - 1u) << (lane / G * G);
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * (kStepThreads / G);
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * kStepThreads + threadIdx.x) / G;
    const uint64_t keep = l2_keep_policy();
    int64_t ev = 0;
    for (int64_t i = g0; i < a.n; i += ngroups) {
        const bool is_e = i < a.n_e;
        float s = 0.f;
        int z = 0;
        if (gl == 0) {
            z = a.spk[i] != 0;
            s = a.trace[i] * (is_e ? a.a_e : a.a_i) + (z ? 1.f : 0.f);
            a.trace[i] = s;
        }
        s = __shfl_sync(gmask, s, 0, G);
        z = __shfl_sync(gmask, z, 0, G);
        if (s == 0.f) continue;
        float* out = is_e ? a.acc_e : a.acc_i;
        const float wh = is_e ? a.w_e : a.w_i;
        if constexpr (CONN == CONN_CSR) {
            const int64_t b0 = a.csr.indptr[i], b1 = a.csr.indptr[i + 1];
            if (z && gl == 0) ev += b1 - b0;
            for (int64_t j = b0 + gl; j < b1; j += 4 * G) {
                int32_t col[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t jj = j + u * G;
                    col[u] = jj < b1 ? ld_stream(a.csr.indices + jj) : -1;
                    w[u] = jj < b1 ? load_weight<WK>(a.csr.data, jj, wh) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (col[u] >= 0) red_add_keep(out + col[u], s * w[u], keep);
            }
        } else {
            const JitArgs& d = is_e ? a.je : a.ji;
            const int64_t c = jit_walk<BP_JIT_HOMO>(d, static_cast<uint32_t>(is_e ? i : i - a.n_e), a.n,
                                                    [&](int64_t q, uint64_t, float) { red_add_keep(out + q, s * wh, keep); });
            if (z) ev += c;
        }
    }
    if (a.totals) block_add_i64(ev, a.totals + 2);
}

// Dense event flags -> spike list (Appendix B's `events` to the compact form).
__global__ void __launch_bounds__(kStepThreads) k_spike_compact(int64_t n, const uint8_t* __restrict__ events,
                                                               int32_t* __restrict__ spike_list,
                                                               int32_t* __restrict__ n_spikes) {
    __shared__ int32_t warp_sum[kStepWarps];
    __shared__ int32_t s_base;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kStepThreads;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * kStepThreads; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool s = (i < n) && events[i] != 0;
        const unsigned m = __ballot_sync(FULL_MASK, s);
        if (lane == 0) warp_sum[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < kStepWarps; ++w) {
                const int v = warp_sum[w];
                warp_sum[w] = run;
                run += v;
            }
            s_base = run ? atomicAdd(n_spikes, run) : 0;
        }
        __syncthreads();
        if (s) {
            const int64_t pos = static_cast<int64_t>(s_base) + warp_sum[warp] + __popc(m & lanemask_lt());
            if (pos < n) spike_list[pos] = static_cast<int32_t>(i);
        }
        __syncthreads();
    }
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Resident CTAs per SM of a kernel instantiation (cached per kernel).
int resident_per_sm(const void* kernel) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kStepThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    cache[kernel] = nb;
    return nb;
}

// One resident wave when it covers the state (so each CTA's delivery tail is
// paid once per step), more CTAs only when the 32-bit spike mask needs them.
template <typename K>
bp_status launch_k(K kernel, const StepArgs& a, int vec, cudaStream_t s) {
    const int64_t nq = (a.n + vec - 1) / vec;
    const int64_t per_thread = kMaskBits / vec;
    int64_t grid = static_cast<int64_t>(sm_count()) * resident_per_sm(reinterpret_cast<const void*>(kernel));
    const int64_t need_min = (nq + kStepThreads * per_thread - 1) / (kStepThreads * per_thread);
    const int64_t need_max = (nq + kStepThreads - 1) / kStepThreads;
    if (grid > need_max) grid = need_max;
    if (grid < need_min) grid = need_min;
    if (grid < 1) grid = 1;
    // a network step whose grid fills at most half a resident wave is launched
    // with programmatic stream serialisation, so its CTAs are scheduled while
    // the previous step finishes (measured: 4-8 % fewer us per step on the
    // 4 000-neuron network; 5 % more at 64 % of a wave, 3 % more on full
    // waves, where it is not used)
    const int64_t wave = static_cast<int64_t>(sm_count()) * resident_per_sm(reinterpret_cast<const void*>(kernel));
    if (a.ctrl && 2 * grid <= wave) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(grid));
        cfg.blockDim = dim3(kStepThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        BP_CUDA(cudaLaunchKernelEx(&cfg, kernel, a));
        return BP_OK;
    }
    kernel<<<static_cast<unsigned>(grid), kStepThreads, 0, s>>>(a);
    BP_LAUNCHED();
    return BP_OK;
}

template <bool COUNTS, int VEC, bool RING>
bp_status launch_step_conn(const StepArgs& a, int conn, int wk, cudaStream_t s) {
    if (conn == CONN_JIT) return launch_k(k_step<COUNTS, VEC, CONN_JIT, WK_HOMO, RING>, a, VEC, s);
    if (wk == WK_F32) return launch_k(k_step<COUNTS, VEC, CONN_CSR, WK_F32, RING>, a, VEC, s);
    if (wk == WK_BF16) return launch_k(k_step<COUNTS, VEC, CONN_CSR, WK_BF16, RING>, a, VEC, s);
    return launch_k(k_step<COUNTS, VEC, CONN_CSR, WK_HOMO, RING>, a, VEC, s);
}

template <bool COUNTS, int VEC>
bp_status launch_step_vec(const StepArgs& a, int conn, int wk, cudaStream_t s) {
    if (conn == CONN_NONE) return launch_k(k_step<COUNTS, VEC, CONN_NONE, WK_HOMO>, a, VEC, s);
    if constexpr (!COUNTS) {
        if (conn == CONN_PRE) return launch_k(k_step<false, VEC, CONN_PRE, WK_HOMO>, a, VEC, s);
    }
    if (a.ring) return launch_step_conn<COUNTS, VEC, true>(a, conn, wk, s);
    return launch_step_conn<COUNTS, VEC, false>(a, conn, wk, s);
}

bp_status launch_step(const StepArgs& a, bool counts, int conn, int wk, cudaStream_t s) {
    if (a.n == 0) {
        if (a.clear_counter) BP_CUDA(cudaMemsetAsync(a.clear_counter, 0, sizeof(int32_t), s));
        return BP_OK;
    }
    const bool vec = aligned(a.V, 16) && aligned(a.ge, 16) && aligned(a.gi, 16) && aligned(a.ref, 4) &&
                     aligned(a.ye_in, 16) && aligned(a.yi_in, 16) && aligned(a.I_vec, 16) && aligned(a.spk, 4);
    if (counts) return vec ? launch_step_vec<true, 4>(a, conn, wk, s) : launch_step_vec<true, 1>(a, conn, wk, s);
    return vec ? launch_step_vec<false, 4>(a, conn, wk, s) : launch_step_vec<false, 1>(a, conn, wk, s);
}

StepArgs base_args(const LifConst& c, int64_t n, int64_t n_e, float* V, float* ge, float* gi, uint8_t* ref) {
    StepArgs a{};
    a.c = c;
    a.n = n;
    a.n_e = n_e;
    a.V = V;
    a.ge = ge;
    a.gi = gi;
    a.ref = ref;
    return a;
}

}  // namespace

bp_status launch_lif_step(const LifConst& c, int64_t n, int64_t n_e, float* V, float* ge, float* gi,
                          uint8_t* ref, void* ye, void* yi, bool counts, const float* I_vec, uint8_t* spk,
                          int32_t* spike_list, int32_t* n_spikes, int32_t* clear_counter, int64_t* totals,
                          const NetCtrl* ctrl, int32_t t_local, cudaStream_t s) {
    StepArgs a = base_args(c, n, n_e, V, ge, gi, ref);
    a.ye_in = ye;
    a.yi_in = yi;
    a.I_vec = I_vec;
    a.spk = spk;
    a.spike_list = spike_list;
    a.n_spikes = n_spikes;
    a.clear_counter = clear_counter;
    a.totals = totals;
    a.ctrl = ctrl;
    a.t_local = t_local;
    return launch_step(a, counts, CONN_NONE, WK_HOMO, s);
}

bp_status launch_network_step(const NetStepLaunch& L, int parity, int32_t t_local, cudaStream_t s, int32_t advance) {
    StepArgs a = base_args(L.c, L.n, L.n_e, L.V, L.ge, L.gi, L.ref);
    a.adv_ctrl = advance > 0 ? L.ctrl : nullptr;
    a.advance = advance > 0 ? advance : 0;
    const size_t half = static_cast<size_t>(L.n) * 4;
    char* ye = static_cast<char*>(L.ye2);
    char* yi = static_cast<char*>(L.yi2);
    a.ye_in = ye + (parity ? half : 0);
    a.yi_in = yi + (parity ? half : 0);
    a.ye_out = ye + (parity ? 0 : half);
    a.yi_out = yi + (parity ? 0 : half);
    a.ring = L.ring;
    a.ring_slots = L.ring_slots;
    a.delay_e = L.delay_e;
    a.delay_i = L.delay_i;
    a.spk = L.spk;
    a.spike_list = L.spike_list;
    a.n_spikes = L.spike_list ? L.n_spikes + parity : nullptr;
    a.clear_counter = L.spike_list ? L.n_spikes + (parity ^ 1) : nullptr;
    a.totals = L.totals;
    a.ctrl = L.ctrl;
    a.t_local = t_local;
    a.csr = L.csr;
    a.group = L.group;
    a.je = L.je;
    a.ji = L.ji;
    if (L.trace) {
        // AlignPre: traces and W^T s into the first halves, then the neurons
        TraceArgs t{};
        t.n = L.n;
        t.n_e = L.n_e;
        t.a_e = L.c.a_e;
        t.a_i = L.c.a_i;
        t.w_e = L.c.w_e;
        t.w_i = L.c.w_i;
        t.trace = L.trace;
        t.spk = L.spk;
        t.acc_e = static_cast<float*>(L.ye2);
        t.acc_i = static_cast<float*>(L.yi2);
        t.totals = L.totals;
        t.csr = L.csr;
        t.group = L.jit ? 32 : L.group;
        t.je = L.je;
        t.ji = L.ji;
        const int64_t groups_per_cta = kStepThreads / t.group;
        int64_t grid = (L.n + groups_per_cta - 1) / groups_per_cta;
        const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
        if (grid > cap) grid = cap;
        if (L.jit) {
            k_trace_scatter<CONN_JIT, WK_HOMO><<<static_cast<unsigned>(grid), kStepThreads, 0, s>>>(t);
        } else if (L.csr.wkind == WK_F32) {
            k_trace_scatter<CONN_CSR, WK_F32><<<static_cast<unsigned>(grid), kStepThreads, 0, s>>>(t);
        } else if (L.csr.wkind == WK_BF16) {
            k_trace_scatter<CONN_CSR, WK_BF16><<<static_cast<unsigned>(grid), kStepThreads, 0, s>>>(t);
        } else {
            k_trace_scatter<CONN_CSR, WK_HOMO><<<static_cast<unsigned>(grid), kStepThreads, 0, s>>>(t);
        }
        BP_LAUNCHED();
        a.ye_in = ye;
        a.yi_in = yi;
        a.ye_out = a.yi_out = nullptr;
        a.ring = nullptr;
        return launch_step(a, false, CONN_PRE, WK_HOMO, s);
    }
    const int conn = L.jit ? CONN_JIT : CONN_CSR;
    return launch_step(a, L.counts, conn, L.csr.wkind, s);
}

bp_status launch_spike_compact(int64_t n, const uint8_t* events, int32_t* spike_list, int32_t* n_spikes,
                               cudaStream_t s) {
    if (n == 0) return BP_OK;
    int64_t grid = (n + kStepThreads - 1) / kStepThreads;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    if (grid > cap) grid = cap;
    k_spike_compact<<<static_cast<unsigned>(grid), kStepThreads, 0, s>>>(n, events, spike_list, n_spikes);
    BP_LAUNCHED();
    return BP_OK;
}

}  // namespace bp

extern "C" {

bp_status bp_lif_step(const bp_coba_params* p, int64_t n, int64_t n_e, float* V, float* ge, float* gi,
                      uint8_t* ref, void* ye, void* yi, int32_t y_is_count, const float* I_vec, uint8_t* spk,
                      int32_t* spike_list, int32_t* n_spikes, int64_t* spike_totals, bp_stream_t stream) {
    bp::clear_error();
    BP_TRY(bp::check_coba(p));
    BP_REQUIRE(n >= 0 && n <= INT32_MAX, "n = %lld out of range", (long long)n);
    BP_REQUIRE(n_e >= 0 && n_e <= n, "n_e = %lld not in [0, n]", (long long)n_e);
    BP_REQUIRE(n == 0 || (V && ge && gi && ref && ye && yi), "a required state pointer is NULL");
    BP_REQUIRE(!spike_list == !n_spikes, "spike_list and n_spikes must both be given or both be NULL");
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
