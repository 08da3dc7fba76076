// snn.cu -- the differentiable recurrent spiking network and its BPTT
// adjoint (a10; Appendix I, Section 4.1: operators with reverse-mode rules).
//
// Model (per batch element; t = 1..T):
//   I_t  = a_s I_{t-1} + W_rec^T z_{t-1} + W_in^T u_t
//   Vp_t = a_m V_{t-1} + (1 - a_m)(V_rest + R I_t),  z_t = [Vp_t > V_th],
//   V_t  = z_t ? V_reset : Vp_t (reset detached from the gradient),
//   y_t  = a_o y_{t-1} + dt (W_out^T z_t + b),  m = mean_t y_t.
// Loss: cross-entropy of softmax(m) (mean over the batch) plus, when
// lambda_v > 0, the voltage regulariser of Appendix I,
//   L_v = (lambda_v / B) sum_{b,t,i} [max(Vp - v_hi, 0)^2 + max(v_lo - Vp, 0)^2].
// Adjoint (t = T..1), with surrogate s'(x) = k s(kx)(1 - s(kx)) (logistic) or
// max(0, alpha (width - |x|)) (ReLU, Appendix I):
//   ybar_t = a_o ybar_{t+1} + g_m / T
//   zbar_t = dt W_out ybar_t + W_rec Ibar_{t+1}          (gather over rows)
//   Vpbar_t = Vbar_t (1 - z_t) + zbar_t s'(Vp_t - V_th) + dL_v/dVp_t
//   Ibar_t = (1 - a_m) R Vpbar_t + a_s Ibar_{t+1},  Vbar_{t-1} = a_m Vpbar_t
//   dW_out += dt z_t ybar_t^T, db += dt ybar_t, dW_in += u_t Ibar_t^T,
//   dw_rec[j] += Ibar_t[col j] for every entry j of rows spiking at t - 1.
//
// One CTA per batch element, the neuron state in shared memory.  Forward:
// input spikes of the step are compacted (ballot) and their W_in rows summed
// per neuron; the previous step's spikes are delivered through the CSR rows
// (one warp per row) into a shared-memory accumulator; the readout sums the
// W_out rows of the step's spikes.  Every K steps the state (I, V, y) is
// checkpointed, and every step's spike bits are recorded (n_rec / 8 bytes per
// step).  Backward: for each K-step segment, last first, the forward is
// recomputed from its checkpoint storing Vp_t, with the recorded spikes
// replayed rather than re-decided (the shared-memory float atomics may round
// differently from the forward, and a near-threshold neuron must not take
// the other branch); the adjoint then runs back through the segment.  The
// forward stores the last segment's potentials itself, so that segment (and,
// with a single segment, the whole run) is not recomputed.  The
// recurrent weights are converted to fixed point once per forward call
// (k_snn_fix_weights), so delivering an event is one integer atomic.
// Recurrent weights are FP32 or BF16 (FP32 arithmetic).  The adjoint stores
// Ibar_t of every step; the input and recurrent weight gradients are then one
// dense contraction over batch and time on the tensor cores,
//   G = [u_t ; z_{t-1}]^T Ibar_t  summed over (b, t)      (tcgemm.cu),
// whose first n_in rows are dW_in and whose recurrent rows, read at the
// stored entries, are dw_rec (k_snn_grad_scatter).  dW_out and db are kept
// per batch element and summed over the batch in a fixed order
// (k_snn_reduce).  Every gradient is reproducible bit for bit.
#include <cmath>

#include "bp_common.cuh"
#include "bp_internal.h"

namespace bp {
namespace {

constexpr int kSnnThreads = 1024;
constexpr int kSnnMaxRec = 4096;
constexpr int kSnnMaxIn = 4096;
constexpr int kSnnMaxOut = 64;

// Surrogate derivative and voltage-regulariser constants.
struct SgK {
    int32_t kind;                        // BP_SG_SIGMOID or BP_SG_RELU
    int32_t reg_on;                      // lambda_v > 0
    float slope, alpha, width;
    float reg_scale, v_hi, v_lo;         // reg_scale = lambda_v / B
};

__device__ __forceinline__ float surrogate(const SgK& g, float x) {
    if (g.kind == BP_SG_RELU) return fmaxf(0.f, g.alpha * (g.width - fabsf(x)));
    const float s = 1.f / (1.f + expf(-g.slope * x));
    return g.slope * s * (1.f - s);
}

__device__ __forceinline__ float penalty(const SgK& g, float vp) {
    const float a = fmaxf(vp - g.v_hi, 0.f), b = fmaxf(g.v_lo - vp, 0.f);
    return a * a + b * b;
}

// dL_v/dVp of one element (zero when the regulariser is off).
__device__ __forceinline__ float penalty_grad(const SgK& g, float vp) {
    if (!g.reg_on) return 0.f;
    return g.reg_scale * (2.f * fmaxf(vp - g.v_hi, 0.f) - 2.f * fmaxf(g.v_lo - vp, 0.f));
}

struct SnnK {
    int32_t B, T, n_in, n_rec, n_out, K;
    float a_s, a_m, a_o, dt, V_rest, V_reset, V_th, R;
    SgK sg;
    const float* W_in;
    const int64_t* indptr;
    const int32_t* indices;
    const void* w_rec;
    const float* W_out;
    const float* b_out;
    // workspace
    float* ck_I;         // [B][n_ck][n_rec]
    float* ck_V;         // [B][n_ck][n_rec]
    float* ck_y;         // [B][n_ck][n_out]
    uint32_t* z_all;     // [B][T][zw]  spike bits of every step (recorded by the forward)
    float* seg_Vp;       // [B][K][n_rec]
    float* ib_all;       // [B][T][n_rec]  Ibar_t of every step (input of the weight-gradient contraction)
    float* g_out;        // [B][n_rec][n_out]  per-batch-element gradient partials
    float* g_b;          // [B][n_out]
    float* vreg;         // [B]  regulariser sums of the forward
    int32_t stage_wout;  // the forward copies W_out into shared memory (it fits)
    unsigned long long* w_fix;  // [nnz] recurrent weights in fixed point (filled by the forward)
    int64_t nnz;
    int32_t n_ck, zw;
};

template <int WK>
__device__ __forceinline__ float w_at(const void* w, int64_t j) {
    if constexpr (WK == BP_W_BF16) {
        const unsigned short raw = static_cast<const unsigned short*>(w)[j];
        return __uint_as_float(static_cast<uint32_t>(raw) << 16);
    } else {
        return static_cast<const float*>(w)[j];
    }
}

// Recurrent input is accumulated as a 64-bit fixed-point number (scale 2^32):
// integer additions commute, so the sum - and with it every spike decision -
// does not depend on the order in which the delivering warps arrive, and the
// backward pass recomputes the forward bit for bit.  Weights of magnitude
// above 2^-9 convert exactly; sums are exact up to |sum| < 2^31.
// Scaling by a power of two is exact in FP32, so the conversions need no FP64
// arithmetic (whose rate is low on this GPU): one rounding float -> int64 on
// the way in, one rounding int64 -> float on the way out.
__device__ __forceinline__ unsigned long long to_fix(float w) {
    return static_cast<unsigned long long>(__float2ll_rn(w * 4294967296.0f));
}
__device__ __forceinline__ float from_fix(unsigned long long v) {
    return __ll2float_rn(static_cast<long long>(v)) * (1.0f / 4294967296.0f);
}

// Compacts the active inputs of step t into list (shared) in increasing index
// order (ballot per warp, prefix over warps), so that the input current sums
// the W_in rows in a fixed order.  Returns the count.
__device__ __forceinline__ int gather_inputs(const uint8_t* __restrict__ ut, int n_in, int32_t* list,
                                             int32_t* counter) {
    __shared__ int32_t s_wpre[kSnnThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) *counter = 0;
    __syncthreads();
    for (int base = 0; base < n_in; base += kSnnThreads) {
        const int k = base + threadIdx.x;
        const bool on = k < n_in && ut[k] != 0;
        const unsigned m = __ballot_sync(FULL_MASK, on);
        if (lane == 0) s_wpre[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = *counter;
            for (int w = 0; w < kSnnThreads / 32; ++w) {
                const int c = s_wpre[w];
                s_wpre[w] = run;
                run += c;
            }
            *counter = run;
        }
        __syncthreads();
        if (on) list[s_wpre[warp] + __popc(m & lanemask_lt())] = k;
        __syncthreads();
    }
    return *counter;
}

// Compensated (Kahan) FP32 running sum: s holds the sum, c the low-order
// part lost so far; the result is s - c.  The regulariser's per-thread sums
// use it so that FP32 keeps ~1e-7 relative accuracy over the T x n_rec terms
// without FP64 arithmetic on the GPU.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s - c; }
};

// One step of the neuron state held in shared memory.  racc holds
// W_rec^T z_{t-1} and is cleared.  Spikes are decided by the threshold, or,
// when force_z is given, taken from those recorded bits (the backward pass
// replays the forward's spikes so that its recomputation cannot take another
// branch).  The step's spikes are appended to spk; zbits (nullable) receives
// their bits; Vp_out (nullable) the potentials before reset; reg (nullable)
// accumulates this thread's regulariser terms.
__device__ __forceinline__ void neuron_step(const SnnK& p, float* I, float* V, unsigned long long* racc,
                                            const int32_t* in_list,
                                            int n_act, int32_t* spk, int32_t* n_spk, float* Vp_out,
                                            uint32_t* zbits, const uint32_t* force_z, KahanF* reg) {
    for (int jb = 0; jb < p.n_rec; jb += kSnnThreads) {
        const int j = jb + threadIdx.x;
        bool z = false;
        if (j < p.n_rec) {
            float in = 0.f;
            int a = 0;
            for (; a + 4 <= n_act; a += 4) {  // four row loads in flight, summed in list order
                const float x0 = __ldg(p.W_in + static_cast<int64_t>(in_list[a]) * p.n_rec + j);
                const float x1 = __ldg(p.W_in + static_cast<int64_t>(in_list[a + 1]) * p.n_rec + j);
                const float x2 = __ldg(p.W_in + static_cast<int64_t>(in_list[a + 2]) * p.n_rec + j);
                const float x3 = __ldg(p.W_in + static_cast<int64_t>(in_list[a + 3]) * p.n_rec + j);
                in += x0;
                in += x1;
                in += x2;
                in += x3;
            }
            for (; a < n_act; ++a) in += __ldg(p.W_in + static_cast<int64_t>(in_list[a]) * p.n_rec + j);
            const float Ij = p.a_s * I[j] + from_fix(racc[j]) + in;
            racc[j] = 0ull;
            I[j] = Ij;
            const float vp = p.a_m * V[j] + (1.f - p.a_m) * (p.V_rest + p.R * Ij);
            z = force_z ? ((force_z[j >> 5] >> (j & 31)) & 1u) != 0 : vp > p.V_th;
            V[j] = z ? p.V_reset : vp;
            if (Vp_out) Vp_out[j] = vp;
            if (reg) reg->add(penalty(p.sg, vp));
        }
        const unsigned m = __ballot_sync(FULL_MASK, z);
        if ((threadIdx.x & 31) == 0) {
            if (zbits && jb + threadIdx.x < p.n_rec) zbits[(jb + threadIdx.x) >> 5] = m;
            if (m) {
                int pos = atomicAdd(n_spk, __popc(m));
                for (unsigned mm = m; mm; mm &= mm - 1) spk[pos++] = jb + threadIdx.x + __ffs(mm) - 1;
            }
        }
    }
}

// racc[col] += w for every entry of the rows in spk[0..n) (one warp per row),
// in fixed point (the weights were converted once per call, so a delivered
// event is one integer shared-memory atomic).
__device__ __forceinline__ void deliver(const SnnK& p, const int32_t* spk, int n, unsigned long long* racc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = warp; e < n; e += kSnnThreads / 32) {
        const int i = spk[e];
        const int64_t b0 = p.indptr[i], b1 = p.indptr[i + 1];
        // four index / weight loads in flight per lane before the atomics: a
        // row of up to 128 entries costs one memory latency
        for (int64_t j = b0 + lane; j < b1; j += 4 * 32) {
            int32_t c[4];
            unsigned long long w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t jj = j + 32 * u;
                c[u] = jj < b1 ? p.indices[jj] : -1;
                w[u] = jj < b1 ? p.w_fix[jj] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c[u] >= 0) atomicAdd(racc + c[u], w[u]);
        }
    }
}

// w_fix[j] = to_fix(w_rec[j]) for all stored recurrent weights.
template <int WK>
__global__ void k_snn_fix_weights(const void* __restrict__ w, int64_t nnz, unsigned long long* __restrict__ w_fix) {
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < nnz;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x)
        w_fix[j] = to_fix(w_at<WK>(w, j));
}

template <int WK>
__global__ void __launch_bounds__(kSnnThreads, 1) k_snn_forward(SnnK p, const uint8_t* __restrict__ u,
                                                               float* __restrict__ m_out) {
    extern __shared__ __align__(16) float sh[];
    unsigned long long* racc = reinterpret_cast<unsigned long long*>(sh);
    float* I = reinterpret_cast<float*>(racc + p.n_rec);
    float* V = I + p.n_rec;
    int32_t* spk = reinterpret_cast<int32_t*>(V + p.n_rec);
    int32_t* in_list = spk + p.n_rec;
    float* s_wout = reinterpret_cast<float*>(in_list + p.n_in);  // [n_rec][n_out] when staged
    __shared__ int32_t s_cnt[2];
    __shared__ float s_y[kSnnMaxOut], s_m[kSnnMaxOut];
    const int b = blockIdx.x;
    for (int j = threadIdx.x; j < p.n_rec; j += kSnnThreads) {
        I[j] = V[j] = 0.f;
        racc[j] = 0ull;
    }
    if (p.stage_wout)
        for (int e = threadIdx.x; e < p.n_rec * p.n_out; e += kSnnThreads) s_wout[e] = __ldg(p.W_out + e);
    const float* Wo = p.stage_wout ? s_wout : p.W_out;  // readout weights, shared or global
    if (threadIdx.x < p.n_out) s_y[threadIdx.x] = s_m[threadIdx.x] = 0.f;
    KahanF reg;
    const int t_last0 = ((p.T - 1) / p.K) * p.K;  // first step of the last checkpoint segment
    __syncthreads();
    for (int t = 0; t < p.T; ++t) {
        if (t % p.K == 0) {  // checkpoint of the state before step t
            const int64_t o = static_cast<int64_t>(b) * p.n_ck + t / p.K;
            for (int j = threadIdx.x; j < p.n_rec; j += kSnnThreads) {
                p.ck_I[o * p.n_rec + j] = I[j];
                p.ck_V[o * p.n_rec + j] = V[j];
            }
            if (threadIdx.x < p.n_out) p.ck_y[o * p.n_out + threadIdx.x] = s_y[threadIdx.x];
        }
        const int n_act = gather_inputs(u + (static_cast<int64_t>(b) * p.T + t) * p.n_in, p.n_in, in_list, &s_cnt[0]);
        if (threadIdx.x == 0) s_cnt[1] = 0;
        __syncthreads();
        // the potentials of the last checkpoint segment go straight to the
        // segment buffer, so the backward need not recompute that segment
        float* vp_out = t >= t_last0 ? p.seg_Vp + (static_cast<int64_t>(b) * p.K + (t - t_last0)) * p.n_rec : nullptr;
        neuron_step(p, I, V, racc, in_list, n_act, spk, &s_cnt[1], vp_out,
                    p.z_all + (static_cast<int64_t>(b) * p.T + t) * p.zw, nullptr, p.sg.reg_on ? &reg : nullptr);
        __syncthreads();
        const int n = s_cnt[1];
        deliver(p, spk, n, racc);
        {
            // W_out^T z_t: one warp per output, lanes over the recorded spike words
            // in a fixed order and a fixed reduction tree, so the readout is reproducible
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const uint32_t* zt = p.z_all + (static_cast<int64_t>(b) * p.T + t) * p.zw;
            for (int o = warp; o < p.n_out; o += kSnnThreads / 32) {
                float acc = 0.f;
                for (int w = lane; w < p.zw; w += 32)
                    for (uint32_t bits = zt[w]; bits; bits &= bits - 1)
                        acc += Wo[static_cast<int64_t>(32 * w + __ffs(bits) - 1) * p.n_out + o];
                acc = group_reduce_sum(acc, 32);
                if (lane == 0) {
                    const float y = p.a_o * s_y[o] + p.dt * (acc + p.b_out[o]);
                    s_y[o] = y;
                    s_m[o] += y;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < p.n_out) m_out[static_cast<int64_t>(b) * p.n_out + threadIdx.x] = s_m[threadIdx.x] / p.T;
    if (p.sg.reg_on) {  // fixed reduction order: lanes by a tree, warps in index order
        __shared__ float s_reg[kSnnThreads / 32];
        const float v = group_reduce_sum(reg.value(), 32);
        if ((threadIdx.x & 31) == 0) s_reg[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            KahanF acc;
            for (int w = 0; w < kSnnThreads / 32; ++w) acc.add(s_reg[w]);
            p.vreg[b] = acc.value();
        }
    }
}

template <int WK>
__global__ void __launch_bounds__(kSnnThreads, 1) k_snn_backward(SnnK p, const uint8_t* __restrict__ u,
                                                                const float* __restrict__ g_m) {
    extern __shared__ __align__(16) float sh[];
    unsigned long long* racc = reinterpret_cast<unsigned long long*>(sh);
    float* I = reinterpret_cast<float*>(racc + p.n_rec);  // recompute state
    float* V = I + p.n_rec;
    float* Ib_next = V + p.n_rec;     // Ibar_{t+1} (overwritten by Ibar_t once zbar_t is formed)
    float* Zb = Ib_next + p.n_rec;    // zbar_t
    float* Vb = Zb + p.n_rec;         // Vbar_t
    int32_t* spk = reinterpret_cast<int32_t*>(Vb + p.n_rec);
    int32_t* in_list = spk + p.n_rec;
    __shared__ int32_t s_cnt[2];
    __shared__ float s_yb[kSnnMaxOut], s_gm[kSnnMaxOut];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31;
    // this batch element's readout-gradient partials (summed over the batch
    // afterwards in a fixed order) and its row of Ibar per step
    float* gout = p.g_out + static_cast<int64_t>(b) * p.n_rec * p.n_out;
    float* ib_b = p.ib_all + static_cast<int64_t>(b) * p.T * p.n_rec;
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(p.n_rec) * p.n_out; e += kSnnThreads) gout[e] = 0.f;
    for (int j = threadIdx.x; j < p.n_rec; j += kSnnThreads) Ib_next[j] = Vb[j] = 0.f;
    if (threadIdx.x < p.n_out) {
        s_yb[threadIdx.x] = 0.f;
        s_gm[threadIdx.x] = g_m[static_cast<int64_t>(b) * p.n_out + threadIdx.x];
    }
    float db_acc = 0.f;
    float* segVp = p.seg_Vp + static_cast<int64_t>(b) * p.K * p.n_rec;
    const uint32_t* zall = p.z_all + static_cast<int64_t>(b) * p.T * p.zw;
    const int nseg = (p.T + p.K - 1) / p.K;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int t0 = seg * p.K;
        const int t1 = min(p.T, t0 + p.K);
        const int64_t o = static_cast<int64_t>(b) * p.n_ck + seg;
        // ---- recompute the segment from its checkpoint (the last segment's
        // potentials were stored by the forward; with a single segment nothing
        // is recomputed)
        __syncthreads();
        if (seg < nseg - 1) {
            for (int j = threadIdx.x; j < p.n_rec; j += kSnnThreads) {
                I[j] = p.ck_I[o * p.n_rec + j];
                V[j] = p.ck_V[o * p.n_rec + j];
                racc[j] = 0ull;
            }
            if (threadIdx.x == 0) s_cnt[1] = 0;
            __syncthreads();
            if (t0 > 0) {  // pending input of the spikes of step t0 - 1
                const uint32_t* zp = zall + static_cast<int64_t>(t0 - 1) * p.zw;
                for (int w = threadIdx.x; w < p.zw; w += kSnnThreads) {
                    uint32_t bits = zp[w];
                    if (bits) {
                        int q = atomicAdd(&s_cnt[1], __popc(bits));
                        for (; bits; bits &= bits - 1) spk[q++] = 32 * w + __ffs(bits) - 1;
                    }
                }
            }
            __syncthreads();
            deliver(p, spk, s_cnt[1], racc);
            __syncthreads();
            for (int t = t0; t < t1; ++t) {
                const int n_act = gather_inputs(u + (static_cast<int64_t>(b) * p.T + t) * p.n_in, p.n_in, in_list, &s_cnt[0]);
                if (threadIdx.x == 0) s_cnt[1] = 0;
                __syncthreads();
                neuron_step(p, I, V, racc, in_list, n_act, spk, &s_cnt[1], segVp + static_cast<int64_t>(t - t0) * p.n_rec,
                            nullptr, zall + static_cast<int64_t>(t) * p.zw, nullptr);
                __syncthreads();
                deliver(p, spk, s_cnt[1], racc);
                __syncthreads();
            }
        }
        // ---- adjoint, t = t1-1 .. t0
        for (int t = t1 - 1; t >= t0; --t) {
            if (threadIdx.x < p.n_out) {
                const float yb = p.a_o * s_yb[threadIdx.x] + s_gm[threadIdx.x] / p.T;
                s_yb[threadIdx.x] = yb;
                db_acc += p.dt * yb;
            }
            __syncthreads();
            const float* Vp = segVp + static_cast<int64_t>(t - t0) * p.n_rec;
            const uint32_t* zb = zall + static_cast<int64_t>(t) * p.zw;
            // zbar_j: recurrent part W_rec Ibar_{t+1} plus the readout part; groups of
            // 8 lanes per row, so a warp has four rows' loads in flight
            {
                constexpr int G = 8;
                const int gl = lane & (G - 1);
                for (int jb = 0; jb < p.n_rec; jb += kSnnThreads / G) {
                    const int j = jb + threadIdx.x / G;
                    float acc = 0.f;
                    if (j < p.n_rec) {
                        const int64_t r0 = p.indptr[j], r1 = p.indptr[j + 1];
                        for (int64_t e = r0 + gl; e < r1; e += G) acc += w_at<WK>(p.w_rec, e) * Ib_next[p.indices[e]];
                        for (int oo = gl; oo < p.n_out; oo += G)
                            acc += p.dt * __ldg(p.W_out + static_cast<int64_t>(j) * p.n_out + oo) * s_yb[oo];
                    }
                    acc = group_reduce_sum(acc, G);
                    if (j < p.n_rec && gl == 0) Zb[j] = acc;
                }
            }
            __syncthreads();
            for (int j = threadIdx.x; j < p.n_rec; j += kSnnThreads) {
                const float zbar = Zb[j];
                const bool z = (zb[j >> 5] >> (j & 31)) & 1u;
                const float vpb = Vb[j] * (z ? 0.f : 1.f) + zbar * surrogate(p.sg, Vp[j] - p.V_th) +
                                  penalty_grad(p.sg, Vp[j]);
                const float ib = (1.f - p.a_m) * p.R * vpb + p.a_s * Ib_next[j];
                Ib_next[j] = ib;  // Ibar_t is the next (earlier) step's Ibar_{t+1}; column j is this thread's
                ib_b[static_cast<int64_t>(t) * p.n_rec + j] = ib;  // dW_in and dw_rec come from these
                Vb[j] = p.a_m * vpb;
                if (z) {  // dW_out[j, :] += dt ybar_t (row j belongs to this thread)
                    float* row = gout + static_cast<int64_t>(j) * p.n_out;
                    for (int oo = 0; oo < p.n_out; ++oo) row[oo] += p.dt * s_yb[oo];
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x < p.n_out) p.g_b[static_cast<int64_t>(b) * p.n_out + threadIdx.x] = db_acc;
}

// out[e] += sum over the batch of part[b][e], b in order (reproducible).
__global__ void k_snn_reduce(const float* __restrict__ part, int32_t B, int64_t n, float* __restrict__ out) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < B; ++b) acc += part[static_cast<int64_t>(b) * n + e];
        out[e] += acc;
    }
}

// dW_in[k][j] += G[k][j] for the n_in input rows of G; dw_rec[e] +=
// G[n_in + i][indices[e]] for every stored entry e of recurrent row i (the
// dense recurrent gradient read at the stored entries).
__global__ void k_snn_grad_scatter(const float* __restrict__ G, int32_t n_in, int32_t n_rec,
                                   const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                   float* __restrict__ dW_in, float* __restrict__ dw_rec) {
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t n_w = static_cast<int64_t>(n_in) * n_rec;
    for (int64_t e = tid; e < n_w; e += stride) dW_in[e] += G[e];
    const int lane = threadIdx.x & 31;
    for (int64_t i = tid >> 5; i < n_rec; i += stride >> 5) {
        const float* g = G + (static_cast<int64_t>(n_in) + i) * n_rec;
        const int64_t e1 = indptr[i + 1];
        for (int64_t e = indptr[i] + lane; e < e1; e += 32) dw_rec[e] += g[indices[e]];
    }
}

// Adjoint of one LIF step, elementwise (the update k_snn_backward applies per
// neuron): Vpbar = Vbar (1 - z) + zbar s'(Vp - V_th) + dL_v/dVp, Ibar =
// (1 - a_m) R Vpbar + a_s Ibar_next, Vbar_prev = a_m Vpbar.
__global__ void k_lif_step_bwd(int64_t n, float a_m, float a_s, float R, float V_th, SgK sg,
                               const float* __restrict__ Vp, const uint8_t* __restrict__ z,
                               const float* __restrict__ Vbar, const float* __restrict__ zbar,
                               const float* __restrict__ Ibar_next, float* __restrict__ Ibar,
                               float* __restrict__ Vbar_prev) {
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float vpb = Vbar[j] * (z[j] ? 0.f : 1.f) + zbar[j] * surrogate(sg, Vp[j] - V_th) + penalty_grad(sg, Vp[j]);
        Ibar[j] = (1.f - a_m) * R * vpb + a_s * Ibar_next[j];
        Vbar_prev[j] = a_m * vpb;
    }
}

// Mean cross-entropy of softmax(m) over the batch and its gradient, in FP32:
// one thread per batch element (max-subtracted log-sum-exp over the outputs
// in index order), the per-element terms added in batch order with a
// compensated sum, so the loss is reproducible and accurate to ~1e-7.
__global__ void k_snn_loss(int32_t B, int32_t n_out, const float* __restrict__ m, const int64_t* __restrict__ labels,
                           float* __restrict__ loss, float* __restrict__ g_m) {
    __shared__ float s_term[256];
    KahanF total;
    for (int b0 = 0; b0 < B; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        float term = 0.f;
        if (b < B) {
            const float* mb = m + static_cast<int64_t>(b) * n_out;
            float mx = mb[0];
            for (int o = 1; o < n_out; ++o) mx = fmaxf(mx, mb[o]);
            float se = 0.f;
            for (int o = 0; o < n_out; ++o) se += expf(mb[o] - mx);
            const int64_t lab = labels[b];
            term = (logf(se) + mx) - mb[lab];
            const float inv = 1.f / se;
            for (int o = 0; o < n_out; ++o) {
                const float sm = expf(mb[o] - mx) * inv;
                g_m[static_cast<int64_t>(b) * n_out + o] = (sm - (o == lab ? 1.f : 0.f)) / static_cast<float>(B);
            }
        }
        s_term[threadIdx.x] = term;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < static_cast<int>(blockDim.x) && b0 + k < B; ++k) total.add(s_term[k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = total.value() / static_cast<float>(B);
}

// loss[0] += scale * sum_b vreg[b], the sum in batch order (compensated FP32).
__global__ void k_snn_reg_add(int32_t B, float scale, const float* __restrict__ vreg, float* __restrict__ loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    KahanF acc;
    for (int b = 0; b < B; ++b) acc.add(vreg[b]);
    loss[0] = loss[0] + scale * acc.value();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct SnnLayout {
    size_t ck_I, ck_V, ck_y, z_all, seg_Vp, ib_all, g_full, tc_work, tc_bytes, g_out, g_b, vreg, w_fix, total;
    int32_t n_ck, zw;
};

SnnLayout snn_layout(const bp_snn_desc& d) {
    SnnLayout L{};
    const int K = d.ckpt_every > 0 ? d.ckpt_every : d.T;
    L.n_ck = (d.T + K - 1) / K;
    if (L.n_ck < 1) L.n_ck = 1;
    L.zw = (d.n_rec + 31) / 32;
    size_t o = 0;
    const size_t B = d.B;
    L.ck_I = o; o = align256(o + B * L.n_ck * d.n_rec * 4);
    L.ck_V = o; o = align256(o + B * L.n_ck * d.n_rec * 4);
    L.ck_y = o; o = align256(o + B * L.n_ck * d.n_out * 4);
    L.z_all = o; o = align256(o + B * static_cast<size_t>(d.T) * L.zw * 4);
    L.seg_Vp = o; o = align256(o + B * static_cast<size_t>(K) * d.n_rec * 4);
    L.ib_all = o; o = align256(o + B * static_cast<size_t>(d.T) * d.n_rec * 4);
    // G = [u ; z_shifted]^T Ibar: rows n_in + n_rec, row stride n_rec
    L.g_full = o; o = align256(o + (static_cast<size_t>(d.n_in) + d.n_rec) * d.n_rec * 4);
    // the contraction's workspace must be 1024-byte aligned in memory, the
    // snn workspace only 256: 768 bytes of slack let snn_kernel_args align it
    L.tc_bytes = tc_spike_gemm_workspace(d.B, d.T, d.n_rec, d.n_in + d.n_rec);
    L.tc_work = o; o = align256(o + L.tc_bytes + 768);
    L.g_out = o; o = align256(o + B * static_cast<size_t>(d.n_rec) * d.n_out * 4);
    L.g_b = o; o = align256(o + B * static_cast<size_t>(d.n_out) * 4);
    L.vreg = o; o = align256(o + B * 4);
    L.w_fix = o; o = align256(o + static_cast<size_t>(d.nnz > 0 ? d.nnz : 0) * 8);
    L.total = o;
    return L;
}

bp_status sg_check(const bp_snn_desc* d) {
    BP_REQUIRE(d->surrogate == BP_SG_SIGMOID || d->surrogate == BP_SG_RELU, "unknown surrogate %d", d->surrogate);
    BP_REQUIRE(d->surrogate != BP_SG_RELU || (d->sg_alpha >= 0 && d->sg_width > 0),
               "ReLU surrogate needs sg_alpha >= 0 and sg_width > 0");
    BP_REQUIRE(d->lambda_v >= 0, "lambda_v < 0");
    BP_REQUIRE(d->lambda_v == 0 || d->v_lo < d->v_hi, "regulariser bounds need v_lo < v_hi");
    return BP_OK;
}

SgK make_sg(const bp_snn_desc& d) {
    SgK g;
    g.kind = d.surrogate;
    g.reg_on = d.lambda_v > 0 ? 1 : 0;
    g.slope = static_cast<float>(d.slope);
    g.alpha = static_cast<float>(d.sg_alpha);
    g.width = static_cast<float>(d.sg_width);
    g.reg_scale = static_cast<float>(d.lambda_v / (d.B > 0 ? d.B : 1));
    g.v_hi = static_cast<float>(d.v_hi);
    g.v_lo = static_cast<float>(d.v_lo);
    return g;
}

bp_status snn_check(const bp_snn_desc* d) {
    BP_REQUIRE(d != nullptr, "desc is NULL");
    BP_REQUIRE(d->B > 0 && d->T > 0, "B and T must be positive");
    BP_REQUIRE(d->n_in > 0 && d->n_in <= kSnnMaxIn, "n_in must be in [1, %d]", kSnnMaxIn);
    BP_REQUIRE(d->n_rec > 0 && d->n_rec <= kSnnMaxRec, "n_rec must be in [1, %d]", kSnnMaxRec);
    BP_REQUIRE(d->n_out > 0 && d->n_out <= kSnnMaxOut, "n_out must be in [1, %d]", kSnnMaxOut);
    BP_REQUIRE(d->ckpt_every >= 0, "ckpt_every < 0");
    BP_REQUIRE(d->w_rec_kind == BP_W_F32 || d->w_rec_kind == BP_W_BF16, "recurrent weights must be F32 or BF16");
    BP_REQUIRE(d->W_in && d->indptr && d->indices && d->w_rec && d->W_out && d->b_out, "a parameter pointer is NULL");
    BP_REQUIRE(d->nnz >= 0, "nnz < 0");
    BP_REQUIRE(d->tau_m > 0 && d->tau_s > 0 && d->tau_o > 0 && d->dt > 0, "time constants must be positive");
    BP_TRY(sg_check(d));
    return BP_OK;
}

SnnK snn_kernel_args(const bp_snn_desc& d, void* ws) {
    const SnnLayout L = snn_layout(d);
    SnnK p;
    p.stage_wout = 0;
    p.B = d.B;
    p.T = d.T;
    p.n_in = d.n_in;
    p.n_rec = d.n_rec;
    p.n_out = d.n_out;
    p.K = d.ckpt_every > 0 ? d.ckpt_every : d.T;
    p.a_s = static_cast<float>(std::exp(-d.dt / d.tau_s));
    p.a_m = static_cast<float>(std::exp(-d.dt / d.tau_m));
    p.a_o = static_cast<float>(std::exp(-d.dt / d.tau_o));
    p.dt = static_cast<float>(d.dt);
    p.V_rest = static_cast<float>(d.V_rest);
    p.V_reset = static_cast<float>(d.V_reset);
    p.V_th = static_cast<float>(d.V_th);
    p.R = static_cast<float>(d.R);
    p.sg = make_sg(d);
    p.W_in = d.W_in;
    p.indptr = d.indptr;
    p.indices = d.indices;
    p.w_rec = d.w_rec;
    p.W_out = d.W_out;
    p.b_out = d.b_out;
    char* w = static_cast<char*>(ws);
    p.ck_I = reinterpret_cast<float*>(w + L.ck_I);
    p.ck_V = reinterpret_cast<float*>(w + L.ck_V);
    p.ck_y = reinterpret_cast<float*>(w + L.ck_y);
    p.z_all = reinterpret_cast<uint32_t*>(w + L.z_all);
    p.seg_Vp = reinterpret_cast<float*>(w + L.seg_Vp);
    p.ib_all = reinterpret_cast<float*>(w + L.ib_all);
    p.g_out = reinterpret_cast<float*>(w + L.g_out);
    p.g_b = reinterpret_cast<float*>(w + L.g_b);
    p.vreg = reinterpret_cast<float*>(w + L.vreg);
    p.w_fix = reinterpret_cast<unsigned long long*>(w + L.w_fix);
    p.nnz = d.nnz;
    p.n_ck = L.n_ck;
    p.zw = L.zw;
    return p;
}

template <typename Kern>
bp_status set_smem(Kern k, size_t bytes) {
    return ensure_smem_attr(reinterpret_cast<const void*>(k), static_cast<int>(bytes));
}

}  // namespace
}  // namespace bp

extern "C" {

bp_status bp_snn_desc_default(bp_snn_desc* d) {
    bp::clear_error();
    BP_REQUIRE(d != nullptr, "desc is NULL");
    *d = bp_snn_desc{};
    d->dt = 1.0;
    d->tau_m = 20.0;
    d->tau_s = 100.0;
    d->tau_o = 20.0;
    d->V_rest = 0.0;
    d->V_reset = 0.0;
    d->V_th = 1.0;
    d->R = 1.0;
    d->slope = 4.0;
    d->surrogate = BP_SG_SIGMOID;
    d->sg_alpha = 0.3;
    d->sg_width = 1.0;
    d->lambda_v = 0.0;
    d->v_hi = 0.4;
    d->v_lo = -2.0;
    d->ckpt_every = 100;
    d->w_rec_kind = BP_W_F32;
    return BP_OK;
}

size_t bp_snn_workspace_bytes(const bp_snn_desc* d) {
    if (!d || d->B <= 0 || d->T <= 0 || d->n_rec <= 0 || d->n_out <= 0) return 0;
    return bp::snn_layout(*d).total;
}

bp_status bp_snn_forward(const bp_snn_desc* d, const uint8_t* u, float* m, void* workspace, bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_snn_forward");
    BP_TRY(bp::snn_check(d));
    BP_REQUIRE(u && m && workspace, "u, m or workspace is NULL");
    BP_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "workspace must be 256-byte aligned");
    bp::SnnK p = bp::snn_kernel_args(*d, workspace);
    // racc (8 B), I, V, spike list (4 B each) per neuron, plus the input list,
    // plus the readout weights when they fit
    size_t smem = static_cast<size_t>(d->n_rec) * (8 + 4 * 3) + static_cast<size_t>(d->n_in) * 4;
    const size_t wout_bytes = static_cast<size_t>(d->n_rec) * d->n_out * 4;
    p.stage_wout = smem + wout_bytes <= static_cast<size_t>(bp::max_smem_optin()) ? 1 : 0;
    if (p.stage_wout) smem += wout_bytes;
    // recurrent weights in fixed point, once per call (the backward's
    // recomputation reads them from the same workspace)
    if (d->nnz > 0) {
        int64_t grid = (d->nnz + 255) / 256;
        if (grid > bp::sm_count() * 8) grid = bp::sm_count() * 8;
        if (d->w_rec_kind == BP_W_BF16)
            bp::k_snn_fix_weights<BP_W_BF16><<<static_cast<unsigned>(grid), 256, 0, stream>>>(d->w_rec, d->nnz, p.w_fix);
        else
            bp::k_snn_fix_weights<BP_W_F32><<<static_cast<unsigned>(grid), 256, 0, stream>>>(d->w_rec, d->nnz, p.w_fix);
        BP_LAUNCHED();
    }
    if (d->w_rec_kind == BP_W_BF16) {
        BP_TRY(bp::set_smem(bp::k_snn_forward<BP_W_BF16>, smem));
        bp::k_snn_forward<BP_W_BF16><<<d->B, bp::kSnnThreads, smem, stream>>>(p, u, m);
    } else {
        BP_TRY(bp::set_smem(bp::k_snn_forward<BP_W_F32>, smem));
        bp::k_snn_forward<BP_W_F32><<<d->B, bp::kSnnThreads, smem, stream>>>(p, u, m);
    }
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_lif_step_bwd(const bp_snn_desc* d, int64_t n, const float* Vp, const uint8_t* z, const float* Vbar,
                          const float* zbar, const float* Ibar_next, float* Ibar, float* Vbar_prev, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(d != nullptr, "desc is NULL");
    BP_REQUIRE(d->dt > 0 && d->tau_m > 0 && d->tau_s > 0, "time constants must be positive");
    BP_REQUIRE(n >= 0, "n < 0");
    BP_TRY(bp::sg_check(d));
    BP_REQUIRE(n == 0 || (Vp && z && Vbar && zbar && Ibar_next && Ibar && Vbar_prev), "a pointer is NULL");
    if (n == 0) return BP_OK;
    const float a_m = static_cast<float>(std::exp(-d->dt / d->tau_m));
    const float a_s = static_cast<float>(std::exp(-d->dt / d->tau_s));
    int64_t grid = (n + 255) / 256;
    if (grid > bp::sm_count() * 16) grid = bp::sm_count() * 16;
    bp::k_lif_step_bwd<<<static_cast<unsigned>(grid), 256, 0, stream>>>(
        n, a_m, a_s, static_cast<float>(d->R), static_cast<float>(d->V_th), bp::make_sg(*d), Vp, z, Vbar,
        zbar, Ibar_next, Ibar, Vbar_prev);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_snn_loss(int32_t B, int32_t n_out, const float* m, const int64_t* labels, float* loss, float* g_m,
                      bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(B > 0 && n_out > 0, "B and n_out must be positive");
    BP_REQUIRE(m && labels && loss && g_m, "a pointer is NULL");
    bp::k_snn_loss<<<1, 256, 0, stream>>>(B, n_out, m, labels, loss, g_m);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_snn_reg_loss(const bp_snn_desc* d, const void* workspace, float* loss, bp_stream_t stream) {
    bp::clear_error();
    BP_TRY(bp::snn_check(d));
    BP_REQUIRE(workspace && loss, "workspace or loss is NULL");
    BP_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "workspace must be 256-byte aligned");
    if (d->lambda_v == 0) return BP_OK;
    const bp::SnnLayout L = bp::snn_layout(*d);
    const float* vreg = reinterpret_cast<const float*>(static_cast<const char*>(workspace) + L.vreg);
    bp::k_snn_reg_add<<<1, 32, 0, stream>>>(d->B, static_cast<float>(d->lambda_v / d->B), vreg, loss);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_snn_backward(const bp_snn_desc* d, const uint8_t* u, const float* g_m, void* workspace, float* dW_in,
                          float* dw_rec, float* dW_out, float* db_out, bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_snn_backward");
    BP_TRY(bp::snn_check(d));
    BP_REQUIRE(u && g_m && workspace && dW_in && dw_rec && dW_out && db_out, "a pointer is NULL");
    BP_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "workspace must be 256-byte aligned");
    const bp::SnnK p = bp::snn_kernel_args(*d, workspace);
    // racc (8 B), I, V, Ibar_{t+1}, Ibar_t, Vbar, spike list (4 B each) per neuron, plus the input list
    const size_t smem = static_cast<size_t>(d->n_rec) * (8 + 4 * 6) + static_cast<size_t>(d->n_in) * 4;
    if (d->w_rec_kind == BP_W_BF16) {
        BP_TRY(bp::set_smem(bp::k_snn_backward<BP_W_BF16>, smem));
        bp::k_snn_backward<BP_W_BF16><<<d->B, bp::kSnnThreads, smem, stream>>>(p, u, g_m);
    } else {
        BP_TRY(bp::set_smem(bp::k_snn_backward<BP_W_F32>, smem));
        bp::k_snn_backward<BP_W_F32><<<d->B, bp::kSnnThreads, smem, stream>>>(p, u, g_m);
    }
    BP_LAUNCHED();
    // input and recurrent weight gradients: one contraction over batch and
    // time on the tensor cores, G = [u_t ; z_{t-1}]^T Ibar_t
    const bp::SnnLayout L = bp::snn_layout(*d);
    char* wsb = static_cast<char*>(workspace);
    float* g_full = reinterpret_cast<float*>(wsb + L.g_full);
    const uintptr_t tw = (reinterpret_cast<uintptr_t>(wsb + L.tc_work) + 1023) & ~uintptr_t(1023);
    BP_TRY(bp::launch_tc_spike_gemm(d->B, d->T, p.ib_all, d->n_rec, u, d->n_in, p.z_all, d->n_rec, L.zw, g_full,
                                    d->n_rec, false, reinterpret_cast<void*>(tw), L.tc_bytes, stream));
    const int grid = bp::sm_count() * 8;
    bp::k_snn_grad_scatter<<<grid, 256, 0, stream>>>(g_full, d->n_in, d->n_rec, d->indptr, d->indices, dW_in, dw_rec);
    bp::k_snn_reduce<<<grid, 256, 0, stream>>>(p.g_out, d->B, static_cast<int64_t>(d->n_rec) * d->n_out, dW_out);
    bp::k_snn_reduce<<<1, 64, 0, stream>>>(p.g_b, d->B, d->n_out, db_out);
    BP_LAUNCHED();
    return BP_OK;
}

}  // extern "C"
