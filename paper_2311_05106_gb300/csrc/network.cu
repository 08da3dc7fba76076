// network.cu -- the COBA E/I network step and the T-step simulation loop
// (a7), plus the FP64 population statistics (a8).
//
// A step is one launch (lif.cu, k_step): the neuron pass, the CTA-local
// compaction of the step's spikes and their delivery through the stored CSR
// or the JIT rows into the merged E and I event accumulators (AlignPost,
// Section 4.3).  The accumulators are double-buffered: step t reads and
// clears half t mod 2 and delivers into the other half, which step t + 1
// reads (zero delay, Appendix N Listing S6), so delivery can run in the same
// kernel as the neuron pass.  A delayed projection (delay d > 0, Appendix D)
// takes its spikes from a ring of per-step spike lists instead (the kernel
// indexes it from the device step counter), so the accumulators keep their
// two halves whatever the delay.  The optional spike-list counter alternates
// between two slots the same way.  bp_simulate replays CUDA graphs of
// captured steps: a 64-step chunk, and one graph per shorter remainder
// length, each captured once per starting parity (so a short call runs the
// same launch path as a long one, and a call launches graphs only); per-step
// indices that differ between replays (the record row) are read from a small
// device control block.
#include <cmath>
#include <map>
#include <new>

#include "bp_common.cuh"
#include "bp_internal.h"

struct bp_net {
    bp_net_desc d;
    bp::NetStepLaunch L;
    int64_t host_step;
    bp::NetCtrl* ctrl;  // device
    cudaStream_t cap_stream;
    // captured graphs of `len` steps (the chunk, and the shorter remainders
    // of bp_simulate calls) from a step of either parity, keyed 2 len +
    // parity, built on first use
    std::map<int64_t, cudaGraphExec_t>* graphs;
    int chunk;
};

namespace bp {
namespace {

constexpr int kChunk = 64;  // steps per captured graph (even: a chunk keeps the parity of the step count)

__global__ void k_set_record(NetCtrl* ctrl, int32_t* record, int64_t len) {
    ctrl->record = record;
    ctrl->record_base = ctrl->step;
    ctrl->record_len = len;
}

__global__ void k_set_step(NetCtrl* ctrl, int64_t step) { ctrl->step = step; }

// The nonzero 32-bit words of x[0, n) as (index, word) pairs: a warp ballot
// per 32 words and one counter atomic per warp; the pairs of a warp are in
// index order, the warps in arrival order.  *count must start at 0.
__global__ void k_compact_words(const uint32_t* __restrict__ x, int64_t n, int32_t* __restrict__ idx,
                                uint32_t* __restrict__ val, int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    // every lane of a warp runs the same number of iterations (the ballot)
    const int64_t base0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31);
    for (int64_t b = base0; b < n; b += stride) {
        const int64_t i = b + lane;
        const uint32_t w = i < n ? x[i] : 0u;
        const unsigned m = __ballot_sync(FULL_MASK, w != 0u);
        if (m == 0u) continue;
        int pos = 0;
        if (lane == 0) pos = atomicAdd(count, __popc(m));
        pos = __shfl_sync(FULL_MASK, pos, 0) + __popc(m & lanemask_lt());
        if (w != 0u) {
            idx[pos] = static_cast<int32_t>(i);
            val[pos] = w;
        }
    }
}

// x[idx[k]] = val[k] for k < count (indices outside [0, n) are skipped).
__global__ void k_scatter_words(const int32_t* __restrict__ idx, const uint32_t* __restrict__ val, int64_t count,
                                uint32_t* __restrict__ x, int64_t n) {
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < count;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t i = idx[k];
        if (i >= 0 && i < n) x[i] = val[k];
    }
}

__global__ void k_reset_ctrl(NetCtrl* ctrl) {
    ctrl->step = 0;
    ctrl->record = nullptr;
    ctrl->record_base = 0;
    ctrl->record_len = 0;
    ctrl->done_ctas = 0;
}

// FP64 rates from the exact integer totals.
__global__ void k_stats(const int64_t* totals, int64_t n, int64_t n_e, double dt_ms, double* out) {
    const double steps = static_cast<double>(totals[3]);
    const double secs = steps * dt_ms * 1e-3;
    const double se = static_cast<double>(totals[0]), si = static_cast<double>(totals[1]);
    out[0] = (n > 0 && secs > 0) ? (se + si) / (static_cast<double>(n) * secs) : 0.0;
    out[1] = (n_e > 0 && secs > 0) ? se / (static_cast<double>(n_e) * secs) : 0.0;
    out[2] = (n - n_e > 0 && secs > 0) ? si / (static_cast<double>(n - n_e) * secs) : 0.0;
    out[3] = steps > 0 ? static_cast<double>(totals[2]) / steps : 0.0;
}

// One step; advance > 0: its last CTA also advances the device step counter
// by `advance` (the steps this launch closes).
bp_status enqueue_step(bp_net* net, int parity, int32_t t_local, cudaStream_t s, int32_t advance) {
    return launch_network_step(net->L, parity, t_local, s, advance);
}

// Graph of `len` steps starting on a step of the given parity (accumulator
// half and counter slot `parity` read first); the last step advances the
// device step counter by len.  Captured once per (length, parity) and cached.
bp_status get_graph(bp_net* net, int len, int parity, cudaGraphExec_t* out) {
    const int64_t key = 2 * static_cast<int64_t>(len) + (parity & 1);
    auto it = net->graphs->find(key);
    if (it != net->graphs->end()) {
        *out = it->second;
        return BP_OK;
    }
    if (!net->cap_stream) BP_CUDA(cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking));
    BP_CUDA(cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal));
    bp_status st = BP_OK;
    for (int t = 0; t < len && st == BP_OK; ++t)
        st = enqueue_step(net, (parity + t) & 1, t, net->cap_stream, t == len - 1 ? len : 0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(net->cap_stream, &g);
    if (st != BP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return BP_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        return BP_ERR_CUDA;
    }
    net->graphs->emplace(key, ex);
    *out = ex;
    return BP_OK;
}

}  // namespace
}  // namespace bp

extern "C" {

bp_status bp_network_create(const bp_net_desc* desc, bp_net** out) {
    bp::clear_error();
    BP_REQUIRE(desc && out, "desc or out is NULL");
    const bp_net_desc& d = *desc;
    BP_REQUIRE(d.n > 0 && d.n <= INT32_MAX, "n = %lld out of range", (long long)d.n);
    BP_REQUIRE(d.n_e >= 0 && d.n_e <= d.n, "n_e not in [0, n]");
    BP_TRY(bp::check_coba(&d.coba));
    BP_REQUIRE(d.V && d.ge && d.gi && d.ref && d.ye && d.yi && d.totals, "a required state pointer is NULL");
    BP_REQUIRE(!d.spike_list || d.n_spikes, "spike_list needs n_spikes");
    BP_REQUIRE(d.conn_kind == BP_CONN_CSR || d.conn_kind == BP_CONN_JIT, "unknown connectivity kind %d",
               d.conn_kind);
    BP_REQUIRE(d.delay_e >= 0 && d.delay_e <= 65535 && d.delay_i >= 0 && d.delay_i <= 65535,
               "delays must be in [0, 65535] steps (got %d, %d)", d.delay_e, d.delay_i);
    BP_REQUIRE((d.delay_e == 0 && d.delay_i == 0) || d.delay_buf, "a delayed projection needs delay_buf");
    BP_REQUIRE(d.align == BP_ALIGN_POST || d.align == BP_ALIGN_PRE, "unknown align %d", d.align);
    BP_REQUIRE(d.align == BP_ALIGN_POST || (d.trace && d.spk && d.delay_e == 0 && d.delay_i == 0),
               "the AlignPre form needs trace and spk and no delay");
    bp::NetStepLaunch L{};
    L.c = bp::make_lif_const(d.coba);
    L.n = d.n;
    L.n_e = d.n_e;
    L.V = d.V;
    L.ge = d.ge;
    L.gi = d.gi;
    L.ref = d.ref;
    L.ye2 = d.ye;
    L.yi2 = d.yi;
    L.spk = d.spk;
    L.spike_list = d.spike_list;
    L.n_spikes = d.n_spikes;
    L.totals = d.totals;
    L.counts = true;
    if (d.delay_e > 0 || d.delay_i > 0) {
        L.ring = d.delay_buf;
        L.ring_slots = (d.delay_e > d.delay_i ? d.delay_e : d.delay_i) + 2;
        L.delay_e = d.delay_e;
        L.delay_i = d.delay_i;
    }
    if (d.conn_kind == BP_CONN_CSR) {
        BP_REQUIRE(d.indptr && d.indices, "CSR indptr or indices is NULL");
        BP_REQUIRE(d.wkind >= BP_W_HOMO && d.wkind <= BP_W_BF16, "unknown weight kind");
        L.counts = (d.wkind == BP_W_HOMO) || d.data == nullptr;
        L.jit = false;
        L.csr.n_pre = d.n;
        L.csr.n_post = d.n;
        L.csr.indptr = d.indptr;
        L.csr.indices = d.indices;
        L.csr.data = L.counts ? nullptr : d.data;
        L.csr.wkind = L.counts ? BP_W_HOMO : d.wkind;
        L.csr.w_homo = 1.0f;
        // lanes per delivered row from the mean row length (one synchronous
        // 8-byte read at set-up)
        int64_t nnz = 0;
        BP_CUDA(cudaMemcpy(&nnz, d.indptr + d.n, sizeof(int64_t), cudaMemcpyDeviceToHost));
        const int64_t mean = nnz / d.n;
        L.group = mean >= 48 ? 32 : mean >= 24 ? 16 : mean >= 12 ? 8 : 4;
    } else {
        bp_jit_desc de, di;
        BP_TRY(bp_jit_desc_init(&de, bp_projection_seed(d.seed, 0), d.p, BP_JIT_HOMO, 1.0f, 0.0f));
        BP_TRY(bp_jit_desc_init(&di, bp_projection_seed(d.seed, 1), d.p, BP_JIT_HOMO, 1.0f, 0.0f));
        L.jit = true;
        L.je = {de.seed, static_cast<uint32_t>(de.K), BP_JIT_HOMO, 1.0f, 0.0f};
        L.ji = {di.seed, static_cast<uint32_t>(di.K), BP_JIT_HOMO, 1.0f, 0.0f};
    }
    if (d.align == BP_ALIGN_PRE) {
        // the accumulators hold float sums s w (the CSR operand keeps its
        // weight kind: stored weights, or w_e / w_i for homogeneous rows)
        L.trace = d.trace;
        L.counts = false;
    }
    bp_net* net = new (std::nothrow) bp_net();
    if (!net) {
        bp::set_error("host allocation failed");
        return BP_ERR_OOM;
    }
    net->d = d;
    net->L = L;
    net->host_step = 0;
    net->chunk = bp::kChunk;
    net->graphs = new (std::nothrow) std::map<int64_t, cudaGraphExec_t>();
    net->cap_stream = nullptr;
    if (!net->graphs) {
        delete net;
        bp::set_error("host allocation failed");
        return BP_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(&net->ctrl, sizeof(bp::NetCtrl));
    if (e != cudaSuccess) {
        delete net->graphs;
        delete net;
        bp::set_error("cudaMalloc of the control block failed: %s", cudaGetErrorString(e));
        return BP_ERR_OOM;
    }
    net->L.ctrl = net->ctrl;
    e = cudaMemset(net->ctrl, 0, sizeof(bp::NetCtrl));
    if (e != cudaSuccess) {
        cudaFree(net->ctrl);
        delete net->graphs;
        delete net;
        bp::set_error("cudaMemset failed: %s", cudaGetErrorString(e));
        return BP_ERR_CUDA;
    }
    *out = net;
    return BP_OK;
}

bp_status bp_network_reset_counters(bp_net* net, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(net, "net is NULL");
    const bp_net_desc& d = net->d;
    if (d.n_spikes) BP_CUDA(cudaMemsetAsync(d.n_spikes, 0, 2 * sizeof(int32_t), stream));
    BP_CUDA(cudaMemsetAsync(d.totals, 0, 4 * sizeof(int64_t), stream));
    BP_CUDA(cudaMemsetAsync(d.ye, 0, static_cast<size_t>(d.n) * 8, stream));
    BP_CUDA(cudaMemsetAsync(d.yi, 0, static_cast<size_t>(d.n) * 8, stream));
    if (net->L.ring) BP_CUDA(cudaMemsetAsync(net->L.ring, 0, static_cast<size_t>(net->L.ring_slots) * 4, stream));
    bp::k_reset_ctrl<<<1, 1, 0, stream>>>(net->ctrl);
    BP_LAUNCHED();
    net->host_step = 0;
    return BP_OK;
}

int64_t bp_network_step_count(const bp_net* net) { return net ? net->host_step : -1; }

bp_status bp_network_set_step_count(bp_net* net, int64_t step, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(net, "net is NULL");
    BP_REQUIRE(step >= 0, "step < 0");
    bp::k_set_step<<<1, 1, 0, stream>>>(net->ctrl, step);
    BP_LAUNCHED();
    net->host_step = step;
    return BP_OK;
}

bp_status bp_network_step(bp_net* net, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(net, "net is NULL");
    BP_TRY(bp::enqueue_step(net, static_cast<int>(net->host_step & 1), 0, stream, 1));
    net->host_step += 1;
    return BP_OK;
}

bp_status bp_simulate_prepare(bp_net* net, int64_t T, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(net, "net is NULL");
    BP_REQUIRE(T >= 0, "T < 0");
    // the graphs bp_simulate(T) would launch from a step of either parity
    // (the step count may change before the call, e.g. by a restore)
    const int64_t lens[2] = {T >= net->chunk ? net->chunk : 0, T % net->chunk};
    for (int parity = 0; parity < 2; ++parity) {
        for (int64_t len : lens) {
            if (len <= 0) continue;
            cudaGraphExec_t g = nullptr;
            BP_TRY(bp::get_graph(net, static_cast<int>(len), parity, &g));
            BP_CUDA(cudaGraphUpload(g, stream));
        }
    }
    return BP_OK;
}

bp_status bp_simulate(bp_net* net, int64_t T, int32_t* record, bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_simulate");
    BP_REQUIRE(net, "net is NULL");
    BP_REQUIRE(T >= 0, "T < 0");
    if (T == 0) return BP_OK;
    // the record is attached only for this call (every call leaves it detached)
    if (record) {
        BP_CUDA(cudaMemsetAsync(record, 0, static_cast<size_t>(T) * 2 * sizeof(int32_t), stream));
        bp::k_set_record<<<1, 1, 0, stream>>>(net->ctrl, record, T);
        BP_LAUNCHED();
    }
    int64_t done = 0;
    // every graph starts at the current parity (a chunk is even, so it
    // leaves the parity unchanged)
    const int parity = static_cast<int>(net->host_step & 1);
    const int64_t chunks = T / net->chunk;
    if (chunks > 0) {
        cudaGraphExec_t g = nullptr;
        BP_TRY(bp::get_graph(net, net->chunk, parity, &g));
        for (int64_t k = 0; k < chunks; ++k) BP_CUDA(cudaGraphLaunch(g, stream));
        net->host_step += chunks * net->chunk;
        done += chunks * net->chunk;
    }
    // the remainder is one cached graph of its length
    const int64_t rem = T - done;
    if (rem > 0) {
        cudaGraphExec_t g = nullptr;
        BP_TRY(bp::get_graph(net, static_cast<int>(rem), parity, &g));
        BP_CUDA(cudaGraphLaunch(g, stream));
        net->host_step += rem;
    }
    // detach the record so that later steps do not write into it
    if (record) {
        bp::k_set_record<<<1, 1, 0, stream>>>(net->ctrl, nullptr, 0);
        BP_LAUNCHED();
    }
    return BP_OK;
}

bp_status bp_words_compact(const void* x, int64_t n, int32_t* idx, uint32_t* val, int32_t* count,
                           bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n >= 0 && n <= INT32_MAX, "n must be in [0, 2^31 - 1]");
    BP_REQUIRE(count != nullptr, "count is NULL");
    BP_REQUIRE(n == 0 || (x && idx && val), "a required pointer is NULL");
    BP_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t), stream));
    if (n == 0) return BP_OK;
    int64_t grid = (n + 255) / 256;
    if (grid > bp::sm_count() * 8) grid = bp::sm_count() * 8;
    bp::k_compact_words<<<static_cast<unsigned>(grid), 256, 0, stream>>>(static_cast<const uint32_t*>(x), n, idx, val,
                                                                        count);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_words_scatter(const int32_t* idx, const uint32_t* val, int64_t count, void* x, int64_t n,
                           bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(count >= 0 && n >= 0, "negative size");
    BP_REQUIRE(count == 0 || (idx && val && x), "a required pointer is NULL");
    if (count == 0) return BP_OK;
    int64_t grid = (count + 255) / 256;
    if (grid > bp::sm_count() * 8) grid = bp::sm_count() * 8;
    bp::k_scatter_words<<<static_cast<unsigned>(grid), 256, 0, stream>>>(idx, val, count, static_cast<uint32_t*>(x), n);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_network_stats(bp_net* net, double* out, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(net && out, "net or out is NULL");
    bp::k_stats<<<1, 1, 0, stream>>>(net->d.totals, net->d.n, net->d.n_e, net->d.coba.dt, out);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_network_destroy(bp_net* net) {
    bp::clear_error();
    if (!net) return BP_OK;
    if (net->graphs) {
        for (auto& kv : *net->graphs) cudaGraphExecDestroy(kv.second);
        delete net->graphs;
    }
    if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
    if (net->ctrl) cudaFree(net->ctrl);
    delete net;
    return BP_OK;
}

}  // extern "C"
