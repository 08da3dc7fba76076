// batch.cu -- many independent COBA E/I networks of uneven sizes advanced
// together by one persistent kernel (a9).
//
// Networks are independent, so a network never spans CTAs: the host packs the
// networks into bins (longest-processing-time first, bounded by the
// shared-memory capacity of a CTA) and CTA b runs every time step of bin b's
// networks on its own, with no inter-CTA synchronisation at all.  Within a
// step the CTA
//   1. updates all neurons of its networks (the same per-neuron arithmetic as
//      the single-network path, 16-byte state loads from global memory),
//      reading and clearing the event counts from shared memory, and appends
//      spikes to its spike list;
//   2. after a CTA barrier, delivers those spikes' rows -- regenerated JIT rows
//      (Appendix C) walked by groups of 16 or 32 lanes, or stored CSR rows
//      walked by groups of 4 to 32 lanes -- adding the events into the
//      shared-memory counts, E and I packed into one 32-bit word (E in the low
//      16 bits; a presynaptic neuron delivers at most one event per target and
//      step, so each half stays below the population size, < 2^16 by
//      construction);
//   3. after another barrier, adds the step's per-network totals.
// The counts survive between launches in a global spill buffer.  The time
// loop is split into launches of a few steps that bp_batch_simulate captures
// once in a CUDA graph.  bp_batch_autotune times, from a snapshot of the
// state, every feasible combination of CTA size, lanes per delivered row and
// bins per SM (packings of 1, 2 or 4 CTAs per SM with proportionally smaller
// shared-memory capacity) and keeps the fastest; every combination computes
// the same trajectories bit for bit (integer counts, same per-neuron order).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "bp_common.cuh"
#include "bp_internal.h"
#include "bp_neuron.cuh"
#include "bp_rows.cuh"

namespace bp {
namespace {

constexpr int kBatchMaxNetsPerBin = 64;
constexpr int kBatchStepsPerLaunch = 100;
constexpr int32_t kBatchCapacity = 56320;  // packed counts per CTA (220 KiB) at one CTA per SM

// Packed-count capacity of a CTA when `per_sm` CTAs share an SM's shared memory.
int32_t bin_capacity(int per_sm) {
    switch (per_sm) {
        case 1: return kBatchCapacity;
        case 2: return 27648;   // 108 KiB
        default: return 13312;  // 52 KiB
    }
}

struct NetInfo {
    int64_t off;       // first neuron in the concatenated state
    int32_t n, n_e;
    uint64_t seed_e, seed_i;
    uint32_t K;
    int32_t pad;
};

struct BinArgs {
    LifConst c;
    const NetInfo* nets;
    const int32_t* bin_nets;   // net ids, grouped by bin
    const int32_t* bin_ptr;    // [bins + 1]
    const int64_t* bin_spk;    // spike-list offset of each bin
    float* V;
    float* ge;
    float* gi;
    uint8_t* ref;
    int32_t* spill;            // packed counts between launches, concatenated layout
    int32_t* spk_list;
    int64_t* totals;           // [n_nets][4]
    const int64_t* indptr;     // stored form: CSR over the padded layout (row off + i: neuron i)
    const int32_t* indices;    // targets local to the row's network
    int32_t steps;
};

// CSR: stored rows, G lanes per row; otherwise JIT rows, G (16 or 32) lanes
// per row.  At most 64 registers per thread, so that 1024 threads of CTAs can
// share an SM whatever the CTA size.
template <int THREADS, bool CSR, int G>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_batch(BinArgs a) {
    extern __shared__ __align__(16) int32_t acc[];
    __shared__ int32_t s_base[kBatchMaxNetsPerBin + 1];
    __shared__ int32_t s_cnt[kBatchMaxNetsPerBin][3];
    __shared__ int32_t s_nspk;
    constexpr int kWarps = THREADS / 32;
    const int bin = blockIdx.x;
    const int nb0 = a.bin_ptr[bin];
    const int nn = a.bin_ptr[bin + 1] - nb0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < nn; ++k) {
            s_base[k] = run;
            run += (a.nets[a.bin_nets[nb0 + k]].n + 3) & ~3;
        }
        s_base[nn] = run;
    }
    __syncthreads();
    // restore the pending counts
    for (int k = 0; k < nn; ++k) {
        const NetInfo& net = a.nets[a.bin_nets[nb0 + k]];
        const int np = (net.n + 3) & ~3;
        for (int t = threadIdx.x; t < np; t += THREADS) acc[s_base[k] + t] = a.spill[net.off + t];
    }
    int32_t* list = a.spk_list + a.bin_spk[bin];

    for (int step = 0; step < a.steps; ++step) {
        if (threadIdx.x < nn) {
            s_cnt[threadIdx.x][0] = 0;
            s_cnt[threadIdx.x][1] = 0;
            s_cnt[threadIdx.x][2] = 0;
        }
        if (threadIdx.x == 0) s_nspk = 0;
        __syncthreads();
        // ---- 1. neuron pass
        for (int k = 0; k < nn; ++k) {
            const NetInfo& net = a.nets[a.bin_nets[nb0 + k]];
            const int nq = (net.n + 3) >> 2;
            int32_t* cnt = acc + s_base[k];
            // warp-uniform trip count: every lane runs every iteration
            for (int qb = 0; qb < nq; qb += THREADS) {
                const int q = qb + threadIdx.x;
                uint32_t bits = 0;
                if (q < nq) {
                    const int64_t g = net.off + 4 * static_cast<int64_t>(q);
                    // evict-last: the whole batch state (about 100 MB at the
                    // configured size) is re-read every step and mostly fits
                    // in L2 (measured 4-6 % faster per step than default loads)
                    const uint64_t pol = l2_keep_policy();
                    float4 v = ld_keep(reinterpret_cast<const float4*>(a.V + g), pol);
                    float4 ge = ld_keep(reinterpret_cast<const float4*>(a.ge + g), pol);
                    float4 gi = ld_keep(reinterpret_cast<const float4*>(a.gi + g), pol);
                    // four one-byte refractory counters in one word
                    const uint32_t r4 = ld_keep(reinterpret_cast<const uint32_t*>(a.ref + g), pol);
                    int4 r = make_int4(r4 & 0xFFu, (r4 >> 8) & 0xFFu, (r4 >> 16) & 0xFFu, r4 >> 24);
                    int4 y = *reinterpret_cast<int4*>(cnt + 4 * q);
                    *reinterpret_cast<int4*>(cnt + 4 * q) = make_int4(0, 0, 0, 0);
                    float* vv = &v.x;
                    float* gg = &ge.x;
                    float* hh = &gi.x;
                    int* rr = &r.x;
                    const int* yy = &y.x;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (4 * q + e < net.n) {  // padding neurons are not simulated
                            const int32_t ce = yy[e] & 0xFFFF;
                            const int32_t ci = static_cast<int32_t>(static_cast<uint32_t>(yy[e]) >> 16);
                            if (neuron_update(a.c, vv[e], gg[e], hh[e], rr[e], event_add<true>(ce, a.c.w_e),
                                              event_add<true>(ci, a.c.w_i), 0.f))
                                bits |= 1u << e;
                        }
                    }
                    st_keep(reinterpret_cast<float4*>(a.V + g), v, pol);
                    st_keep(reinterpret_cast<float4*>(a.ge + g), ge, pol);
                    st_keep(reinterpret_cast<float4*>(a.gi + g), gi, pol);
                    st_keep(reinterpret_cast<uint32_t*>(a.ref + g),
                            static_cast<uint32_t>(r.x) | (static_cast<uint32_t>(r.y) << 8) |
                                (static_cast<uint32_t>(r.z) << 16) | (static_cast<uint32_t>(r.w) << 24),
                            pol);
                }
                // warp-aggregated append of (net slot << 20 | neuron) entries
                const int mine = __popc(bits);
                int incl = mine;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int o = __shfl_up_sync(FULL_MASK, incl, d);
                    if (lane >= d) incl += o;
                }
                const int wtot = __shfl_sync(FULL_MASK, incl, 31);
                int base = 0;
                if (lane == 0 && wtot) base = atomicAdd(&s_nspk, wtot);
                base = __shfl_sync(FULL_MASK, base, 0);
                int pos = base + incl - mine;
                int ne = 0, ni = 0;
                for (uint32_t m = bits; m; m &= m - 1) {
                    const int i = 4 * q + (__ffs(m) - 1);
                    list[pos++] = (k << 20) | i;
                    if (i < net.n_e) ++ne; else ++ni;
                }
                if (ne) atomicAdd(&s_cnt[k][0], ne);
                if (ni) atomicAdd(&s_cnt[k][1], ni);
            }
        }
        __syncthreads();
        // ---- 2. delivery of this step's spikes
        const int nspk = s_nspk;
        if constexpr (CSR) {
            // stored rows (Appendix B), G lanes per row, four index loads in
            // flight per lane before its shared-memory atomics
            constexpr int kGroups = THREADS / G;
            const int gl = threadIdx.x % G;
            for (int e = threadIdx.x / G; e < nspk; e += kGroups) {
                const int32_t ent = list[e];
                const int k = ent >> 20;
                const int i = ent & 0xFFFFF;
                const NetInfo& net = a.nets[a.bin_nets[nb0 + k]];
                const int64_t row = net.off + i;
                const int64_t b0 = a.indptr[row], b1 = a.indptr[row + 1];
                int32_t* cnt = acc + s_base[k];
                const int32_t inc = i < net.n_e ? 1 : 65536;
                const uint32_t n_post = static_cast<uint32_t>(net.n);
                for (int64_t j = b0 + gl; j < b1; j += 4 * G) {
                    int32_t q[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) q[u] = j + u * G < b1 ? ld_stream(a.indices + j + u * G) : -1;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (static_cast<uint32_t>(q[u]) < n_post) atomicAdd(cnt + q[u], inc);
                }
                if (gl == 0 && b1 > b0) atomicAdd(&s_cnt[k][2], static_cast<int32_t>(b1 - b0));
            }
        } else {
            // JIT rows (Appendix C), regenerated by groups of G lanes
            constexpr int kPerWarp = 32 / G;
            constexpr int kGroups = kWarps * kPerWarp;
            const unsigned gmask = G == 32 ? FULL_MASK : (0xFFFFu << (threadIdx.x & 16u));
            for (int e = warp * kPerWarp + lane / G; e < nspk; e += kGroups) {
                const int32_t ent = list[e];
                const int k = ent >> 20;
                const int i = ent & 0xFFFFF;
                const NetInfo& net = a.nets[a.bin_nets[nb0 + k]];
                const bool exc = i < net.n_e;
                JitArgs d;
                d.seed = exc ? net.seed_e : net.seed_i;
                d.K = net.K;
                d.wkind = BP_JIT_HOMO;
                d.w0 = 1.0f;
                d.w1 = 0.0f;
                int32_t* cnt = acc + s_base[k];
                const int32_t inc = exc ? 1 : 65536;
                int64_t ev = jit_walk_g<BP_JIT_HOMO, G>(d, static_cast<uint32_t>(exc ? i : i - net.n_e), net.n,
                                                        [&](int64_t q, uint64_t, float) { atomicAdd(cnt + q, inc); });
#pragma unroll
                for (int dd = G / 2; dd > 0; dd >>= 1) ev += __shfl_xor_sync(gmask, ev, dd, G);
                if ((lane & (G - 1)) == 0 && ev) atomicAdd(&s_cnt[k][2], static_cast<int32_t>(ev));
            }
        }
        __syncthreads();
        // ---- 3. per-network totals
        if (threadIdx.x < nn) {
            int64_t* tot = a.totals + 4 * static_cast<int64_t>(a.bin_nets[nb0 + threadIdx.x]);
            atomicAdd(reinterpret_cast<unsigned long long*>(tot + 0), static_cast<unsigned long long>(s_cnt[threadIdx.x][0]));
            atomicAdd(reinterpret_cast<unsigned long long*>(tot + 1), static_cast<unsigned long long>(s_cnt[threadIdx.x][1]));
            atomicAdd(reinterpret_cast<unsigned long long*>(tot + 2), static_cast<unsigned long long>(s_cnt[threadIdx.x][2]));
            atomicAdd(reinterpret_cast<unsigned long long*>(tot + 3), 1ull);
        }
    }
    __syncthreads();
    // keep the pending counts for the next launch
    for (int k = 0; k < nn; ++k) {
        const NetInfo& net = a.nets[a.bin_nets[nb0 + k]];
        const int np = (net.n + 3) & ~3;
        for (int t = threadIdx.x; t < np; t += THREADS) a.spill[net.off + t] = acc[s_base[k] + t];
    }
}

// Validation of a batched stored CSR: for every padded row, its extent lies
// within [0, nnz] and is ascending, a padding row is empty, and a network's
// row holds strictly increasing targets in [0, n) (no repeated column, which
// the packed 16-bit counts need).  out[0] += the number of bad rows.
__global__ void k_batch_csr_check(const NetInfo* __restrict__ nets, int32_t n_nets, int64_t total, int64_t nnz,
                                  const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                  unsigned long long* __restrict__ out) {
    unsigned long long bad = 0;
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < total;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        // the network whose padded range holds row r: the last with off <= r
        int lo = 0, hi = n_nets;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (nets[mid].off <= r) lo = mid; else hi = mid;
        }
        const NetInfo& net = nets[lo];
        const int64_t b0 = indptr[r], b1 = indptr[r + 1];
        if (b0 < 0 || b1 < b0 || b1 > nnz) {
            ++bad;
            continue;
        }
        if (r - net.off >= net.n) {
            if (b1 > b0) ++bad;
            continue;
        }
        int32_t prev = -1;
        bool ok = true;
        for (int64_t j = b0; j < b1; ++j) {
            const int32_t q = indices[j];
            if (q <= prev || q >= net.n) ok = false;
            prev = q;
        }
        if (!ok) ++bad;
    }
    if (bad) atomicAdd(out, bad);
}

template <int THREADS, bool CSR, int G>
bp_status launch_batch_k(const BinArgs& a, int bins, size_t smem, cudaStream_t s) {
    BP_TRY(ensure_smem_attr(reinterpret_cast<const void*>(k_batch<THREADS, CSR, G>), kBatchCapacity * 4));
    k_batch<THREADS, CSR, G><<<bins, THREADS, smem, s>>>(a);
    BP_LAUNCHED();
    return BP_OK;
}

template <int THREADS>
bp_status launch_batch_t(const BinArgs& a, bool csr, int group, int bins, size_t smem, cudaStream_t s) {
    if (!csr) {
        if (group == 16) return launch_batch_k<THREADS, false, 16>(a, bins, smem, s);
        return launch_batch_k<THREADS, false, 32>(a, bins, smem, s);
    }
    switch (group) {
        case 4: return launch_batch_k<THREADS, true, 4>(a, bins, smem, s);
        case 8: return launch_batch_k<THREADS, true, 8>(a, bins, smem, s);
        case 16: return launch_batch_k<THREADS, true, 16>(a, bins, smem, s);
        default: return launch_batch_k<THREADS, true, 32>(a, bins, smem, s);
    }
}

bp_status launch_batch(const BinArgs& a, bool csr, int threads, int group, int bins, size_t smem, cudaStream_t s) {
    switch (threads) {
        case 256: return launch_batch_t<256>(a, csr, group, bins, smem, s);
        case 512: return launch_batch_t<512>(a, csr, group, bins, smem, s);
        default: return launch_batch_t<1024>(a, csr, group, bins, smem, s);
    }
}

// CTAs of k_batch<threads, csr, group> that fit on one SM with `smem` bytes
// of dynamic shared memory each.
int resident_ctas(bool csr, int threads, int group, size_t smem) {
    const void* k = nullptr;
#define BP_BK(TH)                                                                                         \
    k = !csr ? (group == 16 ? reinterpret_cast<const void*>(k_batch<TH, false, 16>)                      \
                            : reinterpret_cast<const void*>(k_batch<TH, false, 32>))                     \
             : group == 4 ? reinterpret_cast<const void*>(k_batch<TH, true, 4>)                          \
             : group == 8 ? reinterpret_cast<const void*>(k_batch<TH, true, 8>)                          \
             : group == 16 ? reinterpret_cast<const void*>(k_batch<TH, true, 16>)                        \
                           : reinterpret_cast<const void*>(k_batch<TH, true, 32>)
    if (threads == 256) { BP_BK(256); } else if (threads == 512) { BP_BK(512); } else { BP_BK(1024); }
#undef BP_BK
    if (ensure_smem_attr(k, kBatchCapacity * 4) != BP_OK) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace
}  // namespace bp

struct bp_batch {
    bp_batch_desc d;
    int32_t n_nets;
    bool csr;                  // stored rows (else JIT rows)
    int bins;
    int threads;
    int group;                 // lanes per delivered row
    int per_sm;                // bins per SM of the current packing
    size_t smem;
    int64_t total;             // padded neurons
    std::vector<int64_t>* sizes;  // neurons per network (host copy, for re-packing)
    bp::BinArgs args;
    bp::NetInfo* d_nets;
    int32_t* d_bin_nets;
    int32_t* d_bin_ptr;
    int64_t* d_bin_spk;
    int32_t* d_spill;
    int32_t* d_list;
    void* d_snapshot;          // autotuner's copy of the state
    cudaStream_t cap_stream;
    std::map<int64_t, cudaGraphExec_t>* graphs;
};

namespace {

void free_bins(bp_batch* b) {
    cudaFree(b->d_bin_nets);
    cudaFree(b->d_bin_ptr);
    cudaFree(b->d_bin_spk);
    b->d_bin_nets = nullptr;
    b->d_bin_ptr = nullptr;
    b->d_bin_spk = nullptr;
}

void free_batch(bp_batch* b) {
    if (!b) return;
    if (b->graphs) {
        for (auto& kv : *b->graphs) cudaGraphExecDestroy(kv.second);
        delete b->graphs;
    }
    delete b->sizes;
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_nets);
    free_bins(b);
    cudaFree(b->d_spill);
    cudaFree(b->d_list);
    cudaFree(b->d_snapshot);
    delete b;
}

void drop_graphs(bp_batch* b) {
    for (auto& kv : *b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs->clear();
}

// Longest-processing-time packing of the networks into bins of `per_sm` per
// SM (more bins when they do not fit: the kernel then runs in waves), and the
// upload of the bin tables.  Fails with BP_ERR_INVALID if a network exceeds
// the per-bin capacity.
bp_status pack(bp_batch* b, int per_sm) {
    const std::vector<int64_t>& n = *b->sizes;
    const int32_t N = b->n_nets;
    const int32_t cap = bp::bin_capacity(per_sm);
    for (int32_t id = 0; id < N; ++id)
        BP_REQUIRE(((n[id] + 3) & ~int64_t(3)) <= cap, "network %d (%lld neurons) exceeds the %d of a bin", id,
                   (long long)n[id], cap);
    int bins = std::min<int>(bp::sm_count() * per_sm, N);
    std::vector<int32_t> order(N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return n[x] > n[y]; });
    std::vector<std::vector<int32_t>> members;
    std::vector<int64_t> load;
    for (;;) {
        members.assign(bins, {});
        load.assign(bins, 0);
        bool ok = true;
        for (int32_t id : order) {
            const int64_t np = (n[id] + 3) & ~int64_t(3);
            int best = -1;
            for (int k = 0; k < bins; ++k) {
                if (load[k] + np > cap || static_cast<int>(members[k].size()) >= bp::kBatchMaxNetsPerBin) continue;
                if (best < 0 || load[k] < load[best]) best = k;
            }
            if (best < 0) {
                ok = false;
                break;
            }
            members[best].push_back(id);
            load[best] += np;
        }
        if (ok) break;
        bins *= 2;
        BP_REQUIRE(bins <= 65535, "cannot pack the networks");
    }
    std::vector<int32_t> bin_nets, bin_ptr(1, 0);
    std::vector<int64_t> bin_spk;
    int64_t spk_off = 0, max_load = 0;
    for (int k = 0; k < bins; ++k) {
        bin_spk.push_back(spk_off);
        spk_off += load[k];
        max_load = std::max(max_load, load[k]);
        for (int32_t id : members[k]) bin_nets.push_back(id);
        bin_ptr.push_back(static_cast<int32_t>(bin_nets.size()));
    }
    free_bins(b);
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&b->d_bin_nets, sizeof(int32_t) * bin_nets.size());
    e = e ? e : cudaMalloc(&b->d_bin_ptr, sizeof(int32_t) * bin_ptr.size());
    e = e ? e : cudaMalloc(&b->d_bin_spk, sizeof(int64_t) * bin_spk.size());
    e = e ? e : cudaMemcpy(b->d_bin_nets, bin_nets.data(), sizeof(int32_t) * bin_nets.size(), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(b->d_bin_ptr, bin_ptr.data(), sizeof(int32_t) * bin_ptr.size(), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(b->d_bin_spk, bin_spk.data(), sizeof(int64_t) * bin_spk.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_bins(b);
        bp::set_error("upload of the bin tables failed: %s", cudaGetErrorString(e));
        return BP_ERR_CUDA;
    }
    b->bins = bins;
    b->per_sm = per_sm;
    b->smem = static_cast<size_t>(std::max<int64_t>(max_load, 4)) * 4;
    b->args.bin_nets = b->d_bin_nets;
    b->args.bin_ptr = b->d_bin_ptr;
    b->args.bin_spk = b->d_bin_spk;
    return BP_OK;
}

bp_status enqueue_steps(bp_batch* b, int64_t T, cudaStream_t s) {
    for (int64_t done = 0; done < T;) {
        const int64_t k = std::min<int64_t>(bp::kBatchStepsPerLaunch, T - done);
        bp::BinArgs a = b->args;
        a.steps = static_cast<int32_t>(k);
        BP_TRY(bp::launch_batch(a, b->csr, b->threads, b->group, b->bins, b->smem, s));
        done += k;
    }
    return BP_OK;
}

}  // namespace

extern "C" {

int64_t bp_batch_layout(int32_t n_nets, const int64_t* n, int64_t* offsets) {
    if (n_nets < 0 || (n_nets > 0 && !n)) return -1;
    int64_t off = 0;
    for (int32_t b = 0; b < n_nets; ++b) {
        if (offsets) offsets[b] = off;
        off += (n[b] + 3) & ~int64_t(3);
    }
    if (offsets) offsets[n_nets] = off;
    return off;
}

bp_status bp_batch_create(const bp_batch_desc* desc, bp_batch** out) {
    bp::clear_error();
    BP_REQUIRE(desc && out, "desc or out is NULL");
    const bp_batch_desc& d = *desc;
    BP_REQUIRE(d.n_nets > 0 && d.n && d.seed, "n_nets, n or seed missing");
    BP_TRY(bp::check_coba(&d.coba));
    BP_REQUIRE(d.V && d.ge && d.gi && d.ref && d.totals, "a required state pointer is NULL");
    BP_REQUIRE(!d.indptr == !d.indices, "indptr and indices must both be given (stored rows) or both be NULL");
    // the kernel moves four neurons per 16-byte (FP32) and 4-byte (counter) access
    const auto al = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
    BP_REQUIRE(al(d.V, 16) && al(d.ge, 16) && al(d.gi, 16) && al(d.ref, 4),
               "V, ge, gi must be 16-byte and ref 4-byte aligned");
    const int32_t N = d.n_nets;
    std::vector<int64_t> off(N + 1);
    const int64_t total = bp_batch_layout(N, d.n, off.data());
    std::vector<bp::NetInfo> nets(N);
    for (int32_t b = 0; b < N; ++b) {
        const int64_t n = d.n[b];
        const int64_t ne = d.n_e ? d.n_e[b] : (4 * n) / 5;
        BP_REQUIRE(n > 0 && n <= bp::kBatchCapacity, "network %d: n = %lld not in [1, %d]", b, (long long)n,
                   bp::kBatchCapacity);
        BP_REQUIRE(ne >= 0 && ne <= n && ne < 65536 && n - ne < 65536, "network %d: bad n_e", b);
        const double p = d.p ? d.p[b] : 80.0 / static_cast<double>(n);
        bp_jit_desc de;
        BP_TRY(bp_jit_desc_init(&de, bp_projection_seed(d.seed[b], 0), p, BP_JIT_HOMO, 1.0f, 0.0f));
        nets[b].off = off[b];
        nets[b].n = static_cast<int32_t>(n);
        nets[b].n_e = static_cast<int32_t>(ne);
        nets[b].seed_e = de.seed;
        nets[b].seed_i = bp_projection_seed(d.seed[b], 1);
        nets[b].K = static_cast<uint32_t>(de.K);
        nets[b].pad = 0;
    }
    bp_batch* b = new (std::nothrow) bp_batch();
    if (!b) {
        bp::set_error("host allocation failed");
        return BP_ERR_OOM;
    }
    b->d = d;
    b->d.n = nullptr;  // host arrays are not kept
    b->d.n_e = nullptr;
    b->d.seed = nullptr;
    b->d.p = nullptr;
    b->n_nets = N;
    b->csr = d.indptr != nullptr;
    b->threads = 1024;
    b->group = b->csr ? 8 : 32;
    b->total = total;
    b->graphs = new (std::nothrow) std::map<int64_t, cudaGraphExec_t>();
    b->sizes = new (std::nothrow) std::vector<int64_t>(d.n, d.n + N);
    // V, ge, gi (4 B), ref (1 B), the spilled counts (4 B) and the totals
    const size_t state_bytes = static_cast<size_t>(total) * (3 * 4 + 1 + 4) + static_cast<size_t>(N) * 32;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&b->d_nets, sizeof(bp::NetInfo) * N);
    e = e ? e : cudaMalloc(&b->d_spill, sizeof(int32_t) * total);
    e = e ? e : cudaMalloc(&b->d_list, sizeof(int32_t) * std::max<int64_t>(total, 1));
    e = e ? e : cudaMalloc(&b->d_snapshot, state_bytes);
    if (e != cudaSuccess || !b->graphs || !b->sizes) {
        free_batch(b);
        bp::set_error("allocation of the batch tables failed: %s", cudaGetErrorString(e));
        return BP_ERR_OOM;
    }
    e = e ? e : cudaMemcpy(b->d_nets, nets.data(), sizeof(bp::NetInfo) * N, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemset(b->d_spill, 0, sizeof(int32_t) * total);
    if (e != cudaSuccess) {
        free_batch(b);
        bp::set_error("upload of the batch tables failed: %s", cudaGetErrorString(e));
        return BP_ERR_CUDA;
    }
    if (b->csr) {
        // the stored rows are validated once here: the packed counts and the
        // shared-memory targets rely on in-range, unrepeated columns
        int64_t nnz = 0;
        unsigned long long* d_bad = nullptr;
        unsigned long long bad = 0;
        e = cudaMemcpy(&nnz, d.indptr + total, sizeof(int64_t), cudaMemcpyDeviceToHost);
        e = e ? e : cudaMalloc(&d_bad, sizeof(unsigned long long));
        e = e ? e : cudaMemset(d_bad, 0, sizeof(unsigned long long));
        if (e == cudaSuccess) {
            const int64_t grid = std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(bp::sm_count()) * 16);
            bp::k_batch_csr_check<<<static_cast<unsigned>(std::max<int64_t>(grid, 1)), 256>>>(
                b->d_nets, N, total, nnz, d.indptr, d.indices, d_bad);
            e = cudaGetLastError();
        }
        e = e ? e : cudaMemcpy(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost);
        cudaFree(d_bad);
        if (e != cudaSuccess) {
            free_batch(b);
            bp::set_error("validation of the stored rows failed: %s", cudaGetErrorString(e));
            return BP_ERR_CUDA;
        }
        if (bad) {
            free_batch(b);
            bp::set_error("%llu stored rows are invalid (extent, padding row with entries, a target outside its "
                          "network, or unsorted / repeated columns)", bad);
            return BP_ERR_INVALID;
        }
    }
    bp::BinArgs& a = b->args;
    a.c = bp::make_lif_const(d.coba);
    a.nets = b->d_nets;
    a.V = d.V;
    a.ge = d.ge;
    a.gi = d.gi;
    a.ref = d.ref;
    a.spill = b->d_spill;
    a.spk_list = b->d_list;
    a.totals = d.totals;
    a.indptr = d.indptr;
    a.indices = d.indices;
    a.steps = 0;
    const bp_status st = pack(b, 1);
    if (st != BP_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return BP_OK;
}

bp_status bp_batch_info(const bp_batch* b, int32_t* bins, int32_t* threads, int64_t* padded_neurons) {
    bp::clear_error();
    BP_REQUIRE(b, "batch is NULL");
    if (bins) *bins = b->bins;
    if (threads) *threads = b->threads;
    if (padded_neurons) *padded_neurons = b->total;
    return BP_OK;
}

bp_status bp_batch_tuning(const bp_batch* b, int32_t* threads, int32_t* lanes_per_row, int32_t* ctas_per_sm,
                          int32_t* stored_rows) {
    bp::clear_error();
    BP_REQUIRE(b, "batch is NULL");
    if (threads) *threads = b->threads;
    if (lanes_per_row) *lanes_per_row = b->group;
    if (ctas_per_sm) *ctas_per_sm = b->per_sm;
    if (stored_rows) *stored_rows = b->csr ? 1 : 0;
    return BP_OK;
}

bp_status bp_batch_set_tuning(bp_batch* b, int32_t threads, int32_t lanes_per_row, int32_t ctas_per_sm) {
    bp::clear_error();
    BP_REQUIRE(b, "batch is NULL");
    BP_REQUIRE(threads == 256 || threads == 512 || threads == 1024, "threads must be 256, 512 or 1024");
    BP_REQUIRE(b->csr ? (lanes_per_row == 4 || lanes_per_row == 8 || lanes_per_row == 16 || lanes_per_row == 32)
                      : (lanes_per_row == 16 || lanes_per_row == 32),
               "lanes_per_row %d not available for this connectivity", lanes_per_row);
    BP_REQUIRE(ctas_per_sm == 1 || ctas_per_sm == 2 || ctas_per_sm == 4, "ctas_per_sm must be 1, 2 or 4");
    if (ctas_per_sm != b->per_sm) BP_TRY(pack(b, ctas_per_sm));
    b->threads = threads;
    b->group = lanes_per_row;
    drop_graphs(b);
    return BP_OK;
}

bp_status bp_batch_reset_counters(bp_batch* b, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(b, "batch is NULL");
    BP_CUDA(cudaMemsetAsync(b->d_spill, 0, sizeof(int32_t) * b->total, stream));
    BP_CUDA(cudaMemsetAsync(b->d.totals, 0, sizeof(int64_t) * 4 * b->n_nets, stream));
    return BP_OK;
}

namespace {
// The cached graph of T steps (captured on first use).
bp_status batch_graph(bp_batch* b, int64_t T, cudaGraphExec_t* out) {
    auto it = b->graphs->find(T);
    if (it == b->graphs->end()) {
        if (!b->cap_stream) BP_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        BP_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        bp_status st = enqueue_steps(b, T, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != BP_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) {
            bp::set_error("graph capture failed: %s", cudaGetErrorString(e));
            return BP_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            bp::set_error("graph instantiation failed: %s", cudaGetErrorString(e));
            return BP_ERR_CUDA;
        }
        it = b->graphs->emplace(T, ex).first;
    }
    *out = it->second;
    return BP_OK;
}
}  // namespace

bp_status bp_batch_simulate(bp_batch* b, int64_t T, bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_batch_simulate");
    BP_REQUIRE(b, "batch is NULL");
    BP_REQUIRE(T >= 0, "T < 0");
    if (T == 0) return BP_OK;
    cudaGraphExec_t g = nullptr;
    BP_TRY(batch_graph(b, T, &g));
    BP_CUDA(cudaGraphLaunch(g, stream));
    return BP_OK;
}

bp_status bp_batch_prepare(bp_batch* b, int64_t T, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(b, "batch is NULL");
    BP_REQUIRE(T >= 0, "T < 0");
    if (T == 0) return BP_OK;
    cudaGraphExec_t g = nullptr;
    BP_TRY(batch_graph(b, T, &g));
    BP_CUDA(cudaGraphUpload(g, stream));
    return BP_OK;
}

bp_status bp_batch_autotune(bp_batch* b, int32_t probe_steps, int32_t* chosen_threads, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(b, "batch is NULL");
    BP_REQUIRE(probe_steps > 0, "probe_steps must be positive");
    const size_t f = static_cast<size_t>(b->total) * 4;
    char* snap = static_cast<char*>(b->d_snapshot);
    void* src[] = {b->d.V, b->d.ge, b->d.gi, b->d.ref, b->d_spill, b->d.totals};
    const size_t sz[] = {f, f, f, static_cast<size_t>(b->total), f, static_cast<size_t>(b->n_nets) * 32};
    size_t offs[6];
    size_t o = 0;
    for (int k = 0; k < 6; ++k) {
        offs[k] = o;
        o += sz[k];
    }
    for (int k = 0; k < 6; ++k) BP_CUDA(cudaMemcpyAsync(snap + offs[k], src[k], sz[k], cudaMemcpyDeviceToDevice, stream));
    cudaEvent_t e0, e1;
    BP_CUDA(cudaEventCreate(&e0));
    BP_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best_th = b->threads, best_g = b->group, best_ps = b->per_sm;
    const int groups_csr[] = {4, 8, 16, 32};
    const int groups_jit[] = {16, 32};
    const int* groups = b->csr ? groups_csr : groups_jit;
    const int n_groups = b->csr ? 4 : 2;
    bp_status st = BP_OK;
    for (int ps : {1, 2, 4}) {
        // a packing is a candidate only if every network fits its bins
        bool fits = true;
        for (int64_t n : *b->sizes)
            if (((n + 3) & ~int64_t(3)) > bp::bin_capacity(ps)) fits = false;
        if (!fits) continue;
        st = pack(b, ps);
        if (st != BP_OK) break;
        for (int th : {256, 512, 1024}) {
            for (int gi = 0; gi < n_groups; ++gi) {
                // skip a combination whose CTAs cannot share an SM as packed
                if (bp::resident_ctas(b->csr, th, groups[gi], b->smem) < ps) continue;
                for (int k = 0; k < 6; ++k)
                    BP_CUDA(cudaMemcpyAsync(src[k], snap + offs[k], sz[k], cudaMemcpyDeviceToDevice, stream));
                b->threads = th;
                b->group = groups[gi];
                st = enqueue_steps(b, 2, stream);  // warm-up
                if (st != BP_OK) break;
                BP_CUDA(cudaEventRecord(e0, stream));
                st = enqueue_steps(b, probe_steps, stream);
                if (st != BP_OK) break;
                BP_CUDA(cudaEventRecord(e1, stream));
                BP_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                BP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best_th = th;
                    best_g = groups[gi];
                    best_ps = ps;
                }
            }
            if (st != BP_OK) break;
        }
        if (st != BP_OK) break;
    }
    for (int k = 0; k < 6; ++k) BP_CUDA(cudaMemcpyAsync(src[k], snap + offs[k], sz[k], cudaMemcpyDeviceToDevice, stream));
    BP_CUDA(cudaStreamSynchronize(stream));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BP_TRY(st);
    if (b->per_sm != best_ps) BP_TRY(pack(b, best_ps));
    b->threads = best_th;
    b->group = best_g;
    drop_graphs(b);
    if (chosen_threads) *chosen_threads = best_th;
    return BP_OK;
}

bp_status bp_batch_destroy(bp_batch* b) {
    bp::clear_error();
    free_batch(b);
    return BP_OK;
}

}  // extern "C"
