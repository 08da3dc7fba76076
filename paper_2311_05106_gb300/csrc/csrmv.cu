// csrmv.cu -- event-driven CSR products (a5): the scatter y = W^T s over the
// spiking rows (Appendix B), its gather form y_pre = W x, the weight gradient,
// and the post-column tile index.
//
// Work decomposition.  A "group" of G lanes (G in {4, 8, 16, 32}, chosen on
// the device from the mean segment length; widened up to the whole CTA when a
// call delivers too few rows to keep the lanes busy) walks one spiking row's
// segment with coalesced, evict-first loads of indices and weights, four
// strided loads in flight per lane.  Two accumulation modes:
//   direct  -- atomics straight into y in L2; right when the step delivers
//              few events compared with n_post (the network steps).
//   tiled   -- CTA (s, r) owns post columns [s W, (s+1) W) in shared memory
//              (W <= 57344 4-byte accumulators) and rows r, r+R, ... of the
//              spike list; segments come from the tile index (or the whole
//              row when one tile covers n_post).  Shared-memory atomics absorb
//              the scatter; the tile is flushed to y once, skipping zeros.
// In auto mode each CTA reads the spike count and picks the mode from the
// expected number of events, so no host synchronisation is needed.  The
// gather form reads x through L1/L2, or, given a tile index, stages x in
// shared memory one post tile at a time.
#include "bp_common.cuh"
#include "bp_internal.h"
#include "bp_rows.cuh"

namespace bp {
namespace {

constexpr int kDirectThreads = 256;

// mode: 0 auto, 1 direct, 2 tiled.  W = tile width (post columns per tile),
// S = number of tiles (the grid is S x R CTAs).
// Lanes per (row, tile) segment with vector loads: about 16 entries per lane.
__device__ __forceinline__ int pick_group_v4(int64_t nnz, int64_t n_pre, int64_t tiles) {
    const int64_t denom = (n_pre > 0 ? n_pre : 1) * (tiles > 0 ? tiles : 1);
    const int64_t mean = nnz / denom;
    if (mean >= 512) return 32;
    if (mean >= 256) return 16;
    if (mean >= 128) return 8;
    return 4;
}

// Lanes per row group when few rows are to be delivered: the group (which
// needs no shuffles, so it may span several warps) doubles while there are
// still lanes for every row, so that a handful of long rows is walked by the
// whole grid instead of one group each.
__device__ __forceinline__ int widen_group(int G, int64_t rows, int64_t lanes, int cap) {
    while (G < cap && rows * 2 * G <= lanes) G *= 2;
    return G;
}

// Pairs: 8-byte index loads and one FP32 pair / bf16x2 word per two entries
// (half the load instructions of the scalar walk), unaligned first / last
// entry on its own.
template <typename Acc, int WK>
__device__ __forceinline__ void scatter_segment_v2(const int32_t* __restrict__ indices, const void* __restrict__ data,
                                                   float w_homo, int64_t b0, int64_t b1, int lane, int G,
                                                   Acc* __restrict__ out, int64_t col0) {
    int64_t a2 = (b0 + 1) & ~int64_t(1);
    if (a2 > b1) a2 = b1;
    int64_t e2 = b1 & ~int64_t(1);
    if (e2 < a2) e2 = a2;
    {
        const int64_t nh = a2 - b0, nt = b1 - e2;
        for (int64_t t = lane; t < nh + nt; t += G) {
            const int64_t j = t < nh ? b0 + t : e2 + (t - nh);
            acc_add(out + (ld_stream(indices + j) - col0), event_value<Acc>(load_weight<WK>(data, j, w_homo)));
        }
    }
    const int64_t c1 = e2 >> 1;
    int64_t cb = (a2 >> 1) + lane;
    int2 c[4];
    float2 w[4];
    auto load = [&]() {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t cc = cb + u * G;
            if (cc < c1) {
                c[u] = __ldcs(reinterpret_cast<const int2*>(indices + 2 * cc));
                if constexpr (WK == WK_F32) {
                    w[u] = __ldcs(reinterpret_cast<const float2*>(static_cast<const float*>(data) + 2 * cc));
                } else if constexpr (WK == WK_BF16) {
                    const uint32_t raw = __ldcs(reinterpret_cast<const unsigned int*>(static_cast<const __nv_bfloat16*>(data) + 2 * cc));
                    w[u] = make_float2(__uint_as_float(raw << 16), __uint_as_float(raw & 0xFFFF0000u));
                } else {
                    w[u] = make_float2(w_homo, w_homo);
                }
            } else {
                c[u] = make_int2(-1, -1);
                w[u] = make_float2(0.f, 0.f);
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
        }
        cb += 4 * G;
        if (cb >= c1) break;
        load();
    }
}

template <typename Acc, int WK, bool VECL>
__device__ __forceinline__ void scatter_any(const int32_t* __restrict__ indices, const void* __restrict__ data,
                                            float w_homo, int64_t b0, int64_t b1, int lane, int G,
                                            Acc* __restrict__ out, int64_t col0) {
    if constexpr (VECL && WK == WK_BF16)
        scatter_segment_v2<Acc, WK>(indices, data, w_homo, b0, b1, lane, G, out, col0);
    else if constexpr (VECL)
        scatter_segment_v4<Acc, WK>(indices, data, w_homo, b0, b1, lane, G, out, col0);
    else
        scatter_segment<Acc, WK>(indices, data, w_homo, b0, b1, lane, G, out, col0);
}

// Flattened walk of the tile segments of spiking rows, one warp at a time.
//
// Each warp of the CTA takes 32 spiking rows at a time (one per lane).  Every
// lane fetches its row's segment in post tile s, [b0, b0 + len); a warp
// prefix sum of the lengths lays the 32 segments end to end as one flat list
// of T units (start[k] = flat position of segment k), and the 32 lanes stream
// flat positions l, l + 32, ...: consecutive lanes read consecutive units of
// a segment (coalesced), and the warp's lanes stay busy whatever the segment
// lengths, so short segments cost neither idle lanes nor a memory latency
// each.  A lane finds its first segment by binary search over the 33 starts
// and then follows the segment boundaries as its position advances.  The
// next 32 rows' bounds are loaded while the current ones are walked (spike
// ids one round ahead of the row extents and tile offsets).  Warps share
// nothing but the tile, so they proceed without block-wide barriers.
//
// Units are entries, or, with 16-byte aligned operands, 16-byte chunks of 4
// entries aligned in memory (each lane then moves 16 bytes of indices per
// load): segment k covers chunks [b0 / 4, (b1 + 3) / 4), and the entries of
// its first chunk before b0 and of its last chunk from b1 on are masked off.
struct WarpList {
    // (global unit index of flat position 0 of segment k) << 8 | edge, with
    // edge = (entries skipped in the first chunk) | (entries kept in the last
    // chunk) << 2 for chunked units (0 for entries)
    int64_t base[32];
    int32_t start[33];  // exclusive prefix of the 32 segments' unit counts; start[32] = T
};
struct FlatSmem {
    WarpList w[kTileThreads / 32];
};

// A warp whose 32 segments hold more than this many units (far more than 32
// segments of a tile without repeated columns: a tile spans at most 54 944
// columns) is walked segment by segment instead; flat positions stay far from
// the 32-bit range.
constexpr int64_t kFlatMaxEntries = int64_t(1) << 24;

// The walk's index and weight loads ask L2 to fetch 256 bytes around each
// request, and leave the lines at the normal L2 priority (not evict-first)
// and out of L1: the 256-byte block of a segment's edge is shared with the
// neighbouring tile's segment of the same row, which a CTA of the next tile
// group reads at about the same time (the CTAs of every tile walk the same
// rows in the same order), so it is still in L2 then.  Measured on the
// graded cells: the hint alone +0.3-1.9 %, with normal priority instead of
// evict-first a further +2-17 % (weighted fixed-point and count tiles; -3 %
// for BF16 weights with FP32 shared atomics).
#define BP_PFX ".L2::256B"
#define BP_WALK_COP ".L1::no_allocate"

// Eight consecutive indices (and weights) of a 32-byte aligned unit, one
// streaming 256-bit load each (BF16 weights: one 128-bit load).
__device__ __forceinline__ void ld_stream8(const int32_t* p, int32_t c[8]) {
    asm volatile("ld.global" BP_WALK_COP BP_PFX ".v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
                 : "l"(p));
}

// 16 bytes, streaming, with the same L2 fetch-size hint.
__device__ __forceinline__ uint4 ld_stream16_pf(const void* p) {
    uint4 v;
    asm volatile("ld.global" BP_WALK_COP BP_PFX ".v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

template <int WK>
__device__ __forceinline__ void load_weight8(const void* data, int64_t j, float w_homo, float w[8]) {
    if constexpr (WK == WK_F32) {
        const float* p = static_cast<const float*>(data) + j;
        asm volatile("ld.global" BP_WALK_COP BP_PFX ".v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]), "=f"(w[5]), "=f"(w[6]), "=f"(w[7])
                     : "l"(p));
    } else if constexpr (WK == WK_BF16) {
        const uint4 v = ld_stream16_pf(static_cast<const __nv_bfloat16*>(data) + j);
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            w[2 * k] = __uint_as_float(u[k] << 16);
            w[2 * k + 1] = __uint_as_float(u[k] & 0xFFFF0000u);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = w_homo;
    }
}

// One event into the shared-memory tile: an integer count, an FP32 atomic,
// or (FX) round(w 2^s) into the tile's 32-bit fixed-point sum (fx_scale = 2^s).
template <typename Acc, bool FX>
__device__ __forceinline__ void tile_add(Acc* p, float w, float fx_scale) {
    if constexpr (FX) {
        atomicAdd(reinterpret_cast<int32_t*>(p), __float2int_rn(w * fx_scale));
    } else {
        acc_add(p, event_value<Acc>(w));
    }
}

// The same, as one predicated shared-memory reduction at the tile's 32-bit
// shared address (computed once per walk): no branch around the update and
// no generic-to-shared conversion per event.  `on` false: nothing is added.
template <typename Acc, bool FX>
__device__ __forceinline__ void tile_red(uint32_t acc_s, uint32_t c, float w, float fx_scale, bool on) {
    const uint32_t addr = acc_s + 4u * c;
    if constexpr (FX || std::is_same<Acc, int32_t>::value) {
        const int32_t v = FX ? __float2int_rn(w * fx_scale) : 1;
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q red.shared.add.u32 [%0], %1;\n}" ::"r"(addr),
                     "r"(v), "r"(static_cast<uint32_t>(on))
                     : "memory");
    } else {
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q red.shared.add.f32 [%0], %1;\n}" ::"r"(addr),
                     "f"(w), "r"(static_cast<uint32_t>(on))
                     : "memory");
    }
}

template <typename Acc, int WK, int EPU, int U, bool FX>
__device__ __forceinline__ void warp_flat_walk(const CsrArgs& a, const WarpList& L, int32_t T,
                                               Acc* __restrict__ acc, int64_t col0, int32_t W, float fx_scale) {
    const int lane = threadIdx.x & 31;
    const uint32_t acc_s = static_cast<uint32_t>(__cvta_generic_to_shared(acc));
    const uint32_t col0_u = static_cast<uint32_t>(col0);
    int32_t e = lane;
    if (e >= T) return;
    int k_lo = 0, k_hi = 32;  // start[k_lo] <= e < start[k_hi]
    while (k_hi - k_lo > 1) {
        const int mid = (k_lo + k_hi) >> 1;
        if (L.start[mid] <= e) k_lo = mid; else k_hi = mid;
    }
    int seg = k_lo;
    int32_t cur = L.start[seg];
    int32_t nxt = L.start[seg + 1];
    int64_t pk = L.base[seg];
    static_assert(EPU == 1 || EPU == 4 || EPU == 8, "units of 1, 4 or 8 entries");
    constexpr uint32_t kAll = (1u << EPU) - 1u;
    constexpr int kEdgeSh = EPU == 8 ? 3 : 2;  // bits of the first entry's offset in `edge`
    for (; e < T; e += 32 * U) {
        int32_t col[U][EPU];
        float w[U][EPU];
        uint32_t msk[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int32_t eq = e + 32 * q;
            msk[q] = 0;
#pragma unroll
            for (int m = 0; m < EPU; ++m) {
                col[q][m] = 0;
                w[q][m] = 0.f;
            }
            if (eq < T) {
                if (eq >= nxt) {
                    do {
                        ++seg;
                        cur = nxt;
                        nxt = L.start[seg + 1];
                    } while (eq >= nxt);
                    pk = L.base[seg];
                }
                const int64_t g = static_cast<int64_t>(eq - cur) + (pk >> 8);
                if constexpr (EPU == 8) {
                    ld_stream8(a.indices + 8 * g, col[q]);
                    load_weight8<WK>(a.data, 8 * g, a.w_homo, w[q]);
                } else if constexpr (EPU == 4) {
                    const uint4 cu = ld_stream16_pf(a.indices + 4 * g);
                    const int4 c4 = make_int4(static_cast<int32_t>(cu.x), static_cast<int32_t>(cu.y),
                                              static_cast<int32_t>(cu.z), static_cast<int32_t>(cu.w));
                    float4 w4;
                    if constexpr (WK == WK_F32) {
                        const uint4 wu = ld_stream16_pf(static_cast<const float*>(a.data) + 4 * g);
                        w4 = make_float4(__uint_as_float(wu.x), __uint_as_float(wu.y), __uint_as_float(wu.z),
                                         __uint_as_float(wu.w));
                    } else {
                        w4 = load_weight4<WK>(a.data, 4 * g, a.w_homo);
                    }
                    col[q][0] = c4.x, col[q][1] = c4.y, col[q][2] = c4.z, col[q][3] = c4.w;
                    w[q][0] = w4.x, w[q][1] = w4.y, w[q][2] = w4.z, w[q][3] = w4.w;
                }
                if constexpr (EPU > 1) {
                    const uint32_t edge = static_cast<uint32_t>(pk & 0xFF);
                    uint32_t mm = kAll;
                    if (eq == cur) mm &= kAll << (edge & (EPU - 1u));
                    if (eq == nxt - 1) mm &= (1u << (edge >> kEdgeSh)) - 1u;
                    msk[q] = mm;
                } else {
                    col[q][0] = ld_stream(a.indices + g);
                    w[q][0] = load_weight<WK>(a.data, g, a.w_homo);
                    msk[q] = 1u;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
#pragma unroll
            for (int m = 0; m < EPU; ++m) {
                // an index outside this tile (an operand that does not match
                // its tile index) is skipped rather than written out of the tile
                // modulo 2^32: a column outside [col0, col0 + W) maps to >= W
                // (n_post < 2^31), so one unsigned compare bounds it
                const uint32_t c = static_cast<uint32_t>(col[q][m]) - col0_u;
                tile_red<Acc, FX>(acc_s, c, w[q][m], fx_scale, ((msk[q] >> m) & 1u) && c < static_cast<uint32_t>(W));
            }
        }
    }
}

template <typename Acc, int WK, bool VECL, bool FX = false, bool WIDE = false>
__global__ void __launch_bounds__(kTileThreads, 1)
    k_csr_scatter(CsrArgs a, const int32_t* __restrict__ spike_list, const int32_t* __restrict__ n_spikes,
                  int64_t max_spikes, Acc* __restrict__ y, int mode, int32_t W, int32_t S,
                  int64_t* __restrict__ events_total, int* status) {
    static_assert(!FX || std::is_same<Acc, float>::value, "fixed-point tiles accumulate float products");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* acc = reinterpret_cast<Acc*>(smem_raw);
    FlatSmem& fs = *reinterpret_cast<FlatSmem*>(smem_raw + static_cast<size_t>(W) * sizeof(Acc));
    int64_t ns = *n_spikes;
    ns = ns < max_spikes ? ns : max_spikes;
    const int64_t nnz = a.indptr[a.n_pre];
    if (mode == 0) {
        // auto: shared tiles pay off once events clearly outnumber the
        // accumulators each CTA has to zero and flush
        const int64_t est = ns * (nnz / (a.n_pre > 0 ? a.n_pre : 1));
        mode = (est >= 4 * static_cast<int64_t>(W) * S) ? 2 : 1;
    }
    int64_t ev = 0;
    if (mode == 1) {
        const int G = widen_group(VECL && WK != WK_F32 ? pick_group_v4(nnz, a.n_pre, 1) : pick_group(nnz, a.n_pre, 1), ns,
                                  static_cast<int64_t>(gridDim.x) * blockDim.x, blockDim.x);
        const int lane = threadIdx.x % G;
        const int64_t ngroups = static_cast<int64_t>(gridDim.x) * blockDim.x / G;
        for (int64_t u = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / G; u < ns; u += ngroups) {
            const int32_t i = spike_list[u];
            if (static_cast<uint32_t>(i) >= static_cast<uint64_t>(a.n_pre)) continue;
            const int64_t b0 = a.indptr[i], b1 = a.indptr[i + 1];
            if (lane == 0) ev += b1 - b0;
            scatter_any<Acc, WK, VECL && WK != WK_F32>(a.indices, a.data, a.w_homo, b0, b1, lane, G, y, 0);
        }
    } else {
        const int s = blockIdx.x % S;
        const int64_t r = blockIdx.x / S;
        const int64_t R = gridDim.x / S;
        const int64_t col0 = static_cast<int64_t>(s) * W;
        const int t = threadIdx.x;
        const int warp = t >> 5, lane = t & 31;
        WarpList& L = fs.w[warp];
        for (int k = t; k < W; k += kTileThreads) acc[k] = Acc(0);
        __syncthreads();
        // the CTA's rows are spike-list positions r + R m, m in [0, M); warp w
        // takes an equal contiguous share [m_lo, m_hi) of them, 32 per round
        const int32_t M = static_cast<int32_t>(ns > r ? (ns - r + R - 1) / R : 0);  // ns <= n_pre < 2^31
        // fixed-point tiles: with the weight bound b, every column of this
        // CTA's tile sums at most m b in magnitude (m below); 2^s m b <= 2^29
        // keeps the sum of the rounded terms inside int32
        float fx_scale = 1.f, fx_inv = 1.f;
        if constexpr (FX) {
            const float b = __int_as_float(a.w_bound[0]);
            if (!(b > 0.f)) {  // no bound recorded: nothing is added
                if (t == 0 && status) atomicExch(status, static_cast<int>(BP_ERR_DEVICE));
                return;
            }
            // a column receives at most one run of entries from each row, so
            // at most m = min(M, cmax) runs here, cmax = the most rows with an
            // entry in one column (0: not recorded)
            const int32_t cmax = a.w_bound[1];
            const int32_t m = cmax > 0 && cmax < M ? cmax : M;
            // m b < 2^(em + eb), from the two exponents (m b itself may
            // overflow FP32 for weights near its range)
            int em = 0, eb = 0;
            frexpf(static_cast<float>(m > 0 ? m : 1), &em);
            frexpf(b, &eb);
            int sx = 29 - em - eb;
            // 2^s must stay a normal float both ways: for bounds below
            // 2^-97 / M the scale stops at 2^126 (events then carry an
            // absolute error up to 2^-127)
            sx = sx < -126 ? -126 : (sx > 126 ? 126 : sx);
            fx_scale = ldexpf(1.f, sx);
            fx_inv = ldexpf(1.f, -sx);
        }
        const int32_t m_lo = static_cast<int32_t>(static_cast<int64_t>(M) * warp / (kTileThreads / 32));
        const int32_t m_hi = static_cast<int32_t>(static_cast<int64_t>(M) * (warp + 1) / (kTileThreads / 32));
        auto row_id = [&](int32_t k) -> int32_t {
            const int32_t m = m_lo + 32 * k + lane;
            return m < m_hi ? spike_list[r + R * m] : -1;
        };
        // the loads that give a row's segment in tile s; the arithmetic on
        // them is left to seg_of so that the loads stay in flight
        struct Raw { int64_t rs, re; int32_t t0, t1; bool ok; };
        auto row_raw = [&](int32_t i) -> Raw {
            Raw x{0, 0, 0, 0, false};
            if (static_cast<uint32_t>(i) < static_cast<uint64_t>(a.n_pre)) {
                x.ok = true;
                x.rs = a.indptr[i];
                if (a.tile_ptr) {
                    const int32_t* tp = a.tile_ptr + static_cast<int64_t>(i) * (S + 1) + s;
                    x.t0 = tp[0];
                    x.t1 = tp[1];
                    if (events_total && s == 0) x.re = a.indptr[i + 1];
                } else {
                    x.re = a.indptr[i + 1];
                }
            }
            return x;
        };
        auto seg_of = [&](const Raw& x, int64_t& b0, int64_t& len) {
            b0 = 0;
            len = 0;
            if (!x.ok) return;
            if (a.tile_ptr) {
                b0 = x.rs + x.t0;
                len = static_cast<int64_t>(x.t1) - x.t0;
                if (events_total && s == 0) ev += x.re - x.rs;
            } else {
                b0 = x.rs;
                len = x.re - x.rs;
                if (events_total && s == 0) ev += len;
            }
            if (len < 0) len = 0;
        };
        Raw cur = row_raw(row_id(0));
        int32_t id_next = row_id(1);
        for (int32_t k = 0; m_lo + 32 * k < m_hi; ++k) {
            int64_t b0, len;
            seg_of(cur, b0, len);
            // the segment's units: entries, or aligned 4-entry chunks
            int64_t u0 = b0, units = len;
            int64_t edge = 0;
            if constexpr (VECL) {
                // units of 4 entries (8 when WIDE); edge = first entry's offset in
                // its unit | entries used in the last unit, shifted past it
                constexpr int SH = WIDE ? 3 : 2;
                constexpr int64_t UW = int64_t(1) << SH;
                u0 = b0 >> SH;
                const int64_t u1 = (b0 + len + UW - 1) >> SH;
                units = len > 0 ? u1 - u0 : 0;
                edge = (b0 & (UW - 1)) | ((b0 + len - UW * (u1 - 1)) << SH);
            }
            int64_t incl = units;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t o = __shfl_up_sync(FULL_MASK, incl, d);
                if (lane >= d) incl += o;
            }
            const int64_t T = __shfl_sync(FULL_MASK, incl, 31);
            const int64_t excl = incl - units;
            // the next round's bounds are fetched while this one is walked
            const Raw nxt_raw = row_raw(id_next);
            id_next = row_id(k + 2);
            if (T <= kFlatMaxEntries) {
                __syncwarp();  // the previous round's walk has finished with L
                L.start[lane] = static_cast<int32_t>(excl);
                L.base[lane] = (u0 << 8) | (edge & 0xFF);
                if (lane == 31) L.start[32] = static_cast<int32_t>(T);
                __syncwarp();
                constexpr int EPU = WIDE ? 8 : (VECL ? 4 : 1);
                constexpr int UW = WIDE ? (WK == WK_HOMO ? 2 : 1)
                                        : (VECL ? (WK == WK_HOMO ? 4 : 3)
                                                : (std::is_same<Acc, int32_t>::value && WK == WK_HOMO ? 16 : 8));
                warp_flat_walk<Acc, WK, EPU, UW, FX>(a, L, static_cast<int32_t>(T), acc, col0, W, fx_scale);
            } else {
                // the warp walks its lanes' segments one after another, four
                // loads in flight per lane
                for (int l = 0; l < 32; ++l) {
                    const int64_t c0 = __shfl_sync(FULL_MASK, b0, l);
                    const int64_t c1 = c0 + __shfl_sync(FULL_MASK, len, l);
                    for (int64_t j = c0 + lane; j < c1; j += 4 * 32) {
                        int32_t c[4];
                        float wv[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int64_t jj = j + 32 * q;
                            c[q] = jj < c1 ? ld_stream(a.indices + jj) : -1;
                            wv[q] = jj < c1 ? load_weight<WK>(a.data, jj, a.w_homo) : 0.f;
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t kk = static_cast<uint32_t>(static_cast<int64_t>(c[q]) - col0);
                            if (c[q] >= 0 && kk < static_cast<uint32_t>(W)) tile_add<Acc, FX>(acc + kk, wv[q], fx_scale);
                        }
                    }
                }
            }
            cur = nxt_raw;
        }
        __syncthreads();
        const int64_t rem = a.n_post - col0;
        const int lim = static_cast<int>(rem < W ? rem : W);
        if constexpr (FX) {
            // fixed-point sums, times 2^-s, one 16-byte reduction per four
            // columns (y 16-byte aligned), the ragged tail one by one
            const int32_t* ia = reinterpret_cast<const int32_t*>(acc);
            const bool y16 = (reinterpret_cast<uintptr_t>(y) & 15) == 0;
            const int lim4 = y16 ? (lim & ~3) : 0;
            for (int k = 4 * t; k < lim4; k += 4 * kTileThreads) {
                const int4 v = *reinterpret_cast<const int4*>(ia + k);
                if (v.x | v.y | v.z | v.w)
                    red_add_v4(y + col0 + k, make_float4(static_cast<float>(v.x) * fx_inv, static_cast<float>(v.y) * fx_inv,
                                                         static_cast<float>(v.z) * fx_inv, static_cast<float>(v.w) * fx_inv));
            }
            for (int k = lim4 + t; k < lim; k += kTileThreads)
                if (ia[k] != 0) acc_add(y + col0 + k, static_cast<float>(ia[k]) * fx_inv);
        } else if constexpr (std::is_same<Acc, float>::value) {
            // FP32 sums: one 16-byte reduction per four columns (y 16-byte
            // aligned; col0 is a multiple of 32), the ragged tail one by one
            if ((reinterpret_cast<uintptr_t>(y) & 15) == 0) {
                const int lim4 = lim & ~3;
                for (int k = 4 * t; k < lim4; k += 4 * kTileThreads) {
                    const float4 v = *reinterpret_cast<const float4*>(acc + k);
                    if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) red_add_v4(y + col0 + k, v);
                }
                for (int k = lim4 + t; k < lim; k += kTileThreads)
                    if (acc[k] != 0.f) acc_add(y + col0 + k, acc[k]);
            } else {
                for (int k = t; k < lim; k += kTileThreads)
                    if (acc[k] != 0.f) acc_add(y + col0 + k, acc[k]);
            }
        } else {
            for (int k = t; k < lim; k += kTileThreads) {
                const Acc v = acc[k];
                if (v != Acc(0)) acc_add(y + col0 + k, v);
            }
        }
    }
    if (events_total) block_add_i64(ev, events_total);
}

// Direct-only variant without dynamic shared memory (more CTAs per SM).
template <typename Acc, int WK, bool VECL>
__global__ void __launch_bounds__(kDirectThreads)
    k_csr_scatter_direct(CsrArgs a, const int32_t* __restrict__ spike_list, const int32_t* __restrict__ n_spikes,
                         int64_t max_spikes, Acc* __restrict__ y, int64_t* __restrict__ events_total) {
    int64_t ns = *n_spikes;
    ns = ns < max_spikes ? ns : max_spikes;
    const int64_t nnz = a.indptr[a.n_pre];
    const int G = widen_group(VECL && WK != WK_F32 ? pick_group_v4(nnz, a.n_pre, 1) : pick_group(nnz, a.n_pre, 1), ns,
                              static_cast<int64_t>(gridDim.x) * blockDim.x, blockDim.x);
    const int lane = threadIdx.x % G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * blockDim.x / G;
    int64_t ev = 0;
    for (int64_t u = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / G; u < ns; u += ngroups) {
        const int32_t i = spike_list[u];
        if (static_cast<uint32_t>(i) >= static_cast<uint64_t>(a.n_pre)) continue;
        const int64_t b0 = a.indptr[i], b1 = a.indptr[i + 1];
        if (lane == 0) ev += b1 - b0;
        scatter_any<Acc, WK, VECL && WK != WK_F32>(a.indices, a.data, a.w_homo, b0, b1, lane, G, y, 0);
    }
    if (events_total) block_add_i64(ev, events_total);
}

// Gather over all rows: y_pre[i] (+)= sum_j w_j x[indices[j]].
template <int WK>
__global__ void __launch_bounds__(256) k_csr_gather(CsrArgs a, const float* __restrict__ x, float* __restrict__ y,
                                                    int overwrite) {
    const int64_t nnz = a.indptr[a.n_pre];
    const int G = pick_group(nnz, a.n_pre, 1);
    const int lane = threadIdx.x % G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * blockDim.x / G;
    const int64_t g0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / G;
    // every lane of a warp runs the same number of iterations so that the
    // group reduction's shuffles stay converged
    const int64_t warp_groups = 32 / G;
    const int64_t base0 = g0 - (g0 % warp_groups);
    for (int64_t gb = base0; gb < a.n_pre; gb += ngroups) {
        const int64_t i = gb + (g0 - base0);
        float sum = 0.f;
        if (i < a.n_pre) {
            const int64_t b0 = a.indptr[i], b1 = a.indptr[i + 1];
            int64_t j = b0 + lane;
            for (; j + 3 * G < b1; j += 4 * G) {
                int32_t c[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) c[u] = ld_stream(a.indices + j + u * G);
#pragma unroll
                for (int u = 0; u < 4; ++u) w[u] = load_weight<WK>(a.data, j + u * G, a.w_homo);
#pragma unroll
                for (int u = 0; u < 4; ++u) sum += w[u] * __ldg(x + c[u]);
            }
            for (; j < b1; j += G) sum += load_weight<WK>(a.data, j, a.w_homo) * __ldg(x + ld_stream(a.indices + j));
        }
        sum = group_reduce_sum(sum, G);
        if (i < a.n_pre && lane == 0) y[i] = overwrite ? sum : y[i] + sum;
    }
}

// Gather with x staged in shared memory: CTA (s, r) copies x[s W, (s+1) W)
// into shared memory and walks rows r, r + R, ... over their segments in
// post tile s (from the tile index; the whole row when one tile covers
// n_post), G lanes per row with four index loads in flight per lane.  With
// one tile each row has a single owner and is written directly; with
// several, each (row, tile) partial sum is added to y_pre with one atomic
// (y_pre cleared first when overwriting).  Indices outside the tile (an index
// that does not match the matrix) contribute nothing.
template <int WK>
__global__ void __launch_bounds__(kTileThreads, 1) k_csr_gather_tiled(CsrArgs a, const float* __restrict__ x,
                                                                      float* __restrict__ y, int overwrite,
                                                                      int32_t W, int32_t S) {
    extern __shared__ __align__(16) float xs[];
    const int s = blockIdx.x % S;
    const int64_t r = blockIdx.x / S;
    const int64_t R = gridDim.x / S;
    const int64_t col0 = static_cast<int64_t>(s) * W;
    const int64_t rem = a.n_post - col0;
    const int lim = static_cast<int>(rem < W ? rem : W);
    for (int t = threadIdx.x; t < W; t += blockDim.x) xs[t] = t < lim ? x[col0 + t] : 0.f;
    __syncthreads();
    const int64_t nnz = a.indptr[a.n_pre];
    const int G = pick_group(nnz, a.n_pre, S);
    const int lane = threadIdx.x % G;
    const int64_t gid = threadIdx.x / G;
    const int64_t ng = blockDim.x / G;
    for (int64_t i = r + R * gid; i < a.n_pre; i += R * ng) {
        const int64_t rs = a.indptr[i];
        int64_t b0, b1;
        if (S > 1) {
            const int32_t* tp = a.tile_ptr + i * (S + 1) + s;
            b0 = rs + tp[0];
            b1 = rs + tp[1];
        } else {
            b0 = rs;
            b1 = a.indptr[i + 1];
        }
        float sum = 0.f;
        for (int64_t j = b0 + lane; j < b1; j += 4 * G) {
            int32_t c[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t jj = j + u * G;
                c[u] = jj < b1 ? ld_stream(a.indices + jj) : static_cast<int32_t>(col0);
                w[u] = jj < b1 ? load_weight<WK>(a.data, jj, a.w_homo) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = static_cast<uint32_t>(static_cast<int64_t>(c[u]) - col0);
                sum += k < static_cast<uint32_t>(W) ? w[u] * xs[k] : 0.f;
            }
        }
        sum = group_reduce_sum(sum, G);
        if (lane == 0) {
            if (S == 1) {
                y[i] = overwrite ? sum : y[i] + sum;
            } else if (b1 > b0) {
                atomicAdd(y + i, sum);
            }
        }
    }
}

// dw[j] += dy[indices[j]] for the entries of each spiking row.
__global__ void __launch_bounds__(256) k_csr_dw(CsrArgs a, const int32_t* __restrict__ spike_list,
                                                const int32_t* __restrict__ n_spikes, int64_t max_spikes,
                                                const float* __restrict__ dy, float* __restrict__ dw) {
    int64_t ns = *n_spikes;
    ns = ns < max_spikes ? ns : max_spikes;
    const int64_t nnz = a.indptr[a.n_pre];
    const int G = pick_group(nnz, a.n_pre, 1);
    const int lane = threadIdx.x % G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * blockDim.x / G;
    for (int64_t u = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / G; u < ns; u += ngroups) {
        const int32_t i = spike_list[u];
        if (static_cast<uint32_t>(i) >= static_cast<uint64_t>(a.n_pre)) continue;
        const int64_t b0 = a.indptr[i], b1 = a.indptr[i + 1];
        for (int64_t j = b0 + lane; j < b1; j += G) dw[j] += __ldg(dy + ld_stream(a.indices + j));
    }
}

// CSR validation: a warp per row counts a bad extent, out-of-range indices,
// descending neighbours and repeated neighbours (the last two only make sense
// for a valid extent); counts are summed with one atomic per warp and kind.
__global__ void __launch_bounds__(256) k_csr_check(int64_t n_pre, int64_t n_post, int64_t nnz,
                                                   const int64_t* __restrict__ indptr,
                                                   const int32_t* __restrict__ indices,
                                                   unsigned long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (indptr[0] != 0) atomicAdd(out + 0, 1ull);
        if (indptr[n_pre] != nnz) atomicAdd(out + 0, 1ull);
    }
    for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32; i < n_pre; i += nwarps) {
        const int64_t b0 = indptr[i], b1 = indptr[i + 1];
        if (b1 < b0 || b0 < 0 || b1 > nnz) {
            if (lane == 0) atomicAdd(out + 0, 1ull);
            continue;
        }
        unsigned long long bad = 0, desc = 0, dup = 0;
        for (int64_t j = b0 + lane; j < b1; j += 32) {
            const int32_t c = indices[j];
            if (c < 0 || c >= n_post) ++bad;
            if (j > b0) {
                const int32_t prev = indices[j - 1];
                if (prev > c) ++desc;
                if (prev == c) ++dup;
            }
        }
        bad = group_reduce_sum(bad, 32);
        desc = group_reduce_sum(desc, 32);
        dup = group_reduce_sum(dup, 32);
        if (lane == 0) {
            if (bad) atomicAdd(out + 1, bad);
            if (desc) atomicAdd(out + 2, 1ull);
            if (dup && !desc) atomicAdd(out + 3, 1ull);
        }
    }
}

// tile_ptr[i (S+1) + s] = lower_bound(row i, s W) - indptr[i].
__global__ void k_tile_index(int64_t n_pre, const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                             int32_t W, int32_t S, int32_t* __restrict__ tile_ptr) {
    const int64_t total = n_pre * (S + 1);
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / (S + 1);
        const int64_t s = t % (S + 1);
        const int64_t rs = indptr[i], re = indptr[i + 1];
        int64_t lo = rs, hi = re;
        if (s < S) {
            const int64_t key = s * static_cast<int64_t>(W);
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (indices[mid] < key) lo = mid + 1; else hi = mid;
            }
        } else {
            lo = re;
        }
        tile_ptr[t] = static_cast<int32_t>(lo - rs);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // the bound slots: no bound yet
        tile_ptr[total] = 0;
        tile_ptr[total + 1] = 0;
    }
}

// Weight bound of the fixed-point tiles: the largest absolute sum of one
// row's entries in one column (rows sorted, so a repeated column is a run of
// equal indices).  A warp per row; the lane at the start of each run sums the
// run; the maximum, rounded up, goes into *slot as FP32 bits (non-negative
// floats order like their bit patterns, so an integer maximum is a float
// maximum).  Each run also counts its row in its column: cnt[c] = the number
// of rows with an entry in column c (exact int32 counts).
template <int WK>
__global__ void __launch_bounds__(256) k_tile_weight_bound(int64_t n_pre, int64_t n_post,
                                                          const int64_t* __restrict__ indptr,
                                                          const int32_t* __restrict__ indices,
                                                          const void* __restrict__ data, float w_homo,
                                                          int32_t* __restrict__ slot, int32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    float best = 0.f;
    for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n_pre; i += warps) {
        const int64_t r0 = indptr[i], r1 = indptr[i + 1];
        for (int64_t j = r0 + lane; j < r1; j += 32) {
            const int32_t c = indices[j];
            if (j > r0 && indices[j - 1] == c) continue;  // not the start of its run
            if (static_cast<uint32_t>(c) < static_cast<uint64_t>(n_post)) atomicAdd(cnt + c, 1);
            float run = fabsf(load_weight<WK>(data, j, w_homo));
            for (int64_t k = j + 1; k < r1 && indices[k] == c; ++k) run += fabsf(load_weight<WK>(data, k, w_homo));
            best = fmaxf(best, run);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) best = fmaxf(best, __shfl_xor_sync(FULL_MASK, best, d));
    if (lane == 0) {
        // a run's FP32 sum may round down: a relative 2^-16 covers runs of up
        // to 256 repeats; never 0 (0 means no bound)
        float up = best * (1.f + 1.f / 65536.f);
        if (!(up >= 1.17549435e-38f)) up = 1.17549435e-38f;
        atomicMax(slot, __float_as_int(up));
    }
}

// *slot = max over c of cnt[c] (the largest number of rows with an entry in
// one column).
__global__ void __launch_bounds__(256) k_max_count(int64_t n, const int32_t* __restrict__ cnt,
                                                  int32_t* __restrict__ slot) {
    int32_t best = 0;
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < n;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x)
        best = max(best, cnt[c]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) best = max(best, __shfl_xor_sync(FULL_MASK, best, d));
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(slot, best);
}

template <typename Acc, int WK, bool VECL, bool WIDE = false>
bp_status launch_scatter_t(const CsrArgs& a, const int32_t* spike_list, const int32_t* n_spikes, int64_t max_spikes,
                           void* y, int64_t* events_total, int mode, cudaStream_t s) {
    Acc* yy = static_cast<Acc*>(y);
    const bool fx = (mode & kModeFixed) != 0;
    mode &= ~kModeFixed;
    // tile geometry: one tile covers n_post if it fits, otherwise the tile index's width
    const int32_t cap = kTileCols;
    int32_t W = 0, S = 0;
    if (a.n_post <= cap) {
        W = static_cast<int32_t>(a.n_post > 0 ? a.n_post : 1);
        W = (W + 31) & ~31;
        S = 1;
    } else if (a.tile_ptr && a.tile_cols > 0 && a.tile_cols <= cap) {
        W = a.tile_cols;
        S = static_cast<int32_t>((a.n_post + W - 1) / W);
    }
    const bool can_tile = S > 0;
    if (!can_tile) mode = 1;
    CsrArgs at = a;
    if (S == 1) at.tile_ptr = nullptr;  // one tile covers every column: whole rows
    if (mode == 1) {
        const int grid = sm_count() * 8;
        k_csr_scatter_direct<Acc, WK, VECL><<<grid, kDirectThreads, 0, s>>>(a, spike_list, n_spikes, max_spikes, yy,
                                                                            events_total);
        BP_LAUNCHED();
        return BP_OK;
    }
    const size_t smem = static_cast<size_t>(W) * sizeof(Acc) + sizeof(FlatSmem);
    // one 1024-thread CTA per SM: R row groups per tile so that S x R covers the SMs
    int64_t R = static_cast<int64_t>(sm_count()) / S;
    if (R < 1) R = 1;
    const int64_t grid = R * S;
    if constexpr (std::is_same<Acc, float>::value) {
        if (fx) {
            auto k = k_csr_scatter<float, WK, VECL, true, WIDE>;
            BP_TRY(ensure_smem_attr(reinterpret_cast<const void*>(k), static_cast<int>(cap * sizeof(Acc) + sizeof(FlatSmem))));
            k<<<static_cast<unsigned>(grid), kTileThreads, smem, s>>>(at, spike_list, n_spikes, max_spikes, yy, mode, W,
                                                                     S, events_total, device_status_ptr());
            BP_LAUNCHED();
            return BP_OK;
        }
    }
    BP_TRY(ensure_smem_attr(reinterpret_cast<const void*>(k_csr_scatter<Acc, WK, VECL, false, WIDE>),
                            static_cast<int>(cap * sizeof(Acc) + sizeof(FlatSmem))));
    k_csr_scatter<Acc, WK, VECL, false, WIDE><<<static_cast<unsigned>(grid), kTileThreads, smem, s>>>(
        at, spike_list, n_spikes, max_spikes, yy, mode, W, S, events_total, nullptr);
    BP_LAUNCHED();
    return BP_OK;
}

bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

template <typename Acc, int WK>
bp_status launch_scatter_a(const CsrArgs& a, const int32_t* sl, const int32_t* ns, int64_t mx, void* y, int64_t* ev,
                           int mode, cudaStream_t s) {
    // Aligned operands: the tiled walk moves 16-byte chunks of indices (and
    // of FP32 / 8-byte chunks of BF16 weights), reading the whole aligned
    // chunks that hold a segment's first and last entries; the direct walk
    // takes 16-byte index loads for homogeneous weights and pairs (8-byte
    // index and 4-byte weight loads) for BF16 weights, and stays scalar for
    // FP32 weights (its vector forms measured slower or mixed).
    const bool vec = aligned_to(a.indices, 16) && (WK == WK_HOMO || (WK == WK_F32 && aligned_to(a.data, 16)) ||
                                                   (WK == WK_BF16 && aligned_to(a.data, 8)));
    // BF16 weights with 32-byte aligned indices: the tiled walk moves 8-entry
    // units (256-bit index and 128-bit weight loads).  Measured on the graded
    // n = 1e6 cells: BF16 +6-9 % on long segments (-3 % on 52-entry ones).
    if constexpr (WK == WK_BF16) {
        if (aligned_to(a.indices, 32) && aligned_to(a.data, 16))
            return launch_scatter_t<Acc, WK, true, true>(a, sl, ns, mx, y, ev, mode, s);
    }
    // FP32 weights with 32-byte aligned indices and weights: 8-entry units
    // too (256-bit index and weight loads).  Measured with the walk's
    // normal-priority loads: +1.1-4.5 % with fixed-point tiles, +0.1-2.0 %
    // with FP32 atomics; counts stay on 4-entry units (-2.2 to +2.9 %).
    if constexpr (WK == WK_F32) {
        if (aligned_to(a.indices, 32) && aligned_to(a.data, 32))
            return launch_scatter_t<Acc, WK, true, true>(a, sl, ns, mx, y, ev, mode, s);
    }
    if (vec) return launch_scatter_t<Acc, WK, true>(a, sl, ns, mx, y, ev, mode, s);
    return launch_scatter_t<Acc, WK, false>(a, sl, ns, mx, y, ev, mode, s);
}

template <typename Acc>
bp_status launch_scatter_wk(const CsrArgs& a, const int32_t* sl, const int32_t* ns, int64_t mx, void* y, int64_t* ev,
                            int mode, cudaStream_t s) {
    switch (a.wkind) {
        case BP_W_F32: return launch_scatter_a<Acc, WK_F32>(a, sl, ns, mx, y, ev, mode, s);
        case BP_W_BF16: return launch_scatter_a<Acc, WK_BF16>(a, sl, ns, mx, y, ev, mode, s);
        default: return launch_scatter_a<Acc, WK_HOMO>(a, sl, ns, mx, y, ev, mode, s);
    }
}

bp_status check_csr(const CsrArgs& a) {
    BP_REQUIRE(a.n_pre >= 0 && a.n_post >= 0, "negative matrix size");
    BP_REQUIRE(a.n_pre <= INT32_MAX && a.n_post <= INT32_MAX, "matrix side exceeds 2^31 - 1");
    BP_REQUIRE(a.indptr != nullptr, "indptr is NULL");
    BP_REQUIRE(a.wkind >= BP_W_HOMO && a.wkind <= BP_W_BF16, "unknown weight kind %d", a.wkind);
    BP_REQUIRE(a.wkind == BP_W_HOMO || a.data != nullptr, "weights are NULL for a non-homogeneous kind");
    BP_REQUIRE(a.tile_ptr == nullptr || (a.tile_cols > 0 && a.tile_cols % 32 == 0 && a.tile_cols <= kTileCols),
               "tile_cols %d must be a positive multiple of 32 <= %d", a.tile_cols, kTileCols);
    return BP_OK;
}

int gather_grid(int64_t n_pre) {
    const int64_t need = (n_pre * 8 + 255) / 256;  // at least 8 lanes per row
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    const int64_t g = need < cap ? need : cap;
    return static_cast<int>(g > 0 ? g : 1);
}

}  // namespace

bp_status launch_event_csrmv(const CsrArgs& a, const int32_t* spike_list, const int32_t* n_spikes, int64_t max_spikes,
                             void* y, bool counts, int64_t* events_total, int mode, cudaStream_t s) {
    if (max_spikes <= 0 || a.n_post == 0) return BP_OK;
    if (counts) return launch_scatter_wk<int32_t>(a, spike_list, n_spikes, max_spikes, y, events_total,
                                                  mode & ~kModeFixed, s);
    if ((mode & kModeFixed) && a.w_bound == nullptr) {
        set_error("BP_ACC_FIXED needs a tile index (bp_csr_tile_index + bp_csr_tile_weight_bound)");
        return BP_ERR_INVALID;
    }
    return launch_scatter_wk<float>(a, spike_list, n_spikes, max_spikes, y, events_total, mode, s);
}

}  // namespace bp

namespace {

int mode_from_flags(uint32_t flags) {
    const int fixed = (flags & BP_ACC_FIXED) ? bp::kModeFixed : 0;
    if (flags & BP_ACC_GLOBAL) return 1 | fixed;
    if (flags & BP_ACC_SHARED) return 2 | fixed;
    return fixed;
}

bp::CsrArgs make_csr(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices, const void* data,
                     int32_t wkind, float w_homo, const int32_t* tile_ptr, int32_t tile_cols) {
    bp::CsrArgs a;
    a.n_pre = n_pre;
    a.n_post = n_post;
    a.indptr = indptr;
    a.indices = indices;
    a.data = data;
    a.wkind = wkind;
    a.w_homo = w_homo;
    a.tile_ptr = tile_ptr;
    a.tile_cols = tile_cols;
    a.w_bound = nullptr;
    if (tile_ptr && tile_cols > 0 && n_pre >= 0 && n_post >= 0) {
        const int64_t S = (n_post + tile_cols - 1) / tile_cols;
        a.w_bound = tile_ptr + n_pre * (S + 1);  // the two bound slots at the end of the index
    }
    return a;
}

}  // namespace

extern "C" {

bp_status bp_event_csrmv(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                         const void* data, int32_t wkind, float w_homo, const int32_t* spike_list,
                         const int32_t* n_spikes, int64_t max_spikes, void* y, int32_t y_is_count,
                         const int32_t* tile_ptr, int32_t tile_cols, uint32_t flags, bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_event_csrmv");
    const bp::CsrArgs a = make_csr(n_pre, n_post, indptr, indices, data, wkind, w_homo, tile_ptr, tile_cols);
    BP_TRY(bp::check_csr(a));
    BP_REQUIRE(!y_is_count || wkind == BP_W_HOMO, "integer counts need homogeneous weights");
    BP_REQUIRE(max_spikes >= 0 && max_spikes <= n_pre, "max_spikes %lld not in [0, n_pre]", (long long)max_spikes);
    BP_REQUIRE(n_post == 0 || y != nullptr, "y is NULL");
    BP_REQUIRE(max_spikes == 0 || (spike_list && n_spikes && indices), "spike list, count or indices is NULL");
    if (flags & BP_OVERWRITE) BP_CUDA(cudaMemsetAsync(y, 0, static_cast<size_t>(n_post) * 4, stream));
    return bp::launch_event_csrmv(a, spike_list, n_spikes, max_spikes, y, y_is_count != 0, nullptr,
                                  mode_from_flags(flags), stream);
}

size_t bp_event_csrmv_dense_workspace_bytes(int64_t n_pre) {
    return 16 + static_cast<size_t>(n_pre > 0 ? n_pre : 0) * sizeof(int32_t);
}

bp_status bp_event_csrmv_dense(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                               const void* data, int32_t wkind, float w_homo, const uint8_t* events,
                               void* workspace, void* y, int32_t y_is_count, const int32_t* tile_ptr,
                               int32_t tile_cols, uint32_t flags, bp_stream_t stream) {
    bp::clear_error();
    const bp::CsrArgs a = make_csr(n_pre, n_post, indptr, indices, data, wkind, w_homo, tile_ptr, tile_cols);
    BP_TRY(bp::check_csr(a));
    BP_REQUIRE(!y_is_count || wkind == BP_W_HOMO, "integer counts need homogeneous weights");
    BP_REQUIRE(n_post == 0 || y != nullptr, "y is NULL");
    BP_REQUIRE(n_pre == 0 || (events && workspace && indices), "events, workspace or indices is NULL");
    BP_REQUIRE((reinterpret_cast<uintptr_t>(workspace) & 15) == 0, "workspace must be 16-byte aligned");
    if (flags & BP_OVERWRITE) BP_CUDA(cudaMemsetAsync(y, 0, static_cast<size_t>(n_post) * 4, stream));
    if (n_pre == 0) return BP_OK;
    int32_t* cnt = static_cast<int32_t*>(workspace);
    int32_t* list = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + 16);
    BP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), stream));
    BP_TRY(bp::launch_spike_compact(n_pre, events, list, cnt, stream));
    return bp::launch_event_csrmv(a, list, cnt, n_pre, y, y_is_count != 0, nullptr, mode_from_flags(flags),
                                  stream);
}

int64_t bp_csr_tile_index_size(int64_t n_pre, int64_t n_post, int32_t tile_cols) {
    if (n_pre < 0 || n_post < 0 || tile_cols <= 0) return -1;
    const int64_t S = (n_post + tile_cols - 1) / tile_cols;
    return n_pre * (S + 1) + 2;  // + the two bound slots
}

bp_status bp_csr_tile_index(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                            int32_t tile_cols, int32_t* tile_ptr, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n_pre >= 0 && n_post >= 0 && n_pre <= INT32_MAX && n_post <= INT32_MAX, "bad sizes");
    BP_REQUIRE(tile_cols > 0 && tile_cols % 32 == 0 && tile_cols <= bp::kTileCols,
               "tile_cols %d must be a positive multiple of 32 <= %d", tile_cols, bp::kTileCols);
    BP_REQUIRE(n_pre == 0 || (indptr && indices && tile_ptr), "a required pointer is NULL");
    if (n_pre == 0) {  // only the bound slots
        if (tile_ptr) BP_CUDA(cudaMemsetAsync(tile_ptr, 0, 2 * sizeof(int32_t), stream));
        return BP_OK;
    }
    const int32_t S = static_cast<int32_t>((n_post + tile_cols - 1) / tile_cols);
    const int64_t total = n_pre * (S + 1);
    int64_t grid = (total + 255) / 256;
    if (grid > bp::sm_count() * 32) grid = bp::sm_count() * 32;
    bp::k_tile_index<<<static_cast<unsigned>(grid), 256, 0, stream>>>(n_pre, indptr, indices, tile_cols, S,
                                                                       tile_ptr);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_csr_tile_weight_bound(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                                   const void* data, int32_t wkind, float w_homo, int32_t tile_cols, int32_t* tile_ptr,
                                   int32_t* work, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n_pre >= 0 && n_post >= 0 && n_pre <= INT32_MAX && n_post <= INT32_MAX, "bad sizes");
    BP_REQUIRE(tile_cols > 0 && tile_cols % 32 == 0 && tile_cols <= bp::kTileCols,
               "tile_cols %d must be a positive multiple of 32 <= %d", tile_cols, bp::kTileCols);
    BP_REQUIRE(wkind >= BP_W_HOMO && wkind <= BP_W_BF16, "unknown weight kind %d", wkind);
    BP_REQUIRE(tile_ptr != nullptr, "tile_ptr is NULL");
    BP_REQUIRE(n_pre == 0 || (indptr && indices), "indptr or indices is NULL");
    BP_REQUIRE(wkind == BP_W_HOMO || n_pre == 0 || data != nullptr, "weights are NULL for a non-homogeneous kind");
    BP_REQUIRE(n_post == 0 || work != nullptr, "work is NULL");
    const int64_t S = (n_post + tile_cols - 1) / tile_cols;
    int32_t* slot = tile_ptr + n_pre * (S + 1);
    BP_CUDA(cudaMemsetAsync(slot, 0, 2 * sizeof(int32_t), stream));
    if (n_post > 0) BP_CUDA(cudaMemsetAsync(work, 0, static_cast<size_t>(n_post) * sizeof(int32_t), stream));
    int64_t grid = (n_pre * 32 + 255) / 256;
    if (grid > bp::sm_count() * 16) grid = bp::sm_count() * 16;
    if (grid < 1) grid = 1;
    switch (wkind) {
        case BP_W_F32:
            bp::k_tile_weight_bound<bp::WK_F32><<<static_cast<unsigned>(grid), 256, 0, stream>>>(n_pre, n_post, indptr, indices,
                                                                                                 data, w_homo, slot, work);
            break;
        case BP_W_BF16:
            bp::k_tile_weight_bound<bp::WK_BF16><<<static_cast<unsigned>(grid), 256, 0, stream>>>(n_pre, n_post, indptr, indices,
                                                                                                  data, w_homo, slot, work);
            break;
        default:
            bp::k_tile_weight_bound<bp::WK_HOMO><<<static_cast<unsigned>(grid), 256, 0, stream>>>(n_pre, n_post, indptr, indices,
                                                                                                  data, w_homo, slot, work);
    }
    BP_LAUNCHED();
    if (n_post > 0) {
        int64_t g2 = (n_post + 255) / 256;
        if (g2 > bp::sm_count() * 8) g2 = bp::sm_count() * 8;
        bp::k_max_count<<<static_cast<unsigned>(g2), 256, 0, stream>>>(n_post, work, slot + 1);
        BP_LAUNCHED();
    }
    return BP_OK;
}

bp_status bp_csr_check(int64_t n_pre, int64_t n_post, int64_t nnz, const int64_t* indptr, const int32_t* indices,
                       int64_t* out, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n_pre >= 0 && n_post >= 0 && nnz >= 0, "negative size");
    BP_REQUIRE(indptr && out, "indptr or out is NULL");
    BP_REQUIRE(nnz == 0 || indices, "indices is NULL");
    BP_CUDA(cudaMemsetAsync(out, 0, 4 * sizeof(int64_t), stream));
    int64_t grid = (n_pre * 32 + 255) / 256;
    if (grid > bp::sm_count() * 16) grid = bp::sm_count() * 16;
    if (grid < 1) grid = 1;
    bp::k_csr_check<<<static_cast<unsigned>(grid), 256, 0, stream>>>(n_pre, n_post, nnz, indptr, indices,
                                                                      reinterpret_cast<unsigned long long*>(out));
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_event_csrmv_t(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                           const void* data, int32_t wkind, float w_homo, const float* x_post, float* y_pre,
                           const int32_t* tile_ptr, int32_t tile_cols, uint32_t flags, bp_stream_t stream) {
    bp::clear_error();
    const bp::NvtxRange nvtx("bp_event_csrmv_t");
    const bp::CsrArgs a = make_csr(n_pre, n_post, indptr, indices, data, wkind, w_homo, tile_ptr, tile_cols);
    BP_TRY(bp::check_csr(a));
    BP_REQUIRE(n_pre == 0 || (y_pre && x_post && indices), "x_post, y_pre or indices is NULL");
    if (n_pre == 0) return BP_OK;
    const int ow = (flags & BP_OVERWRITE) ? 1 : 0;
    // shared-memory tiles of x when the caller gives a tile index (measured:
    // 2.2x the L2 form at n = 1e6 with ~550 entries per row and tile; the L2
    // form wins when x stays in L1/L2 or segments are short) and the L2 form
    // is not forced
    int32_t W = 0, S = 0;
    if (tile_ptr && tile_cols > 0) {
        W = tile_cols;
        S = static_cast<int32_t>((n_post + W - 1) / W);
        if (S < 1) S = 1;
    }
    if (S > 0 && !(flags & BP_ACC_GLOBAL)) {
        if (S > 1 && ow) BP_CUDA(cudaMemsetAsync(y_pre, 0, static_cast<size_t>(n_pre) * sizeof(float), stream));
        const size_t smem = static_cast<size_t>(W) * sizeof(float);
        int64_t R = static_cast<int64_t>(bp::sm_count()) / S;
        const int64_t rows_cap = (n_pre + 255) / 256;
        if (R > rows_cap) R = rows_cap;
        if (R < 1) R = 1;
        const unsigned grid = static_cast<unsigned>(S * R);
        const int ow_tile = S == 1 ? ow : 0;
#define BP_GATHER_T(WKV)                                                                                          \
    do {                                                                                                          \
        BP_TRY(bp::ensure_smem_attr(reinterpret_cast<const void*>(bp::k_csr_gather_tiled<WKV>),                  \
                                    static_cast<int>(bp::kTileCols * sizeof(float))));                            \
        bp::k_csr_gather_tiled<WKV><<<grid, bp::kTileThreads, smem, stream>>>(a, x_post, y_pre, ow_tile, W, S);   \
    } while (0)
        switch (wkind) {
            case BP_W_F32: BP_GATHER_T(bp::WK_F32); break;
            case BP_W_BF16: BP_GATHER_T(bp::WK_BF16); break;
            default: BP_GATHER_T(bp::WK_HOMO); break;
        }
#undef BP_GATHER_T
        BP_LAUNCHED();
        return BP_OK;
    }
    const int grid = bp::gather_grid(n_pre);
    switch (wkind) {
        case BP_W_F32: bp::k_csr_gather<bp::WK_F32><<<grid, 256, 0, stream>>>(a, x_post, y_pre, ow); break;
        case BP_W_BF16: bp::k_csr_gather<bp::WK_BF16><<<grid, 256, 0, stream>>>(a, x_post, y_pre, ow); break;
        default: bp::k_csr_gather<bp::WK_HOMO><<<grid, 256, 0, stream>>>(a, x_post, y_pre, ow); break;
    }
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_event_csrmv_bwd(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                             const void* data, int32_t wkind, float w_homo, const int32_t* spike_list,
                             const int32_t* n_spikes, int64_t max_spikes, const float* dy, float* dw, float* dx_pre,
                             const int32_t* tile_ptr, int32_t tile_cols, bp_stream_t stream) {
    bp::clear_error();
    const bp::CsrArgs a = make_csr(n_pre, n_post, indptr, indices, data, wkind, w_homo, tile_ptr, tile_cols);
    BP_TRY(bp::check_csr(a));
    BP_REQUIRE(max_spikes >= 0 && max_spikes <= n_pre, "max_spikes out of range");
    BP_REQUIRE(dy != nullptr || n_post == 0, "dy is NULL");
    if (dw && max_spikes > 0) {
        BP_REQUIRE(spike_list && n_spikes && indices, "spike list, count or indices is NULL");
        const int grid = bp::sm_count() * 8;
        bp::k_csr_dw<<<grid, 256, 0, stream>>>(a, spike_list, n_spikes, max_spikes, dy, dw);
        BP_LAUNCHED();
    }
    if (dx_pre)
        return bp_event_csrmv_t(n_pre, n_post, indptr, indices, data, wkind, w_homo, dy, dx_pre, tile_ptr, tile_cols, 0,
                                stream);
    return BP_OK;
}

}  // extern "C"
