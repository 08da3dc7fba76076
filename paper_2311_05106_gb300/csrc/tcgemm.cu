// tcgemm.cu -- the weight gradient of spike-driven connections as one dense
// contraction on the tensor cores (Section 3.1: the reverse-mode rule of an
// event-driven product y = W^T x with binary x is dW = x dy^T, summed over
// time and batch; Appendix I's BPTT needs it for the input weights and, at the
// stored entries, for the recurrent weights).
//
//   G[s][a] = sum_k X[k][s] D[k][a]      k = (b, t) over batch and time
//
// X is binary (spikes), D is FP32 (an adjoint).  On sm_103a this runs as
// tcgen05 BF16 MMAs with FP32 accumulators in tensor memory:
//   * D is split into two BF16 terms, D = hi + lo + r with hi = bf16(D),
//     lo = bf16(D - hi), |r| <= 2^-18 |D|; X is exact in BF16.  Both terms are
//     multiplied into the same accumulator, so G carries the FP32 sum of
//     products of D correct to about 2^-17 relative per term.
//   * Operands are packed once into the tensor cores' K-major layout with the
//     128-byte swizzle: blocks of 128 rows x 64 k (16 KB), row r of a block at
//     byte 128 r, its 16-byte chunk c (k = 8c .. 8c + 7) stored at chunk
//     c XOR (r mod 8).  A block is contiguous in global memory, so a stage is
//     loaded with plain bulk copies (cp.async.bulk) and needs no tensor map.
//   * One CTA per (128 rows of D's features) x (256 rows of X's features) x
//     K split: warp 0 streams stages (3 x 64 KB), warp 1 issues the MMAs
//     (M = 128, N = 256, K = 16; 8 per stage) and commits each stage back to
//     the producer, all four warps read the accumulator out of tensor memory
//     and store their split's partial sums.  A fixed-order sum over the
//     splits finishes G, so results are reproducible bit for bit.
// Every wait on an mbarrier is bounded: when one runs out the CTA records
// BP_ERR_TIMEOUT in the status word, waits (bounded) for the copies it issued,
// frees its tensor memory and returns.
#include "bp_common.cuh"
#include "bp_internal.h"

namespace bp {
namespace {

constexpr int kTcM = 128;                 // rows of D's features per tile (TMEM lanes)
constexpr int kTcN = 256;                 // rows of X's features per tile (TMEM columns)
constexpr int kTcKB = 64;                 // k per block: one 128-byte swizzle row of BF16
constexpr int kTcBlock = 128 * 128;       // bytes of a 128-row x 64-k block
constexpr int kTcStages = 3;
constexpr int kTcStageBytes = 4 * kTcBlock;  // D hi, D lo (128 rows each), X (256 rows)
constexpr int kTcThreads = 128;
constexpr uint32_t kTcSpin = 1u << 24;
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024 + 256;

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit = kTcSpin) {
    const uint32_t a = saddr(b);
    for (uint64_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride), version 1, base offset 0 (1024-aligned blocks).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kTcN >> 3) << 17) | ((kTcM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcShape {
    int32_t B, T, T_pad;   // k = b T_pad + t; steps t >= T are zero
    int64_t KB;            // 64-k blocks: B T_pad / 64
    int32_t na, na_pad;    // features of D (multiple of 128 after padding)
    int32_t ns, ns_pad;    // features of X (multiple of 256 after padding)
    int32_t splits;
};

// D [B][T][na] FP32 (row stride na) -> hi / lo blocks [na_pad / 128][KB][16 KB].
// One CTA per block: 64 k x 128 rows staged through shared memory.
__global__ void __launch_bounds__(256) k_pack_hilo(TcShape s, const float* __restrict__ d, uint8_t* __restrict__ hi,
                                                  uint8_t* __restrict__ lo) {
    __shared__ float tile[kTcKB][129];
    const int64_t kb = blockIdx.x;
    const int rb = blockIdx.y;
    // T_pad is a multiple of 64: the block's 64 k share one batch element
    const int64_t k0 = kb * kTcKB;
    const int64_t b = k0 / s.T_pad, t0 = k0 - b * s.T_pad;
    const float* db = d + b * s.T * static_cast<int64_t>(s.na);
    for (int e = threadIdx.x; e < kTcKB * 128; e += 256) {
        const int kk = e >> 7, r = e & 127;
        const int64_t t = t0 + kk;
        const int a = rb * 128 + r;
        float v = 0.f;
        if (t < s.T && a < s.na) v = db[t * s.na + a];
        tile[kk][r] = v;
    }
    __syncthreads();
    uint8_t* ohi = hi + (static_cast<int64_t>(rb) * s.KB + kb) * kTcBlock;
    uint8_t* olo = lo + (static_cast<int64_t>(rb) * s.KB + kb) * kTcBlock;
    for (int u = threadIdx.x; u < 1024; u += 256) {  // 16-byte chunks, in address order
        const int r = u >> 3, c = u & 7;
        const int kc = c ^ (r & 7);  // logical chunk stored at physical chunk c
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float x0 = tile[8 * kc + 2 * p][r], x1 = tile[8 * kc + 2 * p + 1][r];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            wh[p] = static_cast<uint32_t>(__bfloat16_as_ushort(h0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(h1)) << 16);
            wl[p] = static_cast<uint32_t>(__bfloat16_as_ushort(l0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(l1)) << 16);
        }
        reinterpret_cast<uint4*>(ohi)[u] = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        reinterpret_cast<uint4*>(olo)[u] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
}

// Binary X -> BF16 blocks [ns_pad / 128][KB][16 KB].  Feature s < n_dense is
// x_dense[b][t][s] != 0 (u8, row stride n_dense); feature n_dense + i is bit
// i of z_bits[b][t - 1] (words of zw per step; zero at t = 0), i < n_bits.
// One CTA per block: each warp takes 8 of the 64 k and, per k, forms the bits
// of 32 features at a time with a ballot; the block's 64 x 128 bits are then
// written out as BF16 0 / 1 in the swizzled layout.
__global__ void __launch_bounds__(256) k_pack_spikes(TcShape s, const uint8_t* __restrict__ x_dense, int32_t n_dense,
                                                    const uint32_t* __restrict__ z_bits, int32_t n_bits, int32_t zw,
                                                    uint8_t* __restrict__ out) {
    __shared__ uint32_t bits[kTcKB][4];  // [k][32-feature group]
    const int64_t kb = blockIdx.x;
    const int rb = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // T_pad is a multiple of 64: the block's 64 k share one batch element
    const int64_t k0 = kb * kTcKB;
    const int64_t b = k0 / s.T_pad, t0 = k0 - b * s.T_pad;
    const int64_t row0 = b * s.T;  // step (b, 0)
    for (int kk = warp; kk < kTcKB; kk += 8) {
        const int64_t t = t0 + kk;
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
            const int f = rb * 128 + grp * 32 + lane;
            bool v = false;
            if (t < s.T) {
                if (f < n_dense) {
                    v = x_dense[(row0 + t) * n_dense + f] != 0;
                } else if (f - n_dense < n_bits && t > 0) {
                    const int i = f - n_dense;
                    v = (z_bits[(row0 + t - 1) * zw + (i >> 5)] >> (i & 31)) & 1u;
                }
            }
            const unsigned m = __ballot_sync(FULL_MASK, v);
            if (lane == 0) bits[kk][grp] = m;
        }
    }
    __syncthreads();
    uint8_t* o = out + (static_cast<int64_t>(rb) * s.KB + kb) * kTcBlock;
    constexpr uint32_t one = 0x3F80u;  // BF16 1.0
    for (int u = threadIdx.x; u < 1024; u += 256) {
        const int r = u >> 3, c = u & 7;
        const int kc = c ^ (r & 7);
        const int g = r >> 5, sh = r & 31;
        uint32_t w[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t lo = (bits[8 * kc + 2 * p][g] >> sh) & 1u, hi = (bits[8 * kc + 2 * p + 1][g] >> sh) & 1u;
            w[p] = (lo ? one : 0u) | ((hi ? one : 0u) << 16);
        }
        reinterpret_cast<uint4*>(o)[u] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct TcSmemHdr {
    uint64_t full[kTcStages];
    uint64_t empty[kTcStages];
    uint64_t done;
    uint32_t tmem;
    int32_t abort;
    int32_t issued;
};

// part[split][ns_pad][na_pad] = sum over the split's k blocks of X^T (hi + lo).
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_spike_gemm(TcShape s, const uint8_t* __restrict__ dhi,
                                                               const uint8_t* __restrict__ dlo,
                                                               const uint8_t* __restrict__ xs, float* __restrict__ part,
                                                               int* status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = saddr(smem_raw);
    uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-aligned stages
    TcSmemHdr* h = reinterpret_cast<TcSmemHdr*>(base + kTcStages * kTcStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_a = s.na_pad / kTcM;
    const int tiles_s = s.ns_pad / kTcN;
    const int ta = blockIdx.x % tiles_a;
    const int ts = (blockIdx.x / tiles_a) % tiles_s;
    const int split = blockIdx.x / (tiles_a * tiles_s);
    const int64_t kb0 = s.KB * split / s.splits, kb1 = s.KB * (split + 1) / s.splits;
    const int nkb = static_cast<int>(kb1 - kb0);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            mbar_init(&h->full[i], 1);
            mbar_init(&h->empty[i], 1);
        }
        mbar_init(&h->done, 1);
        h->abort = 0;
        h->issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&h->tmem)),
                     "r"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = h->tmem;
    volatile int32_t* vabort = &h->abort;

    if (warp == 0 && lane == 0) {
        // ---- producer: one stage = D hi, D lo (128 rows), X (256 rows = 2 blocks)
        const uint8_t* a_hi = dhi + static_cast<int64_t>(ta) * s.KB * kTcBlock;
        const uint8_t* a_lo = dlo + static_cast<int64_t>(ta) * s.KB * kTcBlock;
        const uint8_t* x0 = xs + static_cast<int64_t>(2 * ts) * s.KB * kTcBlock;
        const uint8_t* x1 = xs + static_cast<int64_t>(2 * ts + 1) * s.KB * kTcBlock;
        int i = 0;
        for (; i < nkb; ++i) {
            const int st = i % kTcStages;
            if (i >= kTcStages && !mbar_wait(&h->empty[st], ((i / kTcStages) - 1) & 1)) {
                *vabort = 1;
                break;
            }
            if (*vabort) break;
            uint8_t* sb = base + st * kTcStageBytes;
            const int64_t off = (kb0 + i) * kTcBlock;
            mbar_arrive_tx(&h->full[st], kTcStageBytes);
            bulk_load(sb, a_hi + off, kTcBlock, &h->full[st]);
            bulk_load(sb + kTcBlock, a_lo + off, kTcBlock, &h->full[st]);
            bulk_load(sb + 2 * kTcBlock, x0 + off, kTcBlock, &h->full[st]);
            bulk_load(sb + 3 * kTcBlock, x1 + off, kTcBlock, &h->full[st]);
        }
        h->issued = i;
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: 4 k-steps of 16 for each of the two D terms
        for (int i = 0; i < nkb; ++i) {
            const int st = i % kTcStages;
            if (!mbar_wait(&h->full[st], (i / kTcStages) & 1)) {
                *vabort = 1;
                break;
            }
            if (*vabort) break;
            tc_fence_after();
            const uint32_t sb = saddr(base + st * kTcStageBytes);
#pragma unroll
            for (int term = 0; term < 2; ++term)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t da = sw128_desc(sb + term * kTcBlock + 32 * kk);
                    const uint64_t db = sw128_desc(sb + 2 * kTcBlock + 32 * kk);
                    mma_bf16(tmem, da, db, (i | term | kk) != 0 ? 1u : 0u);
                }
            mma_commit(&h->empty[st]);
        }
        mma_commit(&h->done);
    }
    __syncwarp();

    // ---- epilogue: lane = row a of the tile, columns = rows s of the tile
    // the accumulator is complete after all nkb stages: a bound that grows with them
    const uint64_t limit = kTcSpin + static_cast<uint64_t>(nkb) * 4096u;
    const bool ok = __all_sync(FULL_MASK, mbar_wait(&h->done, 0, limit) && !*vabort);
    tc_fence_after();
    if (ok && nkb > 0) {
        const int a = ta * kTcM + warp * 32 + lane;
        float* dst = part + static_cast<int64_t>(split) * s.ns_pad * s.na_pad;
        for (int c = 0; c < kTcN; c += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c), v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int64_t srow = static_cast<int64_t>(ts) * kTcN + c + q;
                dst[srow * s.na_pad + a] = v[q];
            }
        }
    } else if (!ok && threadIdx.x == 0 && status) {
        atomicExch(status, static_cast<int>(BP_ERR_TIMEOUT));
    }
    tc_fence_before();
    __syncthreads();
    if (!ok && threadIdx.x == 0) {
        // copies still in flight land in this CTA's shared memory: wait for them
        const int issued = h->issued;
        for (int i = issued - kTcStages < 0 ? 0 : issued - kTcStages; i < issued; ++i)
            mbar_wait(&h->full[i % kTcStages], (i / kTcStages) & 1);
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
    }
}

// G[s][a] (+)= sum over splits of part[split][s][a] (splits in order), one
// element per thread and pass (32-bit index arithmetic: ns na < 2^31 is
// checked at launch).
__global__ void k_tc_reduce(TcShape s, const float* __restrict__ part, float* __restrict__ g, int64_t ldg,
                            int32_t accumulate) {
    const int32_t n = s.ns * s.na;
    const int64_t plane = static_cast<int64_t>(s.ns_pad) * s.na_pad;
    for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int32_t r = e / s.na, c = e - r * s.na;
        const float* pr = part + static_cast<int64_t>(r) * s.na_pad + c;
        float acc = 0.f;
        for (int p = 0; p < s.splits; ++p) acc += pr[p * plane];
        float* o = g + r * ldg + c;
        *o = accumulate ? *o + acc : acc;
    }
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

TcShape make_shape(int32_t B, int32_t T, int32_t na, int32_t ns) {
    TcShape s{};
    s.B = B;
    s.T = T;
    s.T_pad = static_cast<int32_t>(round_up(T, kTcKB));
    s.KB = static_cast<int64_t>(B) * s.T_pad / kTcKB;
    s.na = na;
    s.na_pad = static_cast<int32_t>(round_up(na, kTcM));
    s.ns = ns;
    s.ns_pad = static_cast<int32_t>(round_up(ns, kTcN));
    // K splits: the fewest that minimise (waves of CTAs) x (k blocks per CTA),
    // so that the tiles x splits CTAs fill the SMs (one CTA per SM); at most
    // 16 splits, at least 4 k blocks each (the stage pipeline's depth)
    const int64_t tiles = static_cast<int64_t>(s.na_pad / kTcM) * (s.ns_pad / kTcN);
    const int64_t sms = sm_count();
    int64_t best = 1, best_cost = -1;
    for (int64_t sp = 1; sp <= 16; ++sp) {
        if (sp > 1 && s.KB / sp < 4) break;
        const int64_t waves = (tiles * sp + sms - 1) / sms;
        const int64_t cost = waves * ((s.KB + sp - 1) / sp);
        if (best_cost < 0 || cost < best_cost) {
            best = sp;
            best_cost = cost;
        }
    }
    s.splits = static_cast<int32_t>(best);
    return s;
}

struct TcWork {
    uint8_t* dhi;
    uint8_t* dlo;
    uint8_t* xs;
    float* part;
    size_t bytes;
};

TcWork carve(const TcShape& s, void* work) {
    TcWork w{};
    const size_t blk_a = static_cast<size_t>(s.na_pad / 128) * s.KB * kTcBlock;
    const size_t blk_x = static_cast<size_t>(s.ns_pad / 128) * s.KB * kTcBlock;
    const size_t part = static_cast<size_t>(s.splits) * s.ns_pad * s.na_pad * sizeof(float);
    uint8_t* p = static_cast<uint8_t*>(work);
    w.dhi = p;
    w.dlo = p + blk_a;
    w.xs = p + 2 * blk_a;
    w.part = reinterpret_cast<float*>(p + 2 * blk_a + blk_x);
    w.bytes = 2 * blk_a + blk_x + part;
    return w;
}

}  // namespace

size_t tc_spike_gemm_workspace(int32_t B, int32_t T, int32_t na, int32_t ns) {
    if (B <= 0 || T <= 0 || na <= 0 || ns <= 0) return 0;
    return carve(make_shape(B, T, na, ns), nullptr).bytes;
}

// G[s][a] (+)= sum_{b,t} X_bt[s] D_bt[a]; X from (x_dense, z_bits) as in
// k_pack_spikes, D [B][T][na].  G has row stride ldg.
bp_status launch_tc_spike_gemm(int32_t B, int32_t T, const float* d, int32_t na, const uint8_t* x_dense,
                               int32_t n_dense, const uint32_t* z_bits, int32_t n_bits, int32_t zw, float* g,
                               int64_t ldg, bool accumulate, void* work, size_t work_bytes, cudaStream_t st) {
    const int32_t ns = n_dense + n_bits;
    if (B <= 0 || T <= 0 || na <= 0 || ns <= 0) return BP_OK;
    const TcShape s = make_shape(B, T, na, ns);
    const TcWork w = carve(s, work);
    BP_REQUIRE(work != nullptr && work_bytes >= w.bytes, "workspace of %zu bytes needed, %zu given", w.bytes,
               work_bytes);
    BP_REQUIRE((reinterpret_cast<uintptr_t>(work) & 1023u) == 0, "workspace must be 1024-byte aligned");
    BP_REQUIRE(s.KB <= 0x7FFFFFFF, "too many k blocks");
    BP_REQUIRE(static_cast<int64_t>(ns) * na < (int64_t(1) << 31), "the output's rows x columns must be below 2^31");
    BP_REQUIRE(s.na_pad / 128 <= 65535 && s.ns_pad / 128 <= 65535, "more than 8 388 480 features on one side");
    k_pack_hilo<<<dim3(static_cast<unsigned>(s.KB), s.na_pad / 128), 256, 0, st>>>(s, d, w.dhi, w.dlo);
    BP_LAUNCHED();
    k_pack_spikes<<<dim3(static_cast<unsigned>(s.KB), s.ns_pad / 128), 256, 0, st>>>(s, x_dense, n_dense, z_bits,
                                                                                    n_bits, zw, w.xs);
    BP_LAUNCHED();
    BP_TRY(ensure_smem_attr(reinterpret_cast<const void*>(k_tc_spike_gemm), kTcSmem));
    const int grid = (s.na_pad / kTcM) * (s.ns_pad / kTcN) * s.splits;
    k_tc_spike_gemm<<<grid, kTcThreads, kTcSmem, st>>>(s, w.dhi, w.dlo, w.xs, w.part, device_status_ptr());
    BP_LAUNCHED();
    int64_t rg = (static_cast<int64_t>(ns) * na + 255) / 256;
    if (rg > static_cast<int64_t>(sm_count()) * 16) rg = static_cast<int64_t>(sm_count()) * 16;
    k_tc_reduce<<<static_cast<unsigned>(rg), 256, 0, st>>>(s, w.part, g, ldg, accumulate ? 1 : 0);
    BP_LAUNCHED();
    return BP_OK;
}

}  // namespace bp

extern "C" {

size_t bp_spike_outer_workspace(int64_t K, int32_t M, int32_t N) {
    if (K <= 0 || K > 0x7FFFFFFF || M <= 0 || N <= 0) return 0;
    return bp::tc_spike_gemm_workspace(1, static_cast<int32_t>(K), N, M);
}

bp_status bp_spike_outer(const uint8_t* x, const float* delta, int64_t K, int32_t M, int32_t N, float* out,
                         uint32_t flags, void* work, size_t work_bytes, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(K >= 0 && K <= 0x7FFFFFFF && M >= 0 && N >= 0, "bad sizes K=%lld M=%d N=%d", (long long)K, M, N);
    if (K == 0 || M == 0 || N == 0) {
        if (!(flags & BP_OVERWRITE) || M == 0 || N == 0) return BP_OK;
        BP_REQUIRE(out != nullptr, "out is NULL");
        BP_CUDA(cudaMemsetAsync(out, 0, static_cast<size_t>(M) * N * sizeof(float), stream));
        return BP_OK;
    }
    BP_REQUIRE(x != nullptr && delta != nullptr && out != nullptr, "x, delta and out must not be NULL");
    return bp::launch_tc_spike_gemm(1, static_cast<int32_t>(K), delta, N, x, M, nullptr, 0, 0, out, N,
                                    !(flags & BP_OVERWRITE), work, work_bytes, stream);
}

}  // extern "C"
