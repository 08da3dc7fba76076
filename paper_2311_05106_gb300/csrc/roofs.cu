// roofs.cu -- measurement kernels that give the roofline denominators of the
// kernels whose bound is not HBM bandwidth:
//   Philox-only draw rate   -- the integer-ALU roof of the JIT rows
//                              (Section 4.2, Appendix C: one 32-bit draw per
//                              synapse, four per Philox4x32-10 block);
//   random L2 reductions    -- the rate at which scattered 4-byte REDs land
//                              in an L2-resident accumulator (the JIT scatter
//                              at n_post = 1e6 and the fused step's delivery);
//   L2-resident copy        -- bytes per second read and written by a copy
//                              between two buffers that stay in L2 (the
//                              fused step below N = 4e5, whose state fits L2).
// Each is a plain grid-stride kernel with every index reduced into its buffer;
// the caller times the launch with CUDA events.
#include "bp_common.cuh"
#include "bp_internal.h"

namespace bp {
namespace {

constexpr int kRoofThreads = 256;

// Each thread draws `blocks` Philox blocks (counters distinct per thread and
// block, one key) and folds the 4 words into a running xor, stored once.
__global__ void __launch_bounds__(kRoofThreads) k_roof_philox(int64_t blocks, uint64_t seed, uint32_t* sink) {
    const uint32_t tid = blockIdx.x * kRoofThreads + threadIdx.x;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    uint32_t acc = 0;
    for (int64_t b = 0; b < blocks; ++b) {
        const uint4 x = Philox::block(make_uint4(static_cast<uint32_t>(b), tid, 0u, 0u), k0, k1);
        acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
    sink[tid] = acc;
}

// Each thread issues `per_thread` 4-byte reductions at pseudo-random
// positions of y[0, n) (a multiply-xorshift hash of (thread, k), mapped into
// [0, n) with a multiply-high), with the keep-in-L2 policy of the delivery.
__global__ void __launch_bounds__(kRoofThreads) k_roof_l2_red(int32_t* y, uint32_t n, int64_t per_thread) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * kRoofThreads + threadIdx.x;
    const uint64_t pol = l2_keep_policy();
    uint64_t h = tid * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    for (int64_t k = 0; k < per_thread; ++k) {
        h ^= h >> 29;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 32;
        const uint32_t i = __umulhi(static_cast<uint32_t>(h), n);
        red_add_keep(y + i, 1, pol);
    }
}

// dst[i] = src[i] for i in [0, n16) (16-byte elements), `reps` passes.
__global__ void __launch_bounds__(kRoofThreads) k_roof_copy(const float4* __restrict__ src, float4* __restrict__ dst,
                                                            int64_t n16, int32_t reps) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kRoofThreads;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kRoofThreads + threadIdx.x;
    for (int32_t r = 0; r < reps; ++r)
        for (int64_t i = i0; i < n16; i += stride) dst[i] = src[i];
}

}  // namespace
}  // namespace bp

extern "C" {

int64_t bp_roof_philox_threads(void) { return static_cast<int64_t>(bp::sm_count()) * 8 * bp::kRoofThreads; }

bp_status bp_roof_philox(int64_t blocks_per_thread, uint64_t seed, uint32_t* sink, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(blocks_per_thread >= 0, "blocks_per_thread < 0");
    BP_REQUIRE(sink != nullptr, "sink is NULL");
    const unsigned grid = static_cast<unsigned>(bp::sm_count() * 8);
    bp::k_roof_philox<<<grid, bp::kRoofThreads, 0, stream>>>(blocks_per_thread, seed, sink);
    BP_LAUNCHED();
    return BP_OK;
}

int64_t bp_roof_l2_red_threads(void) { return static_cast<int64_t>(bp::sm_count()) * 8 * bp::kRoofThreads; }

bp_status bp_roof_l2_red(int32_t* y, int64_t n, int64_t per_thread, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n > 0 && n <= INT32_MAX, "n = %lld not in [1, 2^31)", (long long)n);
    BP_REQUIRE(per_thread >= 0, "per_thread < 0");
    BP_REQUIRE(y != nullptr, "y is NULL");
    const unsigned grid = static_cast<unsigned>(bp::sm_count() * 8);
    bp::k_roof_l2_red<<<grid, bp::kRoofThreads, 0, stream>>>(y, static_cast<uint32_t>(n), per_thread);
    BP_LAUNCHED();
    return BP_OK;
}

bp_status bp_roof_copy(const void* src, void* dst, int64_t bytes, int32_t reps, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(bytes >= 0 && bytes % 16 == 0, "bytes must be a non-negative multiple of 16");
    BP_REQUIRE(reps >= 0, "reps < 0");
    BP_REQUIRE(bytes == 0 || (src && dst), "src or dst is NULL");
    BP_REQUIRE((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0,
               "src and dst must be 16-byte aligned");
    if (bytes == 0 || reps == 0) return BP_OK;
    const unsigned grid = static_cast<unsigned>(bp::sm_count() * 8);
    bp::k_roof_copy<<<grid, bp::kRoofThreads, 0, stream>>>(static_cast<const float4*>(src),
                                                           static_cast<float4*>(dst), bytes / 16, reps);
    BP_LAUNCHED();
    return BP_OK;
}

}  // extern "C"
