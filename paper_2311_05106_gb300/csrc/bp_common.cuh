// bp_common.cuh -- device helpers and host error plumbing shared by libbp's
// translation units.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <type_traits>

#include "bp.h"

namespace bp {

// ---------------------------------------------------------------- host side
// Thread-local message of the last failure; defined in lib.cu.
void set_error(const char* fmt, ...);
void clear_error();

// Device address of the sticky device status word on the current device
// (0 = OK, 3 = timeout, 6 = device-side check).  Defined in lib.cu.
int* device_status_ptr();

// Number of SMs of the current device (cached per device).
int sm_count();

// Maximum opt-in dynamic shared memory per block (bytes, cached per device).
int max_smem_optin();

}  // namespace bp

#define BP_REQUIRE(cond, ...)                    \
    do {                                         \
        if (!(cond)) {                           \
            bp::set_error(__VA_ARGS__);          \
            return BP_ERR_INVALID;               \
        }                                        \
    } while (0)

#define BP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            bp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                          __FILE__, __LINE__);                                          \
            return BP_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

#define BP_LAUNCHED()                                                                   \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess) {                                                        \
            bp::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),   \
                          __FILE__, __LINE__);                                          \
            return BP_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

#define BP_TRY(expr)                       \
    do {                                   \
        bp_status s_ = (expr);             \
        if (s_ != BP_OK) return s_;        \
    } while (0)

namespace bp {

constexpr unsigned FULL_MASK = 0xffffffffu;

// ------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon et al. (SC 2011): each of ten rounds
// multiplies counter words 0 and 2 by the two round multipliers, and the new
// state is (hi(c2 M1) ^ c1 ^ k0, lo(c2 M1), hi(c0 M0) ^ c3 ^ k1, lo(c0 M0));
// the key advances by the two Weyl increments between rounds.
struct Philox {
    static constexpr uint32_t kMulA = 0xD2511F53u;
    static constexpr uint32_t kMulB = 0xCD9E8D57u;
    static constexpr uint32_t kWeylA = 0x9E3779B9u;
    static constexpr uint32_t kWeylB = 0xBB67AE85u;

    __device__ __forceinline__ static uint4 block(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const uint32_t lo_a = kMulA * c.x;
            const uint32_t hi_a = __umulhi(kMulA, c.x);
            const uint32_t lo_b = kMulB * c.z;
            const uint32_t hi_b = __umulhi(kMulB, c.z);
            c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
            k0 += kWeylA;
            k1 += kWeylB;
        }
        return c;
    }
};

// ------------------------------------------------------------ loads / stores
// Streamed (read-once) loads: evict-first so that they do not displace the
// accumulators and state that live in L2.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream_bf16(const __nv_bfloat16* p) {
    unsigned short raw = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(static_cast<uint32_t>(raw) << 16);
}

__device__ __forceinline__ int4 ld_stream4(const int32_t* p) { return __ldcs(reinterpret_cast<const int4*>(p)); }

// Weight kinds of stored CSR entries.
enum { WK_HOMO = 0, WK_F32 = 1, WK_BF16 = 2 };

template <int WK>
__device__ __forceinline__ float load_weight(const void* data, int64_t j, float w_homo) {
    if constexpr (WK == WK_F32) {
        return ld_stream(static_cast<const float*>(data) + j);
    } else if constexpr (WK == WK_BF16) {
        return ld_stream_bf16(static_cast<const __nv_bfloat16*>(data) + j);
    } else {
        return w_homo;
    }
}

// Four consecutive weights starting at a multiple of 4 (16-byte aligned FP32,
// 8-byte aligned BF16).
template <int WK>
__device__ __forceinline__ float4 load_weight4(const void* data, int64_t j, float w_homo) {
    if constexpr (WK == WK_F32) {
        return __ldcs(reinterpret_cast<const float4*>(static_cast<const float*>(data) + j));
    } else if constexpr (WK == WK_BF16) {
        const uint2 raw = __ldcs(reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(data) + j));
        return make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xFFFF0000u),
                           __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xFFFF0000u));
    } else {
        return make_float4(w_homo, w_homo, w_homo, w_homo);
    }
}

// L2 policy that keeps lines resident ahead of evict-normal/evict-first
// lines: used for the event accumulators, which are re-read every step while
// the neuron state streams through L2.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void red_add_keep(int32_t* a, int32_t v, uint64_t pol) {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_keep(float* a, float v, uint64_t pol) {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ int4 ld_keep(const int4* p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_keep(const float4* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_keep(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(int4* p, int4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.s32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_keep(float4* p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}

// Four consecutive FP32 reductions in one 16-byte global operation (the
// address must be 16-byte aligned).
__device__ __forceinline__ void red_add_v4(float* a, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Accumulate into shared or global memory.  Integer counts and FP32 sums
// both use the native red/atom paths.
__device__ __forceinline__ void acc_add(int32_t* p, int32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void acc_add(float* p, float v) { atomicAdd(p, v); }

// ------------------------------------------------------------ warp scans
__device__ __forceinline__ uint64_t warp_inclusive_scan(uint64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t o = __shfl_up_sync(FULL_MASK, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T group_reduce_sum(T v, int width) {
    for (int d = width >> 1; d > 0; d >>= 1) v += __shfl_xor_sync(FULL_MASK, v, d, width);
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace bp
