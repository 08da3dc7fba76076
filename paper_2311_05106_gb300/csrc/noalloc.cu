// noalloc.cu -- bp_event_csrmv_dense_noalloc: the dense-event CSR product
// for callers that cannot allocate device memory.
//
// bp_event_csrmv_dense needs a caller-owned workspace for the compacted spike
// list.  Some callers cannot provide one: code running inside a framework that
// owns the whole device memory pool (a cudaMalloc behind its back fragments
// the pool or fails), and real-time loops where cudaMalloc / cudaFree may
// synchronise the device and stall the loop.  This entry point keeps its
// scratch in a fixed array in device memory that is part of the library
// image, so no call allocates.
//
// Costs and limits: the array holds kNoAllocMaxPre spike ids plus a counter
// (about 4 MiB), and every GPU that loads the library keeps it until the
// process exits.  All calls on a device share the array, so two calls that
// may overlap on the GPU (different streams, or different host threads)
// race on it and must be ordered by the caller.
#include <mutex>

#include "bp_common.cuh"
#include "bp_internal.h"

namespace {

// n_pre limit of bp_event_csrmv_dense_noalloc.
constexpr int64_t kNoAllocMaxPre = int64_t(1) << 20;

// [0..3]: spike counter (and padding to 16 bytes); [4 ..]: spike ids.
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocMaxPre + 4];

constexpr int kMaxDevices = 64;
int32_t* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
bp_status scratch_address(int32_t** out) {
    int dev = 0;
    BP_CUDA(cudaGetDevice(&dev));
    BP_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        BP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return BP_OK;
}

}  // namespace

extern "C" {

int64_t bp_event_csrmv_dense_noalloc_max_pre(void) { return kNoAllocMaxPre; }

bp_status bp_event_csrmv_dense_noalloc(int64_t n_pre, int64_t n_post, const int64_t* indptr, const int32_t* indices,
                                       const void* data, int32_t wkind, float w_homo, const uint8_t* events, void* y,
                                       int32_t y_is_count, uint32_t flags, bp_stream_t stream) {
    bp::clear_error();
    BP_REQUIRE(n_pre >= 0 && n_pre <= kNoAllocMaxPre,
               "n_pre = %lld exceeds the fixed scratch of bp_event_csrmv_dense_noalloc (at most %lld presynaptic "
               "rows); use bp_event_csrmv_dense with a caller-owned workspace",
               (long long)n_pre, (long long)kNoAllocMaxPre);
    bp::CsrArgs a;
    a.n_pre = n_pre;
    a.n_post = n_post;
    a.indptr = indptr;
    a.indices = indices;
    a.data = data;
    a.wkind = wkind;
    a.w_homo = w_homo;
    a.tile_ptr = nullptr;
    a.tile_cols = 0;
    a.w_bound = nullptr;
    BP_REQUIRE(n_post >= 0 && n_post <= INT32_MAX, "bad n_post");
    BP_REQUIRE(indptr != nullptr, "indptr is NULL");
    BP_REQUIRE(wkind >= BP_W_HOMO && wkind <= BP_W_BF16, "unknown weight kind %d", wkind);
    BP_REQUIRE(wkind == BP_W_HOMO || data != nullptr, "weights are NULL for a non-homogeneous kind");
    BP_REQUIRE(!y_is_count || wkind == BP_W_HOMO, "integer counts need homogeneous weights");
    BP_REQUIRE(n_post == 0 || y != nullptr, "y is NULL");
    BP_REQUIRE(n_pre == 0 || (events && indices), "events or indices is NULL");
    int32_t* scratch = nullptr;
    BP_TRY(scratch_address(&scratch));
    if (flags & BP_OVERWRITE) BP_CUDA(cudaMemsetAsync(y, 0, static_cast<size_t>(n_post) * 4, stream));
    if (n_pre == 0) return BP_OK;
    int32_t* cnt = scratch;
    int32_t* list = scratch + 4;
    // the counter keeps the previous call's value: it must start at zero
    BP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), stream));
    BP_TRY(bp::launch_spike_compact(n_pre, events, list, cnt, stream));
    const int mode = (flags & BP_ACC_GLOBAL) ? 1 : ((flags & BP_ACC_SHARED) ? 2 : 0);
    return bp::launch_event_csrmv(a, list, cnt, n_pre, y, y_is_count != 0, nullptr, mode, stream);
}

}  // extern "C"
