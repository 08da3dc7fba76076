// lib.cu -- library-wide entry points: version, error reporting, the sticky
// device status word, parameter defaults and small host-side helpers.
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "bp_common.cuh"
#include "bp_internal.h"

namespace {
thread_local char g_msg[1024] = {0};

// Sticky device status word (one per device that loads the library).
__device__ int g_device_status = 0;

constexpr int kMaxDevices = 64;
int* g_status_addr[kMaxDevices] = {nullptr};
// per-device attributes, queried once; any thread may fill them (the value
// written is the same), so relaxed atomics suffice
std::atomic<int> g_sm_count[kMaxDevices];
std::atomic<int> g_smem_optin[kMaxDevices];
std::mutex g_mu;

// The calling thread's current device ordinal (0 if it cannot be read).
// Ordinals of kMaxDevices or more are valid devices too: they are served
// without the per-device caches below, never folded onto another device.
int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0) return 0;
    return d;
}

bool cached(int d) { return d < kMaxDevices; }
}  // namespace

namespace bp {

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
}

void clear_error() { g_msg[0] = 0; }

// Device address of the status word on the current device, looked up once
// per device and kept for the life of the process (the library is not meant
// to be used across a cudaDeviceReset, which would invalidate it).
int* device_status_ptr() {
    const int d = current_device();
    if (!cached(d)) {
        void* p = nullptr;
        return cudaGetSymbolAddress(&p, g_device_status) == cudaSuccess ? static_cast<int*>(p) : nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_addr[d]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
        g_status_addr[d] = static_cast<int*>(p);
    }
    return g_status_addr[d];
}

int sm_count() {
    const int d = current_device();
    int c = cached(d) ? g_sm_count[d].load(std::memory_order_relaxed) : 0;
    if (!c) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        c = v > 0 ? v : 1;
        if (cached(d)) g_sm_count[d].store(c, std::memory_order_relaxed);
    }
    return c;
}

bp_status ensure_smem_attr(const void* kernel, int bytes) {
    // the limit is a property of the function on each device: record it per
    // (kernel, device) so that a process driving several GPUs sets it on each
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;
    const int d = current_device();
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(kernel, d);
    const auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return BP_OK;
    BP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done[key] = bytes;
    return BP_OK;
}

int max_smem_optin() {
    const int d = current_device();
    int c = cached(d) ? g_smem_optin[d].load(std::memory_order_relaxed) : 0;
    if (!c) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
        c = v > 0 ? v : 48 * 1024;
        if (cached(d)) g_smem_optin[d].store(c, std::memory_order_relaxed);
    }
    return c;
}

LifConst make_lif_const(const bp_coba_params& p) {
    LifConst c;
    c.a_m = static_cast<float>(std::exp(-p.dt / p.tau_m));
    c.a_e = static_cast<float>(std::exp(-p.dt / p.tau_e));
    c.a_i = static_cast<float>(std::exp(-p.dt / p.tau_i));
    c.V_rest = static_cast<float>(p.V_rest);
    c.V_th = static_cast<float>(p.V_th);
    c.V_reset = static_cast<float>(p.V_reset);
    c.E_e = static_cast<float>(p.E_e);
    c.E_i = static_cast<float>(p.E_i);
    c.R = static_cast<float>(p.R);
    c.I_ext = static_cast<float>(p.I_ext);
    c.w_e = static_cast<float>(p.w_e);
    c.w_i = static_cast<float>(p.w_i);
    c.ref_steps = static_cast<int32_t>(std::llround(p.tau_ref / p.dt));
    return c;
}

bp_status check_coba(const bp_coba_params* p) {
    BP_REQUIRE(p != nullptr, "coba params are NULL");
    BP_REQUIRE(p->dt > 0 && p->tau_m > 0 && p->tau_e > 0 && p->tau_i > 0 && p->tau_ref >= 0,
               "coba params: dt and time constants must be positive");
    const double steps = p->tau_ref / p->dt;
    BP_REQUIRE(steps < BP_MAX_REF_STEPS + 0.5,
               "coba params: refractory period of %.1f steps exceeds the %d steps of the uint8 counter",
               steps, BP_MAX_REF_STEPS);
    return BP_OK;
}

}  // namespace bp

extern "C" {

const char* bp_version(void) { return "bp 0.1 sm_103a"; }

const char* bp_last_error(void) { return g_msg; }

int32_t bp_tile_cols(void) { return bp::kTileCols; }

int32_t bp_tile_cols_for(int64_t n_post) {
    const int64_t cap = bp::kTileCols;
    if (n_post <= 0) return 32;
    const int64_t S = (n_post + cap - 1) / cap;
    int64_t W = (n_post + S - 1) / S;
    W = (W + 31) & ~int64_t(31);  // cap is a multiple of 32, so W stays <= cap
    return static_cast<int32_t>(W < cap ? W : cap);
}

bp_status bp_sync_status(bp_stream_t stream) {
    bp::clear_error();
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        bp::set_error("stream error: %s", cudaGetErrorString(e));
        return BP_ERR_CUDA;
    }
    int* addr = bp::device_status_ptr();
    if (!addr) {
        bp::set_error("cannot resolve the device status word");
        return BP_ERR_CUDA;
    }
    int v = 0;
    BP_CUDA(cudaMemcpy(&v, addr, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        int zero = 0;
        BP_CUDA(cudaMemcpy(addr, &zero, sizeof(int), cudaMemcpyHostToDevice));
        if (v == BP_ERR_TIMEOUT) {
            bp::set_error("a bounded device-side wait ran out");
            return BP_ERR_TIMEOUT;
        }
        bp::set_error("device-side check failed (code %d)", v);
        return BP_ERR_DEVICE;
    }
    return BP_OK;
}

bp_status bp_coba_params_default(bp_coba_params* p) {
    BP_REQUIRE(p != nullptr, "p is NULL");
    p->dt = 0.1;
    p->tau_m = 20.0;
    p->tau_e = 5.0;
    p->tau_i = 10.0;
    p->tau_ref = 5.0;
    p->V_rest = -60.0;
    p->V_th = -50.0;
    p->V_reset = -60.0;
    p->E_e = 0.0;
    p->E_i = -80.0;
    p->R = 1.0;
    p->I_ext = 20.0;
    p->w_e = 0.6;
    p->w_i = 6.7;
    return BP_OK;
}

// SplitMix64 (Steele, Lea and Flood 2014): the state advances by the golden
// ratio increment; the output is the state passed through two xor-shift /
// multiply mixing rounds and a final xor-shift.
uint64_t bp_projection_seed(uint64_t net_seed, int32_t projection) {
    uint64_t x = net_seed + 0x9E3779B97F4A7C15ull * (static_cast<uint64_t>(projection) + 1ull);
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

bp_status bp_jit_desc_init(bp_jit_desc* d, uint64_t seed, double p, int32_t wkind, float w0, float w1) {
    bp::clear_error();
    BP_REQUIRE(d != nullptr, "desc is NULL");
    BP_REQUIRE(p > 0.0 && p <= 1.0, "connection probability %g not in (0, 1]", p);
    BP_REQUIRE(wkind >= BP_JIT_HOMO && wkind <= BP_JIT_NORMAL, "unknown JIT weight kind %d", wkind);
    const double x = 2.0 / p - 1.0;
    double K = std::ceil(x - 1e-12 * std::fabs(x));
    if (K < 1.0) K = 1.0;
    BP_REQUIRE(K < 4294967296.0, "gap range K = %.0f exceeds 32 bits (p too small)", K);
    d->seed = seed;
    d->p = p;
    d->K = static_cast<int64_t>(K);
    d->wkind = wkind;
    d->w0 = w0;
    d->w1 = w1;
    return BP_OK;
}

}  // extern "C"
