// Error reporting, argument validation and device queries of libpact.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "pact_internal.cuh"

namespace {
thread_local char g_msg[512] = "";
}

namespace pact {

pact_status fail(pact_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return s;
}

pact_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PACT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return PACT_OK;
}

namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_sms[kMaxDevices];                 // SM count per device, 0 = not queried yet
constexpr unsigned long long kDefaultWaitNs = 200ull * 1000ull * 1000ull;
std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
}  // namespace

pact_status require_sms() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PACT_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PACT_ERR_UNSUPPORTED, "device index %d is not supported", dev);
    if (g_sms[dev].load(std::memory_order_acquire) > 0) return PACT_OK;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n <= 0)
        return fail(PACT_ERR_CUDA, "SM count query failed: %s", cudaGetErrorString(e));
    g_sms[dev].store(n, std::memory_order_release);
    return PACT_OK;
}

int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    const int n = g_sms[dev].load(std::memory_order_acquire);
    return n > 0 ? n : 1;    // entry points call require_sms() first, so 1 is never used
}

unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

pact_status ensure_smem(const void* fn, size_t bytes, const char* what) {
    if (bytes <= 48 * 1024) return PACT_OK;
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return check_launch(what);
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = done[std::make_pair(fn, dev)];
    if (cur >= bytes) return PACT_OK;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return check_launch(what);
    cur = bytes;
    return PACT_OK;
}

pact_status check_geometry(const pact_geometry* g) {
    if (!g) return fail(PACT_ERR_INVALID_ARG, "geometry is NULL");
    if (g->n_t < 4) return fail(PACT_ERR_INVALID_ARG, "n_t must be >= 4 (got %d)", g->n_t);
    if (g->n_t > 65536) return fail(PACT_ERR_SHAPE, "n_t must be <= 65536 (got %d)", g->n_t);
    if (!(g->ring_radius > 0.f)) return fail(PACT_ERR_INVALID_ARG, "ring_radius must be > 0");
    if (!(g->v0 > 0.f) || !(g->v_bg > 0.f)) return fail(PACT_ERR_INVALID_ARG, "v0 and v_bg must be > 0");
    if (g->img_h < 1 || g->img_w < 1) return fail(PACT_ERR_INVALID_ARG, "image size must be positive");
    if (!(g->dx > 0.f)) return fail(PACT_ERR_INVALID_ARG, "dx must be > 0");
    if (g->sos_g < 2 || g->sos_g > 512) return fail(PACT_ERR_SHAPE, "sos_g must be in [2, 512] (got %d)", g->sos_g);
    if (!(g->sos_dx > 0.f)) return fail(PACT_ERR_INVALID_ARG, "sos_dx must be > 0");
    if (!(g->mask_radius >= 0.f)) return fail(PACT_ERR_INVALID_ARG, "mask_radius must be >= 0");
    if (!(g->ray_step > 0.f)) return fail(PACT_ERR_INVALID_ARG, "ray_step must be > 0");
    return PACT_OK;
}

pact_status check_patches(const pact_patches* pt) {
    if (!pt) return fail(PACT_ERR_INVALID_ARG, "patches is NULL");
    if (pt->n < 1) return fail(PACT_ERR_INVALID_ARG, "patch count must be >= 1 (got %d)", pt->n);
    if (pt->n > 65535) return fail(PACT_ERR_SHAPE, "patch count must be <= 65535 (got %d)", pt->n);
    if (pt->p < 4 || pt->p > 128 || (pt->p & 1))
        return fail(PACT_ERR_SHAPE, "patch size must be even and in [4, 128] (got %d)", pt->p);
    if (!pt->centres) return fail(PACT_ERR_INVALID_ARG, "patch centres pointer is NULL");
    if (!(pt->window_fwhm > 0.f)) return fail(PACT_ERR_INVALID_ARG, "window_fwhm must be > 0");
    return PACT_OK;
}

}  // namespace pact

extern "C" const char* pact_version(void) { return "pact-gb300 0.1 (sm_103a)"; }

extern "C" const char* pact_last_error_message(void) { return g_msg; }

using namespace pact;

extern "C" pact_status pact_set_wait_limit_ns(unsigned long long ns) {
    if (ns == 0) ns = kDefaultWaitNs;
    if (ns < 100000ull || ns > 10000000000ull)
        return fail(PACT_ERR_INVALID_ARG, "wait limit must be 0 (default) or in [1e5, 1e10] ns (got %llu)", ns);
    g_wait_ns.store(ns, std::memory_order_relaxed);
    return PACT_OK;
}

extern "C" unsigned long long pact_get_wait_limit_ns(void) { return wait_limit_ns(); }
