// Internal helpers shared by the CUDA translation units of libpact.
// Nothing here is part of the C ABI (see include/pact.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "pact.h"

namespace pact {

// ---------------------------------------------------------------- host side

// Records a thread-local error message and returns `s`.
pact_status fail(pact_status s, const char* fmt, ...);
// Maps a pending launch error (cudaGetLastError) to PACT_ERR_CUDA.
pact_status check_launch(const char* what);
// Queries (once per device) and caches the SM count of the current device;
// PACT_ERR_CUDA if the query fails.  Every entry point that sizes a grid
// from num_sms() calls this first.
pact_status require_sms();
// SM count of the current device from the cache filled by require_sms().
int num_sms();
// Bound on every device-side wait of a launch, in ns (pact_set_wait_limit_ns).
unsigned long long wait_limit_ns();
// Raises the dynamic shared-memory limit of kernel `fn` on the current device
// to at least `bytes` (cached: the attribute call happens once per kernel and
// device, so later launches, e.g. under CUDA-graph capture, make no calls).
pact_status ensure_smem(const void* fn, size_t bytes, const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Validates the geometry struct; returns PACT_OK or records the failure.
pact_status check_geometry(const pact_geometry* g);
pact_status check_patches(const pact_patches* pt);

// Eq. 3 wavefront errors from the image pixels pix0 .. pix0 + npix - 1 with
// p0 != 0 to every transducer of g (rays.cu), written transposed:
// wT[n * ld + (pix - pix0)]; entries of pixels with p0 == 0 are not written.
pact_status launch_pixel_rays(const pact_geometry* g, const float* sos, const float* p0, int pix0, int npix,
                              float* wT, int ld, cudaStream_t st);

// Programmatic dependent launch (PDL).  A kernel launched by launch_pdl may be
// scheduled before its predecessor in the stream has finished (once every CTA
// of the predecessor has called pdl_trigger or exited); it must call pdl_wait
// before it reads or writes anything a kernel launched before it may still
// touch.  Work before pdl_wait may only use inputs no kernel writes
// (geometry, patch centres, constant tables) and the kernel's own shared
// memory.  Without a PDL launch both calls are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#define PACT_TRY(expr)                       \
    do {                                     \
        pact_status _s = (expr);             \
        if (_s != PACT_OK) return _s;        \
    } while (0)

// Kernel-argument copy of the geometry (by value).
struct Geo {
    int n_t;
    float R, phase, v0, v_bg;
    int H, W;
    float dx;
    int G;
    float sos_dx, mask_r, h;
    float inv_h;        // 1 / h
};

inline Geo make_geo(const pact_geometry* g) {
    Geo o;
    o.n_t = g->n_t;
    o.R = g->ring_radius;
    o.phase = g->ring_phase;
    o.v0 = g->v0;
    o.v_bg = g->v_bg;
    o.H = g->img_h;
    o.W = g->img_w;
    o.dx = g->dx;
    o.G = g->sos_g;
    o.sos_dx = g->sos_dx;
    o.mask_r = g->mask_radius;
    o.h = g->ray_step;
    o.inv_h = 1.f / g->ray_step;
    return o;
}

// Delay list by value (HOST array copied into kernel arguments).
struct Delays {
    float d[PACT_MAX_CHANNELS];
    int m;
};

inline Delays make_delays(const float* d, int m) {
    Delays o;
    o.m = m;
    for (int j = 0; j < PACT_MAX_CHANNELS; ++j) o.d[j] = j < m ? d[j] : 0.f;
    return o;
}

// ---------------------------------------------------------------- device side

// Position of pixel (row, col): x along columns, y along rows.
__device__ __forceinline__ float2 pixel_xy(const Geo& g, int row, int col) {
    return make_float2((col - 0.5f * (g.W - 1)) * g.dx, (row - 0.5f * (g.H - 1)) * g.dx);
}

// Spatial frequency of half-spectrum bin k of a P x P patch, in cycles/m
// (rows in fftfreq order).  Sets u, v.
__device__ __forceinline__ float2 bin_freq(int k, int P, float inv_pdx, int& u, int& v) {
    const int half = P / 2 + 1;
    u = k / half;
    v = k - u * half;
    const int us = u < P / 2 ? u : u - P;
    return make_float2(v * inv_pdx, us * inv_pdx);
}

// Ring lookup: the ray from c in direction (ex, ey) meets the ring at ring
// angle alpha; returns the left transducer n1 and the fraction f in
// [0, 1) of the way to n1 + 1 (cyclic).  `disc_sq` = sqrt((c.e)^2 - |c|^2 + R^2).
__device__ __forceinline__ void ring_hit(float cx, float cy, float ex, float ey, float s,
                                         float phase, int n_t, float n_over_2pi, int& n1,
                                         float& f) {
    const float px = fmaf(s, ex, cx);
    const float py = fmaf(s, ey, cy);
    float t = (atan2f(py, px) - phase) * n_over_2pi;
    t -= floorf(t / (float)n_t) * (float)n_t;
    const float fl = floorf(t);
    f = t - fl;
    int n = (int)fl;
    n %= n_t;
    if (n < 0) n += n_t;
    n1 = n;
}

// Both ring hits of the line through c with direction e: +e and -e.
struct Hits {
    int n1a, n1b;
    float fa, fb;
};

__device__ __forceinline__ Hits ring_hits(float cx, float cy, float ex, float ey, const Geo& g,
                                          float n_over_2pi) {
    const float ce = cx * ex + cy * ey;
    const float disc = fmaxf(ce * ce - (cx * cx + cy * cy) + g.R * g.R, 0.f);
    const float sq = sqrtf(disc);
    Hits o;
    ring_hit(cx, cy, ex, ey, sq - ce, g.phase, g.n_t, n_over_2pi, o.n1a, o.fa);
    ring_hit(cx, cy, -ex, -ey, sq + ce, g.phase, g.n_t, n_over_2pi, o.n1b, o.fb);
    return o;
}

// Complex helpers (float2 = re, im).
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) * b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cis_pi(float x) {  // exp(j pi x)
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Adds v to dst[idx] (shared memory) for every lane of a converged warp with one
// atomic per run of consecutive lanes holding the same idx: the run's values
// are summed by a segmented shuffle scan and the run's last lane adds the sum.
// (Shared-memory float atomics are compare-and-swap loops, which neighbouring
// lanes aiming at one address would serialise.)
__device__ __forceinline__ void warp_seg_add(float* dst, int idx, float v) {
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, idx, 1);
    const int next = __shfl_down_sync(0xffffffffu, idx, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != idx);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));   // head of this lane's run
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float x = __shfl_up_sync(0xffffffffu, v, d);
        if (lane - d >= start) v += x;
    }
    if (lane == 31 || next != idx) atomicAdd(dst + idx, v);
}

// Block-wide sum (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ float block_sum(float x, float* red) {
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = x;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    x = threadIdx.x < nw ? red[threadIdx.x] : 0.f;
    if (wid == 0) x = warp_sum(x);
    __syncthreads();
    return x;
}

// ---------------------------------------------------------------- TMA bulk copies, mbarriers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised mbarriers visible to the async proxy (TMA).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before its
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier `id` that completes when `count` threads (a multiple of 32)
// have arrived; returns the AND of their `pred`.
__device__ __forceinline__ bool bar_and(int id, int count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completing `bytes` of transaction on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Asks the L2 to fetch [p, p + bytes) (16-byte aligned, bytes a multiple of
// 16).  A hint: no data reaches the thread, so it may be issued before the
// kernels that write that memory have finished (the L2 is the point of
// coherence; the reads that use the data come after pdl_wait).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the global counter *p reaches `target` (acquire: what the
// counting threads wrote before their fenced increments is then visible),
// giving up after `limit_ns` (returns false then).
__device__ __forceinline__ bool counter_wait_bounded(const int* p, int target, uint64_t limit_ns) {
    auto load = [p]() {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    };
    if (load() >= target) return true;
    const uint64_t t0 = global_ns();
    while (load() < target) {
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    return true;
}

// Waits for phase `parity` of `bar` to complete, giving up after `limit_ns`
// (returns false then; the caller reports the failure instead of hanging).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

}  // namespace pact
