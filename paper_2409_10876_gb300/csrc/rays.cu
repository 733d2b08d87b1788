// Eq. 2-3 on the GPU: straight-ray wavefront errors (pact_sos_to_delays) and
// their adjoint to the pixel-grid SOS (pact_sos_to_delays_adj).
//
// One warp integrates one ray r'_i -> r_n.  The part of the segment inside the
// mask disk is split into midpoint-rule samples of step h (the last partial
// step weighted by its length); lane l takes a contiguous run of samples so
// that the lanes of a warp touch different SOS nodes.  The integrand is the
// slowness excess (v - v0)/v = dv / (v0 + dv) with dv interpolated from the
// node excesses sos - v0 (exact in FP32 for SOS near v0), so no 1/v - 1/v0
// cancellation occurs.  Outside the mask the integrand is (v_bg - v0)/v_bg.
//
// The adjoint scatters dL/dw_{i,n} h_s v0 / v^2 with the bilinear weights
// into a per-CTA shared-memory copy of the SOS grid; each CTA writes its
// partial grid to the workspace and a second kernel sums the partials in a
// fixed order (deterministic).  Grids too large for shared memory scatter
// with global atomics instead.
#include <algorithm>

#include "pact_internal.cuh"

namespace pact {
namespace {

constexpr float kTwoPi = 6.283185307179586f;

struct Ray {
    float cx, cy, ex, ey, L, s_in, chord, rem;
    int nfull, nsamp;
};

__device__ __forceinline__ Ray make_ray(const Geo& g, float2 c, int n) {
    Ray r;
    float sn, cs;
    sincosf(kTwoPi * ((float)n / (float)g.n_t) + g.phase, &sn, &cs);
    const float dx = g.R * cs - c.x, dy = g.R * sn - c.y;
    r.L = sqrtf(dx * dx + dy * dy);
    r.ex = dx / r.L;
    r.ey = dy / r.L;
    r.cx = c.x;
    r.cy = c.y;
    const float ce = c.x * r.ex + c.y * r.ey;
    const float disc = ce * ce - (c.x * c.x + c.y * c.y - g.mask_r * g.mask_r);
    r.s_in = 0.f;
    r.chord = 0.f;
    if (disc > 0.f) {
        const float sq = sqrtf(disc);
        const float s0 = fminf(fmaxf(-ce - sq, 0.f), r.L);
        const float s1 = fminf(fmaxf(-ce + sq, 0.f), r.L);
        r.s_in = s0;
        r.chord = fmaxf(s1 - s0, 0.f);
    }
    r.nfull = (int)floorf(r.chord / g.h);
    r.rem = fmaxf(r.chord - r.nfull * g.h, 0.f);
    r.nsamp = r.nfull + (r.rem > 0.f ? 1 : 0);
    return r;
}

struct Bil {
    int idx;        // node (iy, ix) flattened
    float tx, ty;
};

__device__ __forceinline__ Bil bil_at(const Geo& g, float px, float py) {
    const float half = 0.5f * (g.G - 1);
    float fx = fminf(fmaxf(px / g.sos_dx + half, 0.f), (float)(g.G - 1));
    float fy = fminf(fmaxf(py / g.sos_dx + half, 0.f), (float)(g.G - 1));
    const int ix = min((int)fx, g.G - 2);
    const int iy = min((int)fy, g.G - 2);
    Bil b;
    b.idx = iy * g.G + ix;
    b.tx = fx - ix;
    b.ty = fy - iy;
    return b;
}

// sample m of a ray: position along it and quadrature weight
__device__ __forceinline__ void sample_at(const Ray& r, float h, int m, float& s, float& wgt) {
    if (m < r.nfull) {
        s = r.s_in + (m + 0.5f) * h;
        wgt = h;
    } else {
        s = r.s_in + r.nfull * h + 0.5f * r.rem;
        wgt = r.rem;
    }
}

struct FwdArgs {
    Geo g;
    int N;
    const int2* centres;
    const float* sos;
    float* w;
};

__global__ void __launch_bounds__(256) rays_fwd_kernel(const FwdArgs a) {
    const int ray = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ray >= a.N * a.g.n_t) return;
    const int i = ray / a.g.n_t, n = ray - i * a.g.n_t;
    const int2 cc = a.centres[i];
    const Ray r = make_ray(a.g, pixel_xy(a.g, cc.x, cc.y), n);
    const int per = (r.nsamp + 31) >> 5;
    const int m0 = lane * per, m1 = min(r.nsamp, m0 + per);
    const int G = a.g.G;
    const float v0 = a.g.v0;
    float acc = 0.f;
    for (int m = m0; m < m1; ++m) {
        float s, wgt;
        sample_at(r, a.g.h, m, s, wgt);
        const Bil b = bil_at(a.g, fmaf(s, r.ex, r.cx), fmaf(s, r.ey, r.cy));
        const float d00 = __ldg(a.sos + b.idx) - v0, d01 = __ldg(a.sos + b.idx + 1) - v0;
        const float d10 = __ldg(a.sos + b.idx + G) - v0, d11 = __ldg(a.sos + b.idx + G + 1) - v0;
        const float top = fmaf(b.tx, d01 - d00, d00), bot = fmaf(b.tx, d11 - d10, d10);
        const float dv = fmaf(b.ty, bot - top, top);
        acc = fmaf(wgt, dv / (v0 + dv), acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) a.w[ray] = acc + (r.L - r.chord) * ((a.g.v_bg - v0) / a.g.v_bg);
}

struct AdjArgs {
    Geo g;
    int N;
    const int2* centres;
    const float* sos;
    const float* dLdw;
    float* part;          // [nblocks][G*G] (shared-memory variant)
    float* out;           // [G*G] (global-atomic variant)
    int rays_per_block;
    int use_smem;
};

__global__ void __launch_bounds__(512) rays_adj_kernel(const AdjArgs a) {
    extern __shared__ float grid_s[];
    const int G = a.g.G;
    const int GG = G * G;
    if (a.use_smem) {
        for (int q = threadIdx.x; q < GG; q += blockDim.x) grid_s[q] = 0.f;
        __syncthreads();
    }
    float* acc = a.use_smem ? grid_s : a.out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nrays = a.N * a.g.n_t;
    const int r0 = blockIdx.x * a.rays_per_block;
    const int r1 = min(nrays, r0 + a.rays_per_block);
    const float v0 = a.g.v0;
    for (int ray = r0 + warp; ray < r1; ray += nw) {
        const float gr = a.dLdw[ray];
        if (gr == 0.f) continue;
        const int i = ray / a.g.n_t, n = ray - i * a.g.n_t;
        const int2 cc = a.centres[i];
        const Ray r = make_ray(a.g, pixel_xy(a.g, cc.x, cc.y), n);
        const int per = (r.nsamp + 31) >> 5;
        const int m0 = lane * per, m1 = min(r.nsamp, m0 + per);
        for (int m = m0; m < m1; ++m) {
            float s, wgt;
            sample_at(r, a.g.h, m, s, wgt);
            const Bil b = bil_at(a.g, fmaf(s, r.ex, r.cx), fmaf(s, r.ey, r.cy));
            const float d00 = __ldg(a.sos + b.idx) - v0, d01 = __ldg(a.sos + b.idx + 1) - v0;
            const float d10 = __ldg(a.sos + b.idx + G) - v0, d11 = __ldg(a.sos + b.idx + G + 1) - v0;
            const float top = fmaf(b.tx, d01 - d00, d00), bot = fmaf(b.tx, d11 - d10, d10);
            const float v = v0 + fmaf(b.ty, bot - top, top);
            const float coef = gr * wgt * v0 / (v * v);
            const float cy0 = coef * (1.f - b.ty), cy1 = coef * b.ty;
            atomicAdd(acc + b.idx, cy0 * (1.f - b.tx));
            atomicAdd(acc + b.idx + 1, cy0 * b.tx);
            atomicAdd(acc + b.idx + G, cy1 * (1.f - b.tx));
            atomicAdd(acc + b.idx + G + 1, cy1 * b.tx);
        }
    }
    if (a.use_smem) {
        __syncthreads();
        float* dst = a.part + (size_t)blockIdx.x * GG;
        for (int q = threadIdx.x; q < GG; q += blockDim.x) dst[q] = grid_s[q];
    }
}

__global__ void partial_sum_kernel(const float* part, int nb, int GG, float* out, int accumulate) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= GG) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * GG + q];
    out[q] = accumulate ? out[q] + s : s;
}

struct AdjPlan {
    int nb, rpb, use_smem;
    size_t smem, ws;
};

constexpr size_t kMaxGridSmem = 160 * 1024;

AdjPlan adj_plan(const pact_geometry* g, const pact_patches* pt) {
    AdjPlan p;
    const int nrays = pt->n * g->n_t;
    const size_t gbytes = (size_t)g->sos_g * g->sos_g * sizeof(float);
    p.use_smem = gbytes <= kMaxGridSmem;
    const int sms = num_sms();
    int nb = std::min((nrays + 63) / 64, (p.use_smem ? 2 : 8) * sms);
    nb = std::max(nb, 1);
    p.rpb = (nrays + nb - 1) / nb;
    p.nb = (nrays + p.rpb - 1) / p.rpb;
    p.smem = p.use_smem ? gbytes : 0;
    p.ws = p.use_smem ? align_up((size_t)p.nb * gbytes, 256) : 256;
    return p;
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" pact_status pact_sos_to_delays(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                          float* w, void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!sos || !w) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays: sos and w must not be NULL");
    FwdArgs a;
    a.g = make_geo(g);
    a.N = pt->n;
    a.centres = reinterpret_cast<const int2*>(pt->centres);
    a.sos = sos;
    a.w = w;
    const long long threads = (long long)pt->n * g->n_t * 32;
    rays_fwd_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, as_stream(stream)>>>(a);
    return check_launch("sos_to_delays kernel");
}

extern "C" size_t pact_sos_to_delays_adj_workspace_size(const pact_geometry* g, const pact_patches* pt) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK) return 0;
    return adj_plan(g, pt).ws;
}

extern "C" pact_status pact_sos_to_delays_adj(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                              const float* dL_dw, float* dL_dsos, int accumulate, void* ws,
                                              size_t ws_bytes, void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!sos || !dL_dw || !dL_dsos)
        return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj: sos, dL_dw and dL_dsos must not be NULL");
    if (!ws) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj: workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const AdjPlan pl = adj_plan(g, pt);
    if (ws_bytes < pl.ws) return fail(PACT_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, pl.ws);
    cudaStream_t st = as_stream(stream);
    const int GG = g->sos_g * g->sos_g;
    AdjArgs a;
    a.g = make_geo(g);
    a.N = pt->n;
    a.centres = reinterpret_cast<const int2*>(pt->centres);
    a.sos = sos;
    a.dLdw = dL_dw;
    a.part = static_cast<float*>(ws);
    a.out = dL_dsos;
    a.rays_per_block = pl.rpb;
    a.use_smem = pl.use_smem;
    if (pl.use_smem) {
        PACT_TRY(ensure_smem((const void*)rays_adj_kernel, pl.smem, "sos_to_delays_adj: shared memory attribute"));
        rays_adj_kernel<<<pl.nb, 512, pl.smem, st>>>(a);
        PACT_TRY(check_launch("sos_to_delays_adj kernel"));
        partial_sum_kernel<<<(GG + 255) / 256, 256, 0, st>>>(a.part, pl.nb, GG, dL_dsos, accumulate);
        return check_launch("sos_to_delays_adj reduction");
    }
    if (!accumulate && cudaMemsetAsync(dL_dsos, 0, (size_t)GG * sizeof(float), st) != cudaSuccess)
        return check_launch("sos_to_delays_adj: memset");
    rays_adj_kernel<<<pl.nb, 512, 0, st>>>(a);
    return check_launch("sos_to_delays_adj kernel");
}
