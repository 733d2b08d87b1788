// Eq. 2-3 on the GPU: straight-ray wavefront errors (pact_sos_to_delays) and
// their adjoint to the pixel-grid SOS (pact_sos_to_delays_adj).
//
// A CTA owns a contiguous run of the rays r'_i -> r_n of one patch and stages
// the SOS excess dv_q = sos_q - v0 (exact in FP32 for SOS near v0) in shared
// memory; one warp integrates one ray at a time.  The part of the segment
// inside the mask disk is split into midpoint-rule samples of step h (the last
// partial step weighted by its length); lane l takes a contiguous run of
// samples, so the lanes of a warp touch different SOS nodes.  The integrand is
// the slowness excess (v - v0)/v = dv / (v0 + dv) with dv interpolated from
// the node excesses, so no 1/v - 1/v0 cancellation occurs.  Outside the mask
// the integrand is (v_bg - v0)/v_bg.
//
// The adjoint scatters dL/dw_{i,n} h_s v0 / v^2 times the bilinear weights
// into a per-CTA shared-memory copy of the SOS grid; each CTA writes its
// partial grid to the workspace and two small kernels sum the partials in a
// fixed order (deterministic).  Grids too large for shared memory read the SOS
// from global memory and scatter with global atomics instead.
#include <algorithm>

#include "pact_internal.cuh"

namespace pact {
namespace {

struct Ray {
    float cx, cy, ex, ey, L, s_in, chord, rem;
    int nfull, nsamp;
};

__device__ __forceinline__ Ray make_ray(const Geo& g, float2 c, int n) {
    Ray r;
    float sn, cs;
    // transducer angle 2 pi n / N_t + phase, as pi * (2 n / N_t + phase / pi)
    sincospif(2.f * ((float)n / (float)g.n_t) + g.phase * 0.318309886183790672f, &sn, &cs);
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

// Node-grid coordinates of sample m: fx = (x / sos_dx + (G-1)/2), same for y;
// returns the quadrature weight.
struct Walk {
    float ax, ay, bx, by;     // fractional node coords at s_in and per unit length
    float h;
};

__device__ __forceinline__ Walk make_walk(const Geo& g, const Ray& r) {
    const float inv = 1.f / g.sos_dx, half = 0.5f * (g.G - 1);
    Walk w;
    w.ax = fmaf(fmaf(r.s_in, r.ex, r.cx), inv, half);
    w.ay = fmaf(fmaf(r.s_in, r.ey, r.cy), inv, half);
    w.bx = r.ex * inv;
    w.by = r.ey * inv;
    w.h = g.h;
    return w;
}

__device__ __forceinline__ float sample_xy(const Walk& w, const Ray& r, int m, float& fx, float& fy) {
    float s, wgt;
    if (m < r.nfull) {
        s = (m + 0.5f) * w.h;
        wgt = w.h;
    } else {
        s = r.nfull * w.h + 0.5f * r.rem;
        wgt = r.rem;
    }
    fx = fmaf(s, w.bx, w.ax);
    fy = fmaf(s, w.by, w.ay);
    return wgt;
}

struct Bil {
    int idx;
    float tx, ty;
};

__device__ __forceinline__ Bil bil(int G, float fx, float fy) {
    fx = fminf(fmaxf(fx, 0.f), (float)(G - 1));
    fy = fminf(fmaxf(fy, 0.f), (float)(G - 1));
    const int ix = min((int)fx, G - 2);
    const int iy = min((int)fy, G - 2);
    Bil b;
    b.idx = iy * G + ix;
    b.tx = fx - ix;
    b.ty = fy - iy;
    return b;
}

__device__ __forceinline__ float interp(const float* dv, int G, const Bil& b) {
    const float d00 = dv[b.idx], d01 = dv[b.idx + 1], d10 = dv[b.idx + G], d11 = dv[b.idx + G + 1];
    const float top = fmaf(b.tx, d01 - d00, d00), bot = fmaf(b.tx, d11 - d10, d10);
    return fmaf(b.ty, bot - top, top);
}

struct RayArgs {
    Geo g;
    int N;
    const int2* centres;
    const float* sos;
    float* w;             // forward output
    const float* dLdw;    // adjoint input
    float* part;          // adjoint partial grids [gridDim.x][G*G] (smem variant)
    float* out;           // adjoint output (global-atomic variant)
    int splits;           // CTAs per patch
    int use_smem;
};

// CTA b handles patch b / splits, rays [n0, n1) of it.
__device__ __forceinline__ void cta_rays(const RayArgs& a, int& i, int& n0, int& n1) {
    i = blockIdx.x / a.splits;
    const int s = blockIdx.x - i * a.splits;
    const int per = (a.g.n_t + a.splits - 1) / a.splits;
    n0 = s * per;
    n1 = min(a.g.n_t, n0 + per);
}

__global__ void __launch_bounds__(1024) rays_fwd_kernel(const RayArgs a) {
    extern __shared__ float dv_s[];
    const int G = a.g.G, GG = G * G;
    const float v0 = a.g.v0;
    const float* dv = a.sos;
    if (a.use_smem) {
        for (int q = threadIdx.x; q < GG; q += blockDim.x) dv_s[q] = a.sos[q] - v0;
        __syncthreads();
        dv = dv_s;
    }
    int i, n0, n1;
    cta_rays(a, i, n0, n1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int2 cc = a.centres[i];
    const float2 c = pixel_xy(a.g, cc.x, cc.y);
    const float out_coef = (a.g.v_bg - v0) / a.g.v_bg;
    for (int n = n0 + warp; n < n1; n += nw) {
        const Ray r = make_ray(a.g, c, n);
        const Walk wk = make_walk(a.g, r);
        const int per = (r.nsamp + 31) >> 5;
        const int m0 = lane * per, m1 = min(r.nsamp, m0 + per);
        float acc = 0.f;
        for (int m = m0; m < m1; ++m) {
            float fx, fy;
            const float wgt = sample_xy(wk, r, m, fx, fy);
            const Bil b = bil(G, fx, fy);
            float d;
            if (a.use_smem) {
                d = interp(dv, G, b);
            } else {
                const float d00 = __ldg(a.sos + b.idx) - v0, d01 = __ldg(a.sos + b.idx + 1) - v0;
                const float d10 = __ldg(a.sos + b.idx + G) - v0, d11 = __ldg(a.sos + b.idx + G + 1) - v0;
                const float top = fmaf(b.tx, d01 - d00, d00), bot = fmaf(b.tx, d11 - d10, d10);
                d = fmaf(b.ty, bot - top, top);
            }
            acc = fmaf(wgt, __fdividef(d, v0 + d), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) a.w[(size_t)i * a.g.n_t + n] = fmaf(r.L - r.chord, out_coef, acc);
    }
}

__global__ void __launch_bounds__(1024) rays_adj_kernel(const RayArgs a) {
    extern __shared__ float sm[];
    const int G = a.g.G, GG = G * G;
    const float v0 = a.g.v0;
    float* dv_s = sm;
    float* acc_s = sm + GG;
    if (a.use_smem) {
        for (int q = threadIdx.x; q < GG; q += blockDim.x) {
            dv_s[q] = a.sos[q] - v0;
            acc_s[q] = 0.f;
        }
        __syncthreads();
    }
    float* acc = a.use_smem ? acc_s : a.out;
    int i, n0, n1;
    cta_rays(a, i, n0, n1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int2 cc = a.centres[i];
    const float2 c = pixel_xy(a.g, cc.x, cc.y);
    for (int n = n0 + warp; n < n1; n += nw) {
        const float gr = a.dLdw[(size_t)i * a.g.n_t + n];
        if (gr == 0.f) continue;
        const Ray r = make_ray(a.g, c, n);
        const Walk wk = make_walk(a.g, r);
        const int per = (r.nsamp + 31) >> 5;
        const int m0 = lane * per, m1 = min(r.nsamp, m0 + per);
        const float gv0 = gr * v0;
        for (int m = m0; m < m1; ++m) {
            float fx, fy;
            const float wgt = sample_xy(wk, r, m, fx, fy);
            const Bil b = bil(G, fx, fy);
            float d;
            if (a.use_smem) {
                d = interp(dv_s, G, b);
            } else {
                const float d00 = __ldg(a.sos + b.idx) - v0, d01 = __ldg(a.sos + b.idx + 1) - v0;
                const float d10 = __ldg(a.sos + b.idx + G) - v0, d11 = __ldg(a.sos + b.idx + G + 1) - v0;
                const float top = fmaf(b.tx, d01 - d00, d00), bot = fmaf(b.tx, d11 - d10, d10);
                d = fmaf(b.ty, bot - top, top);
            }
            const float iv = __frcp_rn(v0 + d);
            const float coef = gv0 * wgt * iv * iv;
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
        for (int q = threadIdx.x; q < GG; q += blockDim.x) dst[q] = acc_s[q];
    }
}

constexpr int kGroup = 16;   // partials summed per thread in the first reduction stage

// stage 1: stage1[r][q] = sum of partials r*kGroup .. r*kGroup + kGroup - 1 at node q
__global__ void reduce_stage1_kernel(const float* part, int nb, int GG, float* stage1) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (q >= GG) return;
    const int b0 = r * kGroup;
    float s[kGroup];
#pragma unroll
    for (int k = 0; k < kGroup; ++k) s[k] = (b0 + k < nb) ? part[(size_t)(b0 + k) * GG + q] : 0.f;
#pragma unroll
    for (int k = kGroup / 2; k > 0; k >>= 1)
#pragma unroll
        for (int t = 0; t < k; ++t) s[t] += s[t + k];
    stage1[(size_t)r * GG + q] = s[0];
}

__global__ void reduce_stage2_kernel(const float* stage1, int nr, int GG, float* out, int accumulate) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= GG) return;
    float s = 0.f;
    for (int r = 0; r < nr; ++r) s += stage1[(size_t)r * GG + q];
    out[q] = accumulate ? out[q] + s : s;
}

constexpr size_t kMaxSmem = 200 * 1024;

struct Plan {
    int splits_fwd, splits_adj, nb_fwd, nb_adj, nr, use_smem, threads;
    size_t smem_fwd, smem_adj, off_stage1, ws;
};

// CTAs per patch so that the grid fills the SMs once at the occupancy the
// shared-memory footprint allows (at least 64 rays per CTA).
int splits_for(const pact_geometry* g, const pact_patches* pt, size_t smem, int threads) {
    const int sms = num_sms();
    int per_sm = std::max(1, 2048 / threads);
    if (smem > 0) per_sm = std::min(per_sm, std::max(1, (int)((227 * 1024) / (smem + 1024))));
    int s = (sms * per_sm) / pt->n;
    return std::max(1, std::min(s, std::max(1, g->n_t / 64)));
}

Plan make_plan(const pact_geometry* g, const pact_patches* pt) {
    Plan p;
    const size_t gbytes = (size_t)g->sos_g * g->sos_g * sizeof(float);
    p.use_smem = 2 * gbytes <= kMaxSmem;
    p.threads = 1024;
    p.smem_fwd = p.use_smem ? gbytes : 0;
    p.smem_adj = p.use_smem ? 2 * gbytes : 0;
    p.splits_fwd = splits_for(g, pt, p.smem_fwd, p.threads);
    p.splits_adj = splits_for(g, pt, p.smem_adj, p.threads);
    p.nb_fwd = pt->n * p.splits_fwd;
    p.nb_adj = pt->n * p.splits_adj;
    p.nr = (p.nb_adj + kGroup - 1) / kGroup;
    p.off_stage1 = align_up((size_t)p.nb_adj * gbytes, 256);
    p.ws = p.use_smem ? p.off_stage1 + align_up((size_t)p.nr * gbytes, 256) : 256;
    return p;
}

RayArgs make_args(const pact_geometry* g, const pact_patches* pt, const Plan& pl, int splits, const float* sos) {
    RayArgs a;
    a.g = make_geo(g);
    a.N = pt->n;
    a.centres = reinterpret_cast<const int2*>(pt->centres);
    a.sos = sos;
    a.w = nullptr;
    a.dLdw = nullptr;
    a.part = nullptr;
    a.out = nullptr;
    a.splits = splits;
    a.use_smem = pl.use_smem;
    return a;
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" pact_status pact_sos_to_delays(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                          float* w, void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!sos || !w) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays: sos and w must not be NULL");
    const Plan pl = make_plan(g, pt);
    RayArgs a = make_args(g, pt, pl, pl.splits_fwd, sos);
    a.w = w;
    PACT_TRY(ensure_smem((const void*)rays_fwd_kernel, pl.smem_fwd, "sos_to_delays: shared memory attribute"));
    rays_fwd_kernel<<<pl.nb_fwd, pl.threads, pl.smem_fwd, as_stream(stream)>>>(a);
    return check_launch("sos_to_delays kernel");
}

extern "C" size_t pact_sos_to_delays_adj_workspace_size(const pact_geometry* g, const pact_patches* pt) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK) return 0;
    return make_plan(g, pt).ws;
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
    const Plan pl = make_plan(g, pt);
    if (ws_bytes < pl.ws) return fail(PACT_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, pl.ws);
    cudaStream_t st = as_stream(stream);
    const int GG = g->sos_g * g->sos_g;
    RayArgs a = make_args(g, pt, pl, pl.splits_adj, sos);
    a.dLdw = dL_dw;
    a.part = static_cast<float*>(ws);
    a.out = dL_dsos;
    if (pl.use_smem) {
        PACT_TRY(ensure_smem((const void*)rays_adj_kernel, pl.smem_adj, "sos_to_delays_adj: shared memory attribute"));
        rays_adj_kernel<<<pl.nb_adj, pl.threads, pl.smem_adj, st>>>(a);
        PACT_TRY(check_launch("sos_to_delays_adj kernel"));
        float* stage1 = reinterpret_cast<float*>(static_cast<char*>(ws) + pl.off_stage1);
        dim3 g1((GG + 255) / 256, pl.nr);
        reduce_stage1_kernel<<<g1, 256, 0, st>>>(a.part, pl.nb_adj, GG, stage1);
        PACT_TRY(check_launch("sos_to_delays_adj reduction (1)"));
        reduce_stage2_kernel<<<(GG + 255) / 256, 256, 0, st>>>(stage1, pl.nr, GG, dL_dsos, accumulate);
        return check_launch("sos_to_delays_adj reduction (2)");
    }
    if (!accumulate && cudaMemsetAsync(dL_dsos, 0, (size_t)GG * sizeof(float), st) != cudaSuccess)
        return check_launch("sos_to_delays_adj: memset");
    rays_adj_kernel<<<pl.nb_adj, pl.threads, 0, st>>>(a);
    return check_launch("sos_to_delays_adj kernel");
}
