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
#include <cooperative_groups.h>

#include <algorithm>

#include "pact_internal.cuh"

namespace pact {
namespace {

struct Ray {
    float ax, ay, bx, by;   // fractional node coords at the mask entry and per metre along the ray
    float L, chord, rem;
    int nfull;
};

// Ray r'_i -> r_n clipped to the mask disk, in node-grid coordinates
// fx = x / sos_dx + (G-1)/2 (same for y).
__device__ __forceinline__ Ray make_ray(const Geo& g, float2 c, int n) {
    Ray r;
    float sn, cs;
    // transducer angle 2 pi n / N_t + phase, as pi * (2 n / N_t + phase / pi)
    sincospif(2.f * ((float)n / (float)g.n_t) + g.phase * 0.318309886183790672f, &sn, &cs);
    const float dx = g.R * cs - c.x, dy = g.R * sn - c.y;
    r.L = sqrtf(dx * dx + dy * dy);
    const float ex = dx / r.L, ey = dy / r.L;
    const float ce = c.x * ex + c.y * ey;
    const float disc = ce * ce - (c.x * c.x + c.y * c.y - g.mask_r * g.mask_r);
    float s_in = 0.f;
    r.chord = 0.f;
    if (disc > 0.f) {
        const float sq = sqrtf(disc);
        const float s0 = fminf(fmaxf(-ce - sq, 0.f), r.L);
        const float s1 = fminf(fmaxf(-ce + sq, 0.f), r.L);
        s_in = s0;
        r.chord = fmaxf(s1 - s0, 0.f);
    }
    r.nfull = (int)floorf(r.chord / g.h);
    r.rem = fmaxf(r.chord - r.nfull * g.h, 0.f);
    const float inv = 1.f / g.sos_dx, half = 0.5f * (g.G - 1);
    r.ax = fmaf(fmaf(s_in, ex, c.x), inv, half);
    r.ay = fmaf(fmaf(s_in, ey, c.y), inv, half);
    r.bx = ex * inv;
    r.by = ey * inv;
    return r;
}

// Broadcast lane `src`'s ray to the whole warp.
__device__ __forceinline__ Ray shfl_ray(const Ray& r, int src) {
    Ray o;
    o.ax = __shfl_sync(0xffffffffu, r.ax, src);
    o.ay = __shfl_sync(0xffffffffu, r.ay, src);
    o.bx = __shfl_sync(0xffffffffu, r.bx, src);
    o.by = __shfl_sync(0xffffffffu, r.by, src);
    o.L = __shfl_sync(0xffffffffu, r.L, src);
    o.chord = __shfl_sync(0xffffffffu, r.chord, src);
    o.rem = __shfl_sync(0xffffffffu, r.rem, src);
    o.nfull = __shfl_sync(0xffffffffu, r.nfull, src);
    return o;
}

struct Bil {
    int idx;        // node (iy, ix) in the grid of row pitch `pitch`
    float tx, ty;
};

__device__ __forceinline__ Bil bil(int G, int pitch, float fx, float fy) {
    fx = fminf(fmaxf(fx, 0.f), (float)(G - 1));
    fy = fminf(fmaxf(fy, 0.f), (float)(G - 1));
    const int ix = min((int)fx, G - 2);
    const int iy = min((int)fy, G - 2);
    Bil b;
    b.idx = iy * pitch + ix;
    b.tx = fx - ix;
    b.ty = fy - iy;
    return b;
}

__device__ __forceinline__ float interp(const float* dv, int pitch, const Bil& b) {
    const float d00 = dv[b.idx], d01 = dv[b.idx + 1], d10 = dv[b.idx + pitch], d11 = dv[b.idx + pitch + 1];
    const float top = fmaf(b.tx, d01 - d00, d00), bot = fmaf(b.tx, d11 - d10, d10);
    return fmaf(b.ty, bot - top, top);
}

__device__ __forceinline__ float interp_global(const float* sos, int G, float v0, const Bil& b) {
    const float d00 = __ldg(sos + b.idx) - v0, d01 = __ldg(sos + b.idx + 1) - v0;
    const float d10 = __ldg(sos + b.idx + G) - v0, d11 = __ldg(sos + b.idx + G + 1) - v0;
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
    int cluster;          // adjoint: CTAs per thread-block cluster that pool their grids (0: none)
};

// CTA b handles patch b / splits, rays [n0, n1) of it.
__device__ __forceinline__ void cta_rays(const RayArgs& a, int& i, int& n0, int& n1) {
    i = blockIdx.x / a.splits;
    const int s = blockIdx.x - i * a.splits;
    const int per = (a.g.n_t + a.splits - 1) / a.splits;
    n0 = s * per;
    n1 = min(a.g.n_t, n0 + per);
}

// Shared-memory grid pitch: one extra column so that nodes of one grid column
// fall into different banks.
__host__ __device__ __forceinline__ int smem_pitch(int G) { return G + 1; }

// dv[p][c] = sos[p][c] - v0 into the padded shared grid, with 16-byte loads
// (several in flight per thread) when the layout allows.
__device__ __forceinline__ void load_excess(float* dv, const float* sos, int G, int pitch, float v0) {
    if ((G & 3) == 0 && (reinterpret_cast<uintptr_t>(sos) & 15) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(sos);
        const int G4 = G >> 2, n4 = G * G4;
#pragma unroll 4
        for (int q = threadIdx.x; q < n4; q += blockDim.x) {
            const float4 v = __ldg(s4 + q);
            const int p = q / G4, c = (q - (q / G4) * G4) << 2;
            float* d = dv + p * pitch + c;
            d[0] = v.x - v0;
            d[1] = v.y - v0;
            d[2] = v.z - v0;
            d[3] = v.w - v0;
        }
    } else {
        for (int q = threadIdx.x; q < G * G; q += blockDim.x) {
            const int p = q / G, c = q - (q / G) * G;
            dv[p * pitch + c] = sos[q] - v0;
        }
    }
}

// Warp `warp` of `nw` integrates the rays r'_c -> r_n, n = n0 + warp, n0 + warp
// + nw, ... < n1 (neighbouring rays have similar lengths, so striding balances
// the warps): it sets up 32 of its rays at once (one per lane) and then
// integrates them one after the other (lanes over samples), taking each ray's
// setup by shuffles; out(n, w) runs on the lane that owns ray n.
// SMEM: the SOS excess grid dv is staged in shared memory (else read from global).
template <bool SMEM, class Out>
__device__ __forceinline__ void warp_rays(const RayArgs& a, const float* dv, int pitch, float2 c, int n0, int n1,
                                          int warp, int nw, Out out) {
    const int G = a.g.G, lane = threadIdx.x & 31;
    const float v0 = a.g.v0;
    const float out_coef = (a.g.v_bg - v0) / a.g.v_bg;
    const float h = a.g.h;
    const int nmine = n1 - n0 > warp ? (n1 - n0 - warp + nw - 1) / nw : 0;
    for (int kb = 0; kb < nmine; kb += 32) {
        const int cnt = min(32, nmine - kb);
        const int nl = n0 + warp + (kb + min(lane, cnt - 1)) * nw;
        const Ray mine = make_ray(a.g, c, nl);
        float my_w = 0.f;
        for (int r = 0; r < cnt; ++r) {
            const Ray ry = shfl_ray(mine, r);
            const int nsamp = ry.nfull + (ry.rem > 0.f ? 1 : 0);
            const int per = (nsamp + 31) >> 5;
            const int m0 = lane * per, m1 = min(nsamp, m0 + per);
            const int mf = min(m1, ry.nfull);
            float acc = 0.f;
            for (int m = m0; m < mf; ++m) {
                const float s = (m + 0.5f) * h;
                const Bil b = bil(G, pitch, fmaf(s, ry.bx, ry.ax), fmaf(s, ry.by, ry.ay));
                const float d = SMEM ? interp(dv, pitch, b) : interp_global(a.sos, G, v0, b);
                acc += __fdividef(d, v0 + d);
            }
            acc *= h;
            if (m0 <= ry.nfull && ry.nfull < m1) {    // last partial step, weighted by its length
                const float s = ry.nfull * h + 0.5f * ry.rem;
                const Bil b = bil(G, pitch, fmaf(s, ry.bx, ry.ax), fmaf(s, ry.by, ry.ay));
                const float d = SMEM ? interp(dv, pitch, b) : interp_global(a.sos, G, v0, b);
                acc = fmaf(ry.rem, __fdividef(d, v0 + d), acc);
            }
            acc = warp_sum(acc);
            if (lane == r) my_w = fmaf(ry.L - ry.chord, out_coef, acc);
        }
        if (lane < cnt) out(nl, my_w);
    }
}

// CTA b: rays [n0, n1) of patch b / splits.
template <bool SMEM>
__global__ void __launch_bounds__(512) rays_fwd_kernel(const RayArgs a) {
    extern __shared__ float dv_s[];
    const int G = a.g.G, pitch = SMEM ? smem_pitch(G) : G;
    if (SMEM) {
        load_excess(dv_s, a.sos, G, pitch, a.g.v0);
        __syncthreads();
    }
    int i, n0, n1;
    cta_rays(a, i, n0, n1);
    const int2 cc = a.centres[i];
    float* w = a.w + (size_t)i * a.g.n_t;
    warp_rays<SMEM>(a, dv_s, pitch, pixel_xy(a.g, cc.x, cc.y), n0, n1, threadIdx.x >> 5, blockDim.x >> 5,
                    [&](int n, float wn) { w[n] = wn; });
}

// Rays from image pixels (sources of channel data): the CTAs take the pixels
// pix0 + q, q = blockIdx.x, blockIdx.x + gridDim.x, ... < npix, skip those with
// p0 == 0, and write w from pixel q to every transducer n at wT[n * ld + q].
template <bool SMEM>
__global__ void __launch_bounds__(512) rays_pix_kernel(const RayArgs a, const float* p0, int pix0, int npix,
                                                       float* wT, int ld) {
    extern __shared__ float dv_s[];
    const int G = a.g.G, pitch = SMEM ? smem_pitch(G) : G;
    if (SMEM) {
        load_excess(dv_s, a.sos, G, pitch, a.g.v0);
        __syncthreads();
    }
    for (int q = blockIdx.x; q < npix; q += gridDim.x) {
        const int pix = pix0 + q;
        if (p0[pix] == 0.f) continue;                 // the same for the whole CTA
        const int row = pix / a.g.W, col = pix - (pix / a.g.W) * a.g.W;
        warp_rays<SMEM>(a, dv_s, pitch, pixel_xy(a.g, row, col), 0, a.g.n_t, threadIdx.x >> 5, blockDim.x >> 5,
                        [&](int n, float wn) { wT[(size_t)n * ld + q] = wn; });
    }
}

__device__ __forceinline__ void scatter4(float* acc, int pitch, int idx, float c00, float c01, float c10,
                                         float c11) {
    atomicAdd(acc + idx, c00);
    atomicAdd(acc + idx + 1, c01);
    atomicAdd(acc + idx + pitch, c10);
    atomicAdd(acc + idx + pitch + 1, c11);
}

// CTA b takes the rays r = b, b + nb, b + 2 nb, ... of the flat (patch,
// transducer) index r = i N_t + n, and each warp a contiguous block of them, so
// that its warps integrate rays of different patches and directions at the same
// time (rays of one patch all start at the same centre, where their scatters
// would collide).  A lane walks a contiguous
// run of samples of one ray and keeps the bilinear weights of the current cell
// in registers, adding them to the shared grid only when the walk leaves the
// cell.
template <bool SMEM>
__global__ void __launch_bounds__(1024, 1) rays_adj_kernel(const RayArgs a) {
    extern __shared__ float sm[];
    const int G = a.g.G, pitch = SMEM ? smem_pitch(G) : G;
    const int GP = G * pitch;
    const float v0 = a.g.v0;
    float* dv_s = sm;
    float* acc_s = sm + GP;
    if (SMEM) {
        for (int q = threadIdx.x; q < GP; q += blockDim.x) acc_s[q] = 0.f;
        load_excess(dv_s, a.sos, G, pitch, v0);
    }
    __syncthreads();
    float* acc = SMEM ? acc_s : a.out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nrays = a.N * a.g.n_t, nb = gridDim.x;
    const int mine = nrays > (int)blockIdx.x ? (nrays - (int)blockIdx.x + nb - 1) / nb : 0;   // rays of this CTA
    // warp w takes the contiguous block t0 <= t < t1 of the CTA's rays t (r = b + nb t), so that the
    // warps work on rays of different patches at any moment (rays of one patch share their start)
    const int t0 = (int)((long long)mine * warp / nw), t1 = (int)((long long)mine * (warp + 1) / nw);
    const int nwarp = t1 - t0;
    const float h = a.g.h;
    for (int kb = 0; kb < nwarp; kb += 32) {
        const int cnt = min(32, nwarp - kb);
        const int r = (int)blockIdx.x + nb * (t0 + kb + min(lane, cnt - 1));
        const int i = r / a.g.n_t, n = r - (r / a.g.n_t) * a.g.n_t;
        const int2 cc = a.centres[i];
        const Ray mine_ray = make_ray(a.g, pixel_xy(a.g, cc.x, cc.y), n);
        const float my_g = lane < cnt ? a.dLdw[r] : 0.f;
        for (int rr = 0; rr < cnt; ++rr) {
            const float gr = __shfl_sync(0xffffffffu, my_g, rr);
            if (gr == 0.f) continue;
            const Ray ry = shfl_ray(mine_ray, rr);
            const int nsamp = ry.nfull + (ry.rem > 0.f ? 1 : 0);
            const int per = (nsamp + 31) >> 5;
            const int m0 = lane * per, m1 = min(nsamp, m0 + per);
            const float gv0 = gr * v0;
            int cur = -1;
            float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
            for (int m = m0; m < m1; ++m) {
                const bool last = m >= ry.nfull;
                const float s = last ? ry.nfull * h + 0.5f * ry.rem : (m + 0.5f) * h;
                const float wgt = last ? ry.rem : h;
                const Bil b = bil(G, pitch, fmaf(s, ry.bx, ry.ax), fmaf(s, ry.by, ry.ay));
                const float d = SMEM ? interp(dv_s, pitch, b) : interp_global(a.sos, G, v0, b);
                const float iv = __fdividef(1.f, v0 + d);
                const float coef = gv0 * wgt * iv * iv;
                if (b.idx != cur) {
                    if (cur >= 0) scatter4(acc, pitch, cur, c00, c01, c10, c11);
                    cur = b.idx;
                    c00 = c01 = c10 = c11 = 0.f;
                }
                const float cy0 = coef * (1.f - b.ty), cy1 = coef * b.ty;
                c00 = fmaf(cy0, 1.f - b.tx, c00);
                c01 = fmaf(cy0, b.tx, c01);
                c10 = fmaf(cy1, 1.f - b.tx, c10);
                c11 = fmaf(cy1, b.tx, c11);
            }
            if (cur >= 0) scatter4(acc, pitch, cur, c00, c01, c10, c11);
        }
    }
    if (SMEM && a.cluster) {
        // the CTAs of a cluster sum their shared grids through distributed shared
        // memory (CTA rank r takes a band of rows, in a fixed order of ranks) and
        // write one partial grid per cluster
        namespace cg = cooperative_groups;
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        const int csize = (int)cl.num_blocks(), rank = (int)cl.block_rank();
        const int rows = (G + csize - 1) / csize;
        const int r0 = min(G, rank * rows), r1 = min(G, r0 + rows);
        float* dst = a.part + (size_t)(blockIdx.x / csize) * G * G;
        for (int q = threadIdx.x; q < (r1 - r0) * G; q += blockDim.x) {
            const int p = r0 + q / G, cq = q - (q / G) * G;
            float sum = 0.f;
            for (int r = 0; r < csize; ++r) sum += cl.map_shared_rank(acc_s, r)[p * pitch + cq];
            dst[p * G + cq] = sum;
        }
        cl.sync();                                   // remote reads end before any CTA exits
    } else if (SMEM) {
        __syncthreads();
        float* dst = a.part + (size_t)blockIdx.x * G * G;
        for (int q = threadIdx.x; q < G * G; q += blockDim.x) {
            const int p = q / G, cq = q - (q / G) * G;
            dst[q] = acc_s[p * pitch + cq];
        }
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

constexpr int kCluster = 4;   // CTAs per cluster in the ray adjoint (8 would not fit in one wave)

struct Plan {
    int splits_fwd, splits_adj, nb_fwd, nb_adj, nr, use_smem, cluster, nparts;
    size_t smem_fwd, smem_adj, off_stage1, ws;
};

// CTAs per patch so that the grid fills every SM once at the occupancy the
// kernel's registers and shared memory allow (at least 32 rays per CTA).
int splits_for(const pact_geometry* g, const pact_patches* pt, const void* fn, int threads, size_t smem) {
    const int sms = num_sms();
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int s = (sms * per_sm) / pt->n;
    return std::max(1, std::min(s, std::max(1, g->n_t / 32)));
}

// Whether clusters of kCluster adjoint CTAs (1024 threads, `smem` bytes each) can
// be resident on this device (queried once per device).
bool cluster_fits(size_t smem) {
    static int cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (cached[dev] == 0) {
        int ok = -1;
        const void* fn = (const void*)rays_adj_kernel<true>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(kCluster);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeClusterDimension;
            attr.val.clusterDim.x = kCluster;
            attr.val.clusterDim.y = 1;
            attr.val.clusterDim.z = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0) ok = 1;
        }
        cudaGetLastError();
        cached[dev] = ok;
    }
    return cached[dev] > 0;
}

Plan make_plan(const pact_geometry* g, const pact_patches* pt) {
    Plan p;
    const int G = g->sos_g;
    const size_t gbytes = (size_t)G * smem_pitch(G) * sizeof(float);
    p.use_smem = 2 * gbytes <= kMaxSmem;
    p.smem_fwd = p.use_smem ? gbytes : 0;
    p.smem_adj = p.use_smem ? 2 * gbytes : 0;
    p.splits_fwd = splits_for(g, pt, p.use_smem ? (const void*)rays_fwd_kernel<true> : (const void*)rays_fwd_kernel<false>,
                              512, p.smem_fwd);
    p.splits_adj = splits_for(g, pt, p.use_smem ? (const void*)rays_adj_kernel<true> : (const void*)rays_adj_kernel<false>,
                              1024, p.smem_adj);
    p.nb_fwd = pt->n * p.splits_fwd;
    p.nb_adj = pt->n * p.splits_adj;
    p.cluster = 0;
    if (p.use_smem && cluster_fits(p.smem_adj)) {
        p.cluster = kCluster;
        p.nb_adj = (p.nb_adj + kCluster - 1) / kCluster * kCluster;
    }
    p.nparts = p.cluster ? p.nb_adj / p.cluster : p.nb_adj;
    p.nr = (p.nparts + kGroup - 1) / kGroup;
    const size_t plane = (size_t)G * G * sizeof(float);
    p.off_stage1 = align_up((size_t)p.nparts * plane, 256);
    p.ws = p.use_smem ? p.off_stage1 + align_up((size_t)p.nr * plane, 256) : 256;
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
    a.cluster = pl.cluster;
    return a;
}

}  // namespace

pact_status launch_pixel_rays(const pact_geometry* g, const float* sos, const float* p0, int pix0, int npix,
                              float* wT, int ld, cudaStream_t st) {
    if (npix <= 0) return PACT_OK;
    const int G = g->sos_g;
    const size_t gbytes = (size_t)G * smem_pitch(G) * sizeof(float);
    const bool smem = gbytes <= kMaxSmem;
    const void* fn = smem ? (const void*)rays_pix_kernel<true> : (const void*)rays_pix_kernel<false>;
    if (smem) PACT_TRY(ensure_smem(fn, gbytes, "rf_synth: shared memory attribute"));
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 512, smem ? gbytes : 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int grid = std::min(npix, num_sms() * per_sm);
    RayArgs a = {};
    a.g = make_geo(g);
    a.N = 0;
    a.sos = sos;
    a.use_smem = smem;
    if (smem)
        rays_pix_kernel<true><<<grid, 512, gbytes, st>>>(a, p0, pix0, npix, wT, ld);
    else
        rays_pix_kernel<false><<<grid, 512, 0, st>>>(a, p0, pix0, npix, wT, ld);
    return check_launch("rf_synth: ray kernel");
}

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
    if (pl.use_smem) {
        PACT_TRY(ensure_smem((const void*)rays_fwd_kernel<true>, pl.smem_fwd, "sos_to_delays: shared memory attribute"));
        rays_fwd_kernel<true><<<pl.nb_fwd, 512, pl.smem_fwd, as_stream(stream)>>>(a);
    } else {
        rays_fwd_kernel<false><<<pl.nb_fwd, 512, 0, as_stream(stream)>>>(a);
    }
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
        PACT_TRY(ensure_smem((const void*)rays_adj_kernel<true>, pl.smem_adj,
                             "sos_to_delays_adj: shared memory attribute"));
        if (pl.cluster) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(pl.nb_adj);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = pl.smem_adj;
            cfg.stream = st;
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeClusterDimension;
            attr.val.clusterDim.x = pl.cluster;
            attr.val.clusterDim.y = 1;
            attr.val.clusterDim.z = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, rays_adj_kernel<true>, a) != cudaSuccess)
                return check_launch("sos_to_delays_adj kernel (cluster launch)");
            PACT_TRY(check_launch("sos_to_delays_adj kernel"));
            // one partial grid per cluster: a single fixed-order sum
            reduce_stage2_kernel<<<(GG + 255) / 256, 256, 0, st>>>(a.part, pl.nparts, GG, dL_dsos, accumulate);
            return check_launch("sos_to_delays_adj reduction");
        }
        rays_adj_kernel<true><<<pl.nb_adj, 1024, pl.smem_adj, st>>>(a);
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
    rays_adj_kernel<false><<<pl.nb_adj, 1024, 0, st>>>(a);
    return check_launch("sos_to_delays_adj kernel");
}
