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

__device__ __forceinline__ void scatter4(int* acc, int pitch, int idx, float S, float c00, float c01, float c10,
                                         float c11) {
    atomicAdd(acc + idx, __float2int_rn(c00 * S));
    atomicAdd(acc + idx + 1, __float2int_rn(c01 * S));
    atomicAdd(acc + idx + pitch, __float2int_rn(c10 * S));
    atomicAdd(acc + idx + pitch + 1, __float2int_rn(c11 * S));
}

__device__ __forceinline__ float block_min(float x, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = x;
    __syncthreads();
    x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
    if (wid == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    __syncthreads();
    return x;
}

// Ray adjoint.  CTA b takes the rays r = b, b + nb, b + 2 nb, ... of the flat
// (patch, transducer) index r = i N_t + n, and each warp a contiguous block of
// them, so that its warps integrate rays of different patches and directions
// at the same time (rays of one patch all start at the same centre, where their
// scatters would collide).  A lane walks a contiguous run of samples of one ray
// and keeps the bilinear weights of the current cell in registers, adding them
// to the shared grid only when the walk leaves the cell.
//
// The shared grid holds 32-bit fixed-point sums (shared-memory integer atomics
// are single instructions; float ones are compare-and-swap loops), which also
// makes the result independent of the order of the additions.  Every
// contribution is g h_s v0 / v^2 times a bilinear weight; v is a convex
// combination of node values, so v >= vmin, and the weights h_s of a ray add up
// to its chord <= 2 mask_r.  The absolute sum of all contributions of the CTA
// is therefore at most  Mb = sum_r |g_r| 2 mask_r v0 / vmin^2 , and with the
// scale S = 2^30 / Mb no partial sum of a node can leave the int32 range
// (each flush rounds by at most 1/2).  A non-finite bound (NaN in dL/dw or the
// SOS, or SOS <= 0) turns the CTA's partial grid into NaN.
//
// Grids are processed in bands of R cell rows (node rows r0 .. r0 + R), so
// that the SOS excess rows and the accumulator of a band fit in shared memory
// for every G <= 512; a ray visits each band with the samples whose cell row
// lies in it.  Node row r0 + R is shared with the next band: its sums move to
// that band's first row.  With clusters, the CTAs of a cluster sum each band of
// their grids through distributed shared memory in a fixed order of ranks and
// write one partial grid per cluster; otherwise every CTA writes its own.
__global__ void __launch_bounds__(1024, 1) rays_adj_kernel(const RayArgs a, int R, int nbands) {
    extern __shared__ float sm[];
    __shared__ float red_s[32];
    __shared__ float scale_s[2];      // S and 1/S (NaN: poisoned)
    const int G = a.g.G, pitch = smem_pitch(G);
    float* dv_s = sm;                                              // [R + 1][pitch]
    int* acc_s = reinterpret_cast<int*>(sm + (R + 1) * pitch);      // [R + 1][pitch]
    const float v0 = a.g.v0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nrays = a.N * a.g.n_t, nb = gridDim.x;
    const int mine = nrays > (int)blockIdx.x ? (nrays - (int)blockIdx.x + nb - 1) / nb : 0;   // rays of this CTA

    // fixed-point scale of this CTA
    float gsum = 0.f, vmin = INFINITY, bad = 0.f;
    for (int t = threadIdx.x; t < mine; t += blockDim.x) gsum += fabsf(a.dLdw[(size_t)blockIdx.x + (size_t)nb * t]);
    for (int q = threadIdx.x; q < G * G; q += blockDim.x) {
        const float v = __ldg(a.sos + q);
        if (!(v > 0.f) || !isfinite(v)) bad = 1.f;
        vmin = fminf(vmin, v);
    }
    gsum = block_sum(gsum, red_s);
    bad = block_sum(bad, red_s);
    vmin = block_min(vmin, red_s);
    if (threadIdx.x == 0) {
        const float vm = vmin * (1.f - 1e-5f);
        const float Mb = gsum * (2.f * a.g.mask_r) * (v0 / (vm * vm));
        const bool poison = bad > 0.f || !isfinite(Mb);
        const float S = Mb > 0.f ? fminf(1073741824.f / Mb, 1e30f) : 0.f;
        scale_s[0] = poison ? 0.f : S;
        scale_s[1] = poison ? __int_as_float(0x7fc00000) : (S > 0.f ? 1.f / S : 0.f);
    }
    __syncthreads();
    const float S = scale_s[0];

    // warp w takes the contiguous block t0 <= t < t1 of the CTA's rays t (r = b + nb t)
    const int t0 = (int)((long long)mine * warp / nw), t1 = (int)((long long)mine * (warp + 1) / nw);
    const int nwarp = t1 - t0;
    const float h = a.g.h;
    namespace cg = cooperative_groups;
    for (int band = 0; band < nbands; ++band) {
        const bool last_band = band == nbands - 1;
        const int r0 = band * R;
        const int r1 = last_band ? G - 1 : r0 + R;        // cell rows r0 <= iy < r1
        const int rows = min(R + 1, G - r0);              // node rows r0 .. r0 + rows - 1 of the band
        for (int q = threadIdx.x; q < rows * G; q += blockDim.x) {
            const int p = q / G, c = q - (q / G) * G;
            dv_s[p * pitch + c] = __ldg(a.sos + (size_t)(r0 + p) * G + c) - v0;
        }
        for (int q = threadIdx.x + (band > 0 ? pitch : 0); q < rows * pitch; q += blockDim.x) acc_s[q] = 0;
        __syncthreads();
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
                // samples whose cell row can lie in the band (the test below is exact;
                // this range only needs to contain them)
                int mlo = 0, mhi = nsamp;
                if (nbands > 1 && ry.by != 0.f) {
                    const float inv = 1.f / (ry.by * h);
                    float ma = ((float)r0 - ry.ay) * inv - 0.5f, mb = ((float)r1 - ry.ay) * inv - 0.5f;
                    if (r0 == 0) ma = ry.by > 0.f ? -INFINITY : INFINITY;          // clamped rows below 0
                    if (r1 == G - 1) mb = ry.by > 0.f ? INFINITY : -INFINITY;      // clamped rows above G - 2
                    const float lo = fmaxf(fminf(ma, mb), -1e9f), hi = fminf(fmaxf(ma, mb), 1e9f);
                    mlo = max(0, (int)floorf(lo) - 2);
                    mhi = min(nsamp, (int)ceilf(hi) + 2);
                }
                if (mhi <= mlo) continue;
                const int per = (mhi - mlo + 31) >> 5;
                const int m0 = mlo + lane * per, m1 = min(mhi, m0 + per);
                const float gv0 = gr * v0;
                int cur = -1;
                float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
                for (int m = m0; m < m1; ++m) {
                    const bool last = m >= ry.nfull;
                    const float s = last ? ry.nfull * h + 0.5f * ry.rem : (m + 0.5f) * h;
                    const float fx = fminf(fmaxf(fmaf(s, ry.bx, ry.ax), 0.f), (float)(G - 1));
                    const float fy = fminf(fmaxf(fmaf(s, ry.by, ry.ay), 0.f), (float)(G - 1));
                    const int iy = min((int)fy, G - 2);
                    if (iy < r0 || iy >= r1) continue;
                    const int ix = min((int)fx, G - 2);
                    Bil b;
                    b.idx = (iy - r0) * pitch + ix;
                    b.tx = fx - ix;
                    b.ty = fy - iy;
                    const float d = interp(dv_s, pitch, b);
                    const float iv = __fdividef(1.f, v0 + d);
                    const float coef = gv0 * (last ? ry.rem : h) * iv * iv;
                    if (b.idx != cur) {
                        if (cur >= 0) scatter4(acc_s, pitch, cur, S, c00, c01, c10, c11);
                        cur = b.idx;
                        c00 = c01 = c10 = c11 = 0.f;
                    }
                    const float cy0 = coef * (1.f - b.ty), cy1 = coef * b.ty;
                    c00 = fmaf(cy0, 1.f - b.tx, c00);
                    c01 = fmaf(cy0, b.tx, c01);
                    c10 = fmaf(cy1, 1.f - b.tx, c10);
                    c11 = fmaf(cy1, b.tx, c11);
                }
                if (cur >= 0) scatter4(acc_s, pitch, cur, S, c00, c01, c10, c11);
            }
        }
        // node rows written by this band: r0 .. r0 + R - 1 (its last row moves to the next band)
        const int out_rows = last_band ? rows : R;
        if (a.cluster) {
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            const int csize = (int)cl.num_blocks(), rank = (int)cl.block_rank();
            const int share = (out_rows + csize - 1) / csize;
            const int p0 = min(out_rows, rank * share), p1 = min(out_rows, p0 + share);
            float* dst = a.part + (size_t)(blockIdx.x / csize) * G * G + (size_t)r0 * G;
            for (int q = threadIdx.x; q < (p1 - p0) * G; q += blockDim.x) {
                const int p = p0 + q / G, c = q - (q / G) * G;
                float sum = 0.f;
                for (int k = 0; k < csize; ++k)
                    sum += (float)cl.map_shared_rank(acc_s, k)[p * pitch + c] * *cl.map_shared_rank(scale_s + 1, k);
                dst[p * G + c] = sum;
            }
            cl.sync();                               // remote reads end before any CTA changes its grid
        } else {
            __syncthreads();
            const float invS = scale_s[1];
            float* dst = a.part + (size_t)blockIdx.x * G * G + (size_t)r0 * G;
            for (int q = threadIdx.x; q < out_rows * G; q += blockDim.x) {
                const int p = q / G, c = q - (q / G) * G;
                dst[p * G + c] = (float)acc_s[p * pitch + c] * invS;
            }
            __syncthreads();
        }
        if (!last_band) {
            for (int c = threadIdx.x; c < pitch; c += blockDim.x) acc_s[c] = acc_s[R * pitch + c];
            __syncthreads();
        }
    }
}

// out[q] (+)= sum of the partial grids part[0 .. np)[q], in order.
__global__ void reduce_parts_kernel(const float* part, int np, int GG, float* out, int accumulate) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= GG) return;
    float s = 0.f;
    for (int r = 0; r < np; ++r) s += part[(size_t)r * GG + q];
    out[q] = accumulate ? out[q] + s : s;
}

constexpr size_t kMaxSmem = 200 * 1024;

constexpr int kCluster = 4;   // CTAs per cluster in the ray adjoint (8 would not fit in one wave)

struct Plan {
    int splits_fwd, nb_fwd, use_smem_fwd;
    int R, nbands, nb_adj, cluster, nparts;
    size_t smem_fwd, smem_adj, ws;
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

// How many clusters of kCluster adjoint CTAs (1024 threads, `smem` bytes each)
// can be resident at once on this device (0: clusters unavailable); cached
// per device and shared-memory size.
int max_clusters(size_t smem) {
    struct Entry {
        int dev;
        size_t smem;
        int n;
    };
    static Entry cache[16];
    static int used = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int k = 0; k < used; ++k)
        if (cache[k].dev == dev && cache[k].smem == smem) return cache[k].n;
    int n = 0;
    const void* fn = (const void*)rays_adj_kernel;
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
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    if (used < 16) cache[used++] = Entry{dev, smem, n};
    return n;
}

Plan make_plan(const pact_geometry* g, const pact_patches* pt) {
    Plan p;
    const int G = g->sos_g, pitch = smem_pitch(G);
    const size_t gbytes = (size_t)G * pitch * sizeof(float);
    p.use_smem_fwd = gbytes <= kMaxSmem;
    p.smem_fwd = p.use_smem_fwd ? gbytes : 0;
    p.splits_fwd = splits_for(g, pt, p.use_smem_fwd ? (const void*)rays_fwd_kernel<true>
                                                    : (const void*)rays_fwd_kernel<false>, 512, p.smem_fwd);
    p.nb_fwd = pt->n * p.splits_fwd;
    // adjoint: bands of R cell rows, excess rows and accumulator of a band in shared memory
    p.R = std::max(1, std::min(G - 1, (int)(kMaxSmem / (2 * sizeof(float) * (size_t)pitch)) - 1));
    p.nbands = (G - 1 + p.R - 1) / p.R;
    p.smem_adj = 2 * sizeof(float) * (size_t)(p.R + 1) * pitch;
    const int nrays = pt->n * g->n_t;
    const int want = std::max(1, std::min(num_sms(), (nrays + 31) / 32));   // one persistent CTA per SM
    const int nc = max_clusters(p.smem_adj);
    p.cluster = 0;
    p.nb_adj = want;
    if (nc > 0 && want >= kCluster) {
        p.cluster = kCluster;
        p.nb_adj = std::min(nc, want / kCluster) * kCluster;
    }
    p.nparts = p.cluster ? p.nb_adj / p.cluster : p.nb_adj;
    p.ws = align_up((size_t)p.nparts * G * G * sizeof(float), 256);
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
    a.use_smem = pl.use_smem_fwd;
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
    if (pl.use_smem_fwd) {
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
    RayArgs a = make_args(g, pt, pl, 1, sos);
    a.dLdw = dL_dw;
    a.part = static_cast<float*>(ws);
    a.out = dL_dsos;
    PACT_TRY(ensure_smem((const void*)rays_adj_kernel, pl.smem_adj, "sos_to_delays_adj: shared memory attribute"));
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
        if (cudaLaunchKernelEx(&cfg, rays_adj_kernel, a, pl.R, pl.nbands) != cudaSuccess)
            return check_launch("sos_to_delays_adj kernel (cluster launch)");
    } else {
        rays_adj_kernel<<<pl.nb_adj, 1024, pl.smem_adj, st>>>(a, pl.R, pl.nbands);
    }
    PACT_TRY(check_launch("sos_to_delays_adj kernel"));
    // one partial grid per cluster (or CTA): a single fixed-order sum
    reduce_parts_kernel<<<(GG + 255) / 256, 256, 0, st>>>(a.part, pl.nparts, GG, dL_dsos, accumulate);
    return check_launch("sos_to_delays_adj reduction");
}
