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
#include <cmath>

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
    int use_smem;
    float4* clear;        // forward: [n_clear4] set to zero in the same launch (or NULL)
    size_t n_clear4;
    float tv_lambda;      // forward: with tv_grad, lambda times the TV terms of Eq. 7
    float* tv_grad;       //   [G*G] lambda * TV subgradient (or NULL)
    float* tv_part;       //   [gridDim.x] lambda * TV(v) over each CTA's nodes
};

__device__ __forceinline__ float tv_sgn(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// TV regulariser of Eq. 7, TV(v) = sum |v[p+1][q] - v[p][q]| + |v[p][q+1] - v[p][q]|,
// on this CTA's share of the nodes: lambda times its subgradient (sign(0) = 0)
// into tv_grad, lambda times its part of the value into tv_part[blockIdx.x]
// (summed later in a fixed order).  All threads of the CTA take part.
__device__ void tv_terms(const RayArgs& a) {
    __shared__ float red[32];
    const int G = a.g.G, GG = G * G;
    const int q0 = (int)((long long)GG * blockIdx.x / gridDim.x);
    const int q1 = (int)((long long)GG * (blockIdx.x + 1) / gridDim.x);
    float part = 0.f;
    for (int q = q0 + (int)threadIdx.x; q < q1; q += blockDim.x) {
        const int p = q / G, c = q - p * G;
        const float v = __ldg(a.sos + q);
        float gq = 0.f;
        if (p + 1 < G) {
            const float dn = __ldg(a.sos + q + G) - v;
            part += fabsf(dn);
            gq -= tv_sgn(dn);
        }
        if (c + 1 < G) {
            const float rt = __ldg(a.sos + q + 1) - v;
            part += fabsf(rt);
            gq -= tv_sgn(rt);
        }
        if (p > 0) gq += tv_sgn(v - __ldg(a.sos + q - G));
        if (c > 0) gq += tv_sgn(v - __ldg(a.sos + q - 1));
        a.tv_grad[q] = a.tv_lambda * gq;
    }
    const float tot = block_sum(part, red);
    if (threadIdx.x == 0) a.tv_part[blockIdx.x] = a.tv_lambda * tot;
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

// Padded staging for the forward integrals: node (p, c) of the excess grid at
// (p + 2, c + 2) of a (G + 4) x (G + 4) array of row pitch G + 5, the two outer
// rings replicating the edge nodes, so that bilinear interpolation on the
// padded array equals the edge-clamped interpolation of the grid for node
// coordinates in [-2, G + 1] and needs no clamps.
__host__ __device__ __forceinline__ int pad_pitch(int G) { return G + 5; }
__host__ __device__ __forceinline__ size_t pad_bytes(int G) { return (size_t)(G + 4) * pad_pitch(G) * sizeof(float); }

// Padded rows r0 .. r0 + rows - 1 of the SOS grid (raw values, edge-clamped
// sources) into dv[row - r0][.] with 4-byte asynchronous copies, all in flight
// at once (the grid comes from L2, whose latency would otherwise be paid per
// load); the caller waits with cp_async_wait_all and a barrier.
__device__ __forceinline__ void stage_padded_async(float* dv, const float* sos, int G, int r0, int rows) {
    const int pitch = pad_pitch(G), P = G + 4;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int pl = threadIdx.x >> 5; pl < rows; pl += nw) {
        const float* row = sos + (size_t)min(max(r0 + pl - 2, 0), G - 1) * G;
        for (int cc = lane; cc < P; cc += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dv + pl * pitch + cc)),
                         "l"(row + min(max(cc - 2, 0), G - 1))
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The whole padded excess grid dv = sos - v0 (see pad_pitch).
__device__ __forceinline__ void load_excess_padded(float* dv, const float* sos, int G, float v0) {
    const int pitch = pad_pitch(G), P = G + 4;
    stage_padded_async(dv, sos, G, 0, P);
    cp_async_wait_all();
    __syncthreads();
    for (int pl = threadIdx.x >> 5; pl < P; pl += blockDim.x >> 5)
        for (int cc = threadIdx.x & 31; cc < P; cc += 32) dv[pl * pitch + cc] -= v0;
}

// Slowness excess (v - v0)/v = dv / (v0 + dv) at padded node coordinates
// (x, y) in [1, G + 2] (node coordinate + 2): bilinear dv on the padded grid.
// floor() without conversions: adding 2^23 - 1/2 to x >= 1/2 rounds x - 1/2 to
// an integer in the low mantissa bits of the sum, which is floor(x) (or x - 1
// for integral x, where the weight 1 on the upper node gives the same value).
__device__ __forceinline__ float excess_padded(const float* dv, int pitch, float x, float y, float v0) {
    const float tX = x + 8388607.5f, tY = y + 8388607.5f;
    const int ix = __float_as_int(tX) - 0x4B000000, iy = __float_as_int(tY) - 0x4B000000;
    const float tx = x - (tX - 8388608.f), ty = y - (tY - 8388608.f);
    const float* q = dv + iy * pitch + ix;
    const float d00 = q[0], d01 = q[1], d10 = q[pitch], d11 = q[pitch + 1];
    const float top = fmaf(tx, d01 - d00, d00), bot = fmaf(tx, d11 - d10, d10);
    const float d = fmaf(ty, bot - top, top);
    return __fdividef(d, v0 + d);
}

// The part of ray `ry` that lane `sub` of a group of L lanes integrates: a
// contiguous run of its midpoint samples (the last one, of length rem, at
// nfull h + rem/2), weighted by their lengths.
// PAD: padded shared grid (see above); else SMEM: clamped shared grid of row
// pitch `pitch`; else the SOS grid in global memory.
template <int L, bool SMEM, bool PAD>
__device__ __forceinline__ float ray_part(const RayArgs& a, const float* dv, int pitch, const Ray& ry, int sub) {
    const int G = a.g.G;
    const float h = a.g.h, v0 = a.g.v0;
    const int nsamp = ry.nfull + (ry.rem > 0.f ? 1 : 0);
    const int per = (nsamp + L - 1) / L;
    const int m0 = sub * per, m1 = min(nsamp, m0 + per);
    const float hbx = h * ry.bx, hby = h * ry.by;
    const float ax = PAD ? ry.ax + 2.f : ry.ax, ay = PAD ? ry.ay + 2.f : ry.ay;
    auto excess = [&](float u) {
        const float x = fmaf(u, hbx, ax), y = fmaf(u, hby, ay);
        if (PAD) return excess_padded(dv, pitch, x, y, v0);
        const Bil b = bil(G, pitch, x, y);
        const float d = SMEM ? interp(dv, pitch, b) : interp_global(a.sos, G, v0, b);
        return __fdividef(d, v0 + d);
    };
    // full samples (length h) first, then the partial last one if this lane has it
    const int mf = min(m1, ry.nfull);
    float acc = 0.f, uf = m0 + 0.5f;
#pragma unroll 8
    for (int m = m0; m < mf; ++m, uf += 1.f) acc += excess(uf);
    acc *= h;
    if (m0 <= ry.nfull && m1 > ry.nfull)    // the lane whose run holds the partial sample
        acc = fmaf(ry.rem, excess(ry.nfull + 0.5f * (ry.rem / h)), acc);
    return acc;
}

// Forward rays.  Work item t = (patch i, block of 32/L consecutive
// transducers); warp-strided over the grid (persistent CTAs), a warp's lanes
// form 32/L groups of L lanes, one ray per group (neighbouring transducers:
// similar directions and lengths), each lane a contiguous run of samples;
// the group's partial sums meet in a fixed butterfly order.
template <int L, bool SMEM, bool PAD>
__global__ void __launch_bounds__(512) rays_fwd_kernel(const RayArgs a) {
    extern __shared__ float dv_s[];
    pdl_trigger();            // a dependent launch (the fused pass) may set up meanwhile
    const int G = a.g.G;
    const int pitch = PAD ? pad_pitch(G) : (SMEM ? smem_pitch(G) : G);
    if (SMEM) {
        if (PAD)
            load_excess_padded(dv_s, a.sos, G, a.g.v0);
        else
            load_excess(dv_s, a.sos, G, pitch, a.g.v0);
        __syncthreads();
    }
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n_clear4; q += (size_t)gridDim.x * blockDim.x)
        a.clear[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.tv_grad) tv_terms(a);
    constexpr int RB = 32 / L;
    const int n_t = a.g.n_t;
    const int lane = threadIdx.x & 31, sub = lane % L, grp = lane / L;
    const int nblk = (n_t + RB - 1) / RB, items = a.N * nblk;
    const int wpb = blockDim.x >> 5, W = gridDim.x * wpb;
    const float out_coef = (a.g.v_bg - a.g.v0) / a.g.v_bg;
    for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < items; t += W) {
        const int i = t / nblk;
        const int n = (t - i * nblk) * RB + grp;
        const bool valid = n < n_t;
        const int2 cc = a.centres[i];
        const Ray ry = make_ray(a.g, pixel_xy(a.g, cc.x, cc.y), valid ? n : 0);
        float acc = valid ? ray_part<L, SMEM, PAD>(a, dv_s, pitch, ry, sub) : 0.f;
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (valid && sub == 0) a.w[(size_t)i * n_t + n] = fmaf(ry.L - ry.chord, out_coef, acc);
    }
}

// Rays from image pixels (sources of channel data): the CTAs take the pixels
// pix0 + q, q = blockIdx.x, blockIdx.x + gridDim.x, ... < npix, skip those with
// p0 == 0, and write w from pixel q to every transducer n at wT[n * ld + q]
// (warps over blocks of 32/L transducers, groups of L lanes per ray).
template <int L, bool SMEM, bool PAD>
__global__ void __launch_bounds__(512) rays_pix_kernel(const RayArgs a, const float* p0, int pix0, int npix,
                                                       float* wT, int ld) {
    extern __shared__ float dv_s[];
    const int G = a.g.G;
    const int pitch = PAD ? pad_pitch(G) : (SMEM ? smem_pitch(G) : G);
    if (SMEM) {
        if (PAD)
            load_excess_padded(dv_s, a.sos, G, a.g.v0);
        else
            load_excess(dv_s, a.sos, G, pitch, a.g.v0);
        __syncthreads();
    }
    constexpr int RB = 32 / L;
    const int n_t = a.g.n_t;
    const int lane = threadIdx.x & 31, sub = lane % L, grp = lane / L;
    const int nblk = (n_t + RB - 1) / RB, wpb = blockDim.x >> 5;
    const float out_coef = (a.g.v_bg - a.g.v0) / a.g.v_bg;
    for (int q = blockIdx.x; q < npix; q += gridDim.x) {
        const int pix = pix0 + q;
        if (p0[pix] == 0.f) continue;                 // the same for the whole CTA
        const int row = pix / a.g.W, col = pix - (pix / a.g.W) * a.g.W;
        const float2 c = pixel_xy(a.g, row, col);
        for (int blk = threadIdx.x >> 5; blk < nblk; blk += wpb) {
            const int n = blk * RB + grp;
            const bool valid = n < n_t;
            const Ray ry = make_ray(a.g, c, valid ? n : 0);
            float acc = valid ? ray_part<L, SMEM, PAD>(a, dv_s, pitch, ry, sub) : 0.f;
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (valid && sub == 0) wT[(size_t)n * ld + q] = fmaf(ry.L - ry.chord, out_coef, acc);
        }
    }
}

constexpr int kAdjLanes = 4;   // lanes per ray in the adjoint
constexpr int kOrder = 2048;   // largest item count per CTA put in claim order

// Round-to-nearest int of |x| < 2^22 without a conversion instruction: adding
// 1.5 * 2^23 leaves round(x) in the low mantissa bits of the sum.
__device__ __forceinline__ int fixed_round(float x) { return __float_as_int(x + 12582912.f) - 0x4B400000; }

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

__device__ __forceinline__ float block_max(float x, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = x;
    __syncthreads();
    x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
    if (wid == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    __syncthreads();
    return x;
}

// Node column c of a padded row: the padded columns that clamp to it.
template <class T>
__device__ __forceinline__ T fold_col(const T* row, int c, int G) {
    T v = row[c + 2];
    if (c == 0) v += row[0] + row[1];
    if (c == G - 1) v += row[G + 2] + row[G + 3];
    return v;
}

// Ray adjoint.  CTA b takes the work items t = b, b + nb, b + 2 nb, ... (item =
// a patch and a block of 32 / kAdjLanes consecutive transducers), its warps
// items of different patches at the same time (rays of one patch all start at
// the same centre, where their scatters would collide).  Within a warp, groups
// of kAdjLanes lanes take the rays to consecutive transducers of one patch
// (similar lengths, so the lanes finish together); a lane walks a contiguous
// run of samples of its ray, from a staggered start, and adds each sample's
// four bilinear contributions to the shared grid.  (Keeping the current
// cell's weights in registers and adding them on cell change was measured
// slower: a cell changes every ~1.4 samples, and the branch diverges.)
//
// Coordinates are those of the padded grid (node (p, c) at (p + 2, c + 2), see
// load_excess_padded), clamped to [1, G + 2]; floor() takes no conversion
// (see excess_padded); the sums that land on the two outer rings belong to the
// edge nodes they replicate and are folded onto them when the grid is written.
//
// The shared grid holds 32-bit fixed-point sums (shared-memory integer atomics
// are single instructions; float ones are compare-and-swap loops), which also
// makes the result independent of the order of the additions.  Every
// contribution is g h_s v0 / v^2 times a bilinear weight; v is a convex
// combination of node values, so v >= vmin, and the weights h_s of a ray add up
// to its chord <= 2 mask_r.  The absolute sum of all contributions of the CTA
// is therefore at most  Mb = sum_r |g_r| 2 mask_r v0 / vmin^2 , and one
// contribution at most  F = max|g| h v0 / vmin^2.  The scale
// S = 0.99 min(2^30 / Mb, 2^22 / F) keeps every node's sum inside the int32
// range (each addition rounds by at most 1/2) and every added value below 2^22
// (rounded without a conversion instruction).  A non-finite bound (NaN in
// dL/dw or the SOS, or SOS <= 0) turns the CTA's partial grid into NaN.
//
// The padded grid is processed in bands of R cell rows (padded node rows
// r0 .. r0 + R), so that the excess rows and the accumulator of a band fit in
// shared memory for every G <= 512; a ray visits each band with the samples
// whose cell row lies in it.  Node row r0 + R is shared with the next band: its
// sums move to that band's first row.  Every CTA writes its own partial grid;
// one fixed-order kernel sums them.  (Clusters of four CTAs summing their grids
// through distributed shared memory were measured slower: fewer SMs in use and
// the cluster barriers per band.)
// ONE: the padded grid fits in one band (no per-sample band test).  NARROW:
// every sample inside the mask disk has padded node coordinates in [1, G + 2]
// (no clamps; the host checks it, as for the padded forward kernel).
template <bool ONE, bool NARROW>
__global__ void __launch_bounds__(1024, 1) rays_adj_kernel(const RayArgs a, int R, int nbands) {
    extern __shared__ float sm[];
    __shared__ float red_s[32];
    __shared__ float scale_s[2];      // S and 1/S (NaN: poisoned)
    __shared__ int next_s;            // next unclaimed item of the band
    const int G = a.g.G, pitch = pad_pitch(G), PG = G + 4;
    float* dv_s = sm;                                              // [R + 1][pitch] padded excess rows
    int* acc_s = reinterpret_cast<int*>(sm + (R + 1) * pitch);      // [R + 1][pitch] padded sums
    int* edge_s = acc_s + (R + 1) * pitch;                          // [2][G] sums of the first / last node row
    float* cost_s = reinterpret_cast<float*>(edge_s + 2 * G);       // [kOrder] item costs, then
    int* order_s = reinterpret_cast<int*>(cost_s + kOrder);         // [kOrder] items, longest first
    const float v0 = a.g.v0, h = a.g.h;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int L = kAdjLanes, RB = 32 / L;
    const int n_t = a.g.n_t, nblk = (n_t + RB - 1) / RB, nb = gridDim.x;
    const int items = a.N * nblk;                                  // (patch, block of RB transducers)
    const int mine = items > (int)blockIdx.x ? (items - (int)blockIdx.x + nb - 1) / nb : 0;   // items of this CTA
    pdl_trigger();

    // claim order: the CTA's items by decreasing estimated length (the chord
    // through the mask toward the item's middle transducer), so that the last
    // claims are short and the warps finish together
    const bool sorted = mine <= kOrder;
    if (sorted) {
        int np2 = 1;
        while (np2 < mine) np2 <<= 1;
        for (int j = threadIdx.x; j < np2; j += blockDim.x) {
            float c = -1.f;
            if (j < mine) {
                const int t = (int)blockIdx.x + nb * j, i = t / nblk, n = min((t - i * nblk) * RB + RB / 2, n_t - 1);
                const int2 cc = a.centres[i];
                c = make_ray(a.g, pixel_xy(a.g, cc.x, cc.y), n).chord;
            }
            cost_s[j] = c;
            order_s[j] = j;
        }
        __syncthreads();
        for (int k = 2; k <= np2; k <<= 1)              // bitonic sort, descending
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int x = threadIdx.x; x < np2; x += blockDim.x) {
                    const int y = x ^ jj;
                    if (y > x) {
                        const bool desc = (x & k) == 0;
                        const float cx = cost_s[x], cy = cost_s[y];
                        if (desc ? cx < cy : cx > cy) {
                            cost_s[x] = cy;
                            cost_s[y] = cx;
                            const int o = order_s[x];
                            order_s[x] = order_s[y];
                            order_s[y] = o;
                        }
                    }
                }
                __syncthreads();
            }
    }
    // everything below reads or writes what earlier kernels produce (dL/dw, the
    // SOS, the partial grids): wait for them (no-op without a dependent launch)
    pdl_wait();

    // fixed-point scale of this CTA
    float gsum = 0.f, gmax = 0.f, vmin = INFINITY, bad = 0.f;
    for (int q = threadIdx.x; q < mine * RB; q += blockDim.x) {
        const int t = (int)blockIdx.x + nb * (q / RB), i = t / nblk, n = (t - i * nblk) * RB + q % RB;
        const float gv = n < n_t ? fabsf(a.dLdw[(size_t)i * n_t + n]) : 0.f;
        gsum += gv;
        gmax = fmaxf(gmax, gv);
    }
    // band b's padded excess rows r0 .. r0 + rows - 1 into dv_s (raw values by
    // asynchronous copies, then v - v0 in place); those of a one-band grid also
    // give the minimum SOS
    auto stage = [&](int r0, int rows, bool track) {
        stage_padded_async(dv_s, a.sos, G, r0, rows);
        cp_async_wait_all();
        __syncthreads();
        for (int pl = warp; pl < rows; pl += nw)
            for (int cc = lane; cc < PG; cc += 32) {
                const float v = dv_s[pl * pitch + cc];
                if (track) {
                    if (!(v > 0.f) || !isfinite(v)) bad = 1.f;
                    vmin = fminf(vmin, v);
                }
                dv_s[pl * pitch + cc] = v - v0;
            }
    };
    stage(0, min(R + 1, PG), nbands == 1);
    if (nbands > 1)
        for (int q = threadIdx.x; q < G * G; q += blockDim.x) {
            const float v = __ldg(a.sos + q);
            if (!(v > 0.f) || !isfinite(v)) bad = 1.f;
            vmin = fminf(vmin, v);
        }
    for (int q = threadIdx.x; q < 2 * G; q += blockDim.x) edge_s[q] = 0;
    gsum = block_sum(gsum, red_s);
    gmax = block_max(gmax, red_s);
    bad = block_sum(bad, red_s);
    vmin = block_min(vmin, red_s);
    if (threadIdx.x == 0) {
        const float vm = vmin * (1.f - 1e-5f);
        const float k = v0 / (vm * vm);
        const float Mb = gsum * (2.f * a.g.mask_r) * k;
        const float F = gmax * h * k;
        const bool poison = bad > 0.f || !isfinite(Mb) || !isfinite(F) || !isfinite(gsum);
        const float S = (Mb > 0.f && F > 0.f) ? 0.99f * fminf(fminf(1073741824.f / Mb, 4194304.f / F), 1e30f) : 0.f;
        scale_s[0] = poison ? 0.f : S;
        scale_s[1] = poison ? __int_as_float(0x7fc00000) : (S > 0.f ? 1.f / S : 0.f);
    }
    __syncthreads();
    const float S = scale_s[0];

    const int sub = lane % L, grp = lane / L;
    for (int band = 0; band < nbands; ++band) {
        const bool last_band = band == nbands - 1;
        const int r0 = band * R;
        const int r1 = last_band ? G + 3 : r0 + R;        // padded cell rows r0 <= iy < r1
        const int rows = min(R + 1, PG - r0);             // padded node rows r0 .. r0 + rows - 1
        if (band > 0) stage(r0, rows, false);
        for (int q = threadIdx.x + (band > 0 ? pitch : 0); q < rows * pitch; q += blockDim.x) acc_s[q] = 0;
        if (threadIdx.x == 0) next_s = nw;
        __syncthreads();
        // warp w starts on the CTA's item j = w and then claims the next free one
        // (item t = b + nb j: the concurrent warps of a CTA work on different
        // patches); group grp of L
        // lanes takes transducer blk RB + grp, each lane a contiguous run of the
        // ray's samples in this band, started at an offset that grows with grp
        // (the RB rays of a warp leave the same centre in neighbouring directions:
        // staggered, their lanes are never at the same place at the same time)
        for (int j = warp; j < mine;) {
            const int t = (int)blockIdx.x + nb * (sorted ? order_s[j] : j), i = t / nblk, n = (t - i * nblk) * RB + grp;
            const float gr = n < n_t ? a.dLdw[(size_t)i * n_t + n] : 0.f;
            if (gr != 0.f) {
                const int2 cc = a.centres[i];
                const Ray ry = make_ray(a.g, pixel_xy(a.g, cc.x, cc.y), n);
                const float hbx = h * ry.bx, hby = h * ry.by;
                const float ax = ry.ax + 2.f, ay = ry.ay + 2.f;
                // the last cell's four corner excesses: consecutive samples of a run
                // are half a cell apart and often share a cell, whose corners then
                // need no second load (lanes that skip it add no shared traffic)
                int cell = -1;
                float d00 = 0.f, d01 = 0.f, d10 = 0.f, d11 = 0.f;
                // one midpoint sample at ray parameter u (in steps), its weight
                // (step length x dL/dw x v0 x S) given: dw/dv = weight / v^2, spread
                // bilinearly over the four nodes as fixed-point integers
                auto sample = [&](float u, float gsc) {
                    float x = fmaf(u, hbx, ax), y = fmaf(u, hby, ay);
                    if (!NARROW) {      // clamped to the padded grid: the edge-clamped interpolation
                        x = fminf(fmaxf(x, 1.f), (float)(G + 2));
                        y = fminf(fmaxf(y, 1.f), (float)(G + 2));
                    }
                    const float tY = y + 8388607.5f;
                    const int iy = __float_as_int(tY) - 0x4B000000;
                    if (!ONE && (iy < r0 || iy >= r1)) return;
                    const float tX = x + 8388607.5f;
                    const int ix = __float_as_int(tX) - 0x4B000000;
                    const float tx = x - (tX - 8388608.f), ty = y - (tY - 8388608.f);
                    const int idx = (ONE ? iy : iy - r0) * pitch + ix;
                    if (idx != cell) {
                        const float* q = dv_s + idx;
                        d00 = q[0];
                        d01 = q[1];
                        d10 = q[pitch];
                        d11 = q[pitch + 1];
                        cell = idx;
                    }
                    const float top = fmaf(tx, d01 - d00, d00), bot = fmaf(tx, d11 - d10, d10);
                    const float d = fmaf(ty, bot - top, top);
                    const float iv = __fdividef(1.f, v0 + d);
                    const float coef = gsc * iv * iv;
                    const float cy1 = coef * ty, cy0 = coef - cy1;
                    const float c01 = cy0 * tx, c11 = cy1 * tx;
                    int* acc = acc_s + idx;
                    atomicAdd(acc, fixed_round(cy0 - c01));
                    atomicAdd(acc + 1, fixed_round(c01));
                    atomicAdd(acc + pitch, fixed_round(cy1 - c11));
                    atomicAdd(acc + pitch + 1, fixed_round(c11));
                };
                // full samples m = 0 .. nfull - 1 at u = m + 1/2, in contiguous runs
                // per lane (only those whose cell row can lie in the band; the test
                // in sample() is exact, this range only needs to contain them);
                // the partial last sample (length rem) goes to the group's last lane
                int mlo = 0, mhi = ry.nfull;
                if (!ONE && NARROW && hby != 0.f) {
                    const float inv = 1.f / hby;
                    float ma = ((float)r0 - ay) * inv - 0.5f, mb = ((float)r1 - ay) * inv - 0.5f;
                    if (r0 == 0) ma = hby > 0.f ? -INFINITY : INFINITY;
                    if (last_band) mb = hby > 0.f ? INFINITY : -INFINITY;
                    const float lo = fmaxf(fminf(ma, mb), -1e9f), hi = fminf(fmaxf(ma, mb), 1e9f);
                    mlo = max(0, (int)floorf(lo) - 2);
                    mhi = min(ry.nfull, (int)ceilf(hi) + 2);
                }
                const int per = (max(mhi - mlo, 0) + L - 1) / L;
                const int m0 = mlo + sub * per, len = max(0, min(mhi, m0 + per) - m0);
                const int off = len * grp / RB;                   // staggered start within the run
                const float gfull = gr * v0 * h * S;
                int m = m0 + off;
                float uf = m + 0.5f;
#pragma unroll 2
                for (int k = 0; k < len; ++k) {
                    const float u = uf;
                    if (++m == m0 + len) {                        // wrap to the start of the run
                        m = m0;
                        uf = m0 + 0.5f;
                    } else {
                        uf += 1.f;
                    }
                    sample(u, gfull);
                }
                if (ry.rem > 0.f && sub == L - 1)
                    sample(ry.nfull + 0.5f * (ry.rem * a.g.inv_h), gr * v0 * ry.rem * S);
            }
            // next item of this CTA: claimed dynamically, so that warps whose
            // items were short take more
            int nj = 0;
            if (lane == 0) nj = atomicAdd(&next_s, 1);
            j = __shfl_sync(0xffffffffu, nj, 0);
        }
        // padded rows written by this band: r0 .. r0 + out_rows - 1 (its last row moves to the next band);
        // rows 3 .. G are node rows 1 .. G - 2, the rest fold onto node rows 0 and G - 1
        const int out_rows = last_band ? rows : R;
        __syncthreads();
        {
            const int t_end = min(3, r0 + out_rows), b_beg = max(G + 1, r0);      // padded rows [r0, t_end), [b_beg, r0 + out_rows)
            for (int c = threadIdx.x; c < G; c += blockDim.x) {
                int top = 0, bottom = 0;
                for (int pp = r0; pp < t_end; ++pp) top += fold_col(acc_s + (pp - r0) * pitch, c, G);
                for (int pp = b_beg; pp < r0 + out_rows; ++pp) bottom += fold_col(acc_s + (pp - r0) * pitch, c, G);
                edge_s[c] += top;
                edge_s[G + c] += bottom;
            }
        }
        const int i0 = max(3, r0), i1 = min(G + 1, r0 + out_rows);    // interior padded rows [i0, i1)
        {
            const float invS = scale_s[1];
            float* dst = a.part + (size_t)blockIdx.x * G * G;
            for (int pp = i0 + warp; pp < i1; pp += nw)
                for (int c = lane; c < G; c += 32)
                    dst[(pp - 2) * G + c] = (float)fold_col(acc_s + (pp - r0) * pitch, c, G) * invS;
            __syncthreads();
        }
        if (!last_band) {
            for (int c = threadIdx.x; c < pitch; c += blockDim.x) acc_s[c] = acc_s[R * pitch + c];
            __syncthreads();
        }
    }
    // node rows 0 and G - 1
    {
        const float invS = scale_s[1];
        float* dst = a.part + (size_t)blockIdx.x * G * G;
        for (int q = threadIdx.x; q < 2 * G; q += blockDim.x)
            dst[q < G ? q : (G - 1) * G + (q - G)] = (float)edge_s[q] * invS;
    }
}

// Sum of the partial grids part[0 .. np) at the 32 consecutive nodes q0 + lane
// of this block: warp w adds the partials of its chunk [np w / nw, np (w+1) / nw)
// in order, warp 0 then adds the chunk sums in order (a fixed order, with
// np / nw loads in flight per lane instead of np).  Valid in warp 0.
__device__ __forceinline__ float sum_parts32(const float* part, int np, int GG, int q0, float* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int q = q0 + lane;
    const int r0 = np * w / nw, r1 = np * (w + 1) / nw;
    float s = 0.f;
    if (q < GG) {
        int r = r0;
        for (; r + 16 <= r1; r += 16) {          // sixteen loads in flight, added in order
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = __ldcg(part + (size_t)(r + k) * GG + q);
#pragma unroll
            for (int k = 0; k < 16; ++k) s += v[k];
        }
        for (; r < r1; ++r) s += __ldcg(part + (size_t)r * GG + q);
    }
    red[w * 32 + lane] = s;
    __syncthreads();
    float tot = 0.f;
    if (w == 0)
        for (int k = 0; k < nw; ++k) tot += red[k * 32 + lane];
    return tot;
}

// out[q] (+)= sum of the partial grids part[0 .. np)[q] (block: 32 nodes).
__global__ void __launch_bounds__(256) reduce_parts_kernel(const float* part, int np, int GG, float* out,
                                                           int accumulate) {
    __shared__ float red[256];
    pdl_trigger();
    pdl_wait();
    const int q = blockIdx.x * 32 + (threadIdx.x & 31);
    const float g = sum_parts32(part, np, GG, blockIdx.x * 32, red);
    if (threadIdx.x < 32 && q < GG) out[q] = accumulate ? out[q] + g : g;
}

// The tail of a recovery iteration (Sec. 3.3) in one launch: per node
//   g = (sum of the adjoint's partial grids, fixed order) + tv_grad (optional),
// written to grad_out (optional), then one Adam step on param in place.  The
// TV terms come from the ray forward kernel of the same iteration, taken
// before this update, so no CTA reads a node another CTA updates.  CTA 0 also
// adds the forward kernel's lambda * TV partials (fixed order) to loss.
struct TailArgs {
    const float* part;
    int np, GG;
    const float* tv_grad;
    const float* tv_part;
    int ntv;
    float* loss;
    float* grad_out;
    float* param;
    float* m;
    float* v;
    float lr, b1, b2, eps, bc1, bc2;
    int* counter;                 // [2] as pact_adam_step's step counter, or NULL (bc1, bc2 fixed)
    const unsigned char* mask;
};

__global__ void __launch_bounds__(256) adj_adam_kernel(const TailArgs a) {
    __shared__ float red[256];
    pdl_trigger();
    pdl_wait();
    float bc1 = a.bc1, bc2 = a.bc2;
    if (a.counter) {              // t = steps so far + 1
        const float t = (float)(a.counter[0] + 1);
        bc1 = 1.f - powf(a.b1, t);
        bc2 = 1.f - powf(a.b2, t);
    }
    const int q = blockIdx.x * 32 + (threadIdx.x & 31);
    const bool mine = threadIdx.x < 32 && q < a.GG;
    // this node's Adam operands first: their loads overlap the partial-grid sum
    float m0 = 0.f, v0 = 0.f, p0 = 0.f, tg = 0.f;
    bool train = false;
    if (mine) {
        train = !a.mask || a.mask[q];
        tg = a.tv_grad ? a.tv_grad[q] : 0.f;
        if (train) {
            m0 = a.m[q];
            v0 = a.v[q];
            p0 = a.param[q];
        }
    }
    float g = sum_parts32(a.part, a.np, a.GG, blockIdx.x * 32, red);
    if (mine) {
        g += tg;
        if (a.grad_out) a.grad_out[q] = g;
        if (train) {
            const float mq = fmaf(a.b1, m0, (1.f - a.b1) * g);
            const float vq = fmaf(a.b2, v0, (1.f - a.b2) * g * g);
            a.m[q] = mq;
            a.v[q] = vq;
            a.param[q] = p0 - a.lr * (mq / bc1) / (sqrtf(vq / bc2) + a.eps);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 32 && a.loss && a.tv_part) {   // warp 0: loads in parallel,
        float s = 0.f;                                                        // a fixed-order butterfly
        for (int k = threadIdx.x; k < a.ntv; k += 32) s += a.tv_part[k];
        s = warp_sum(s);
        if (threadIdx.x == 0) a.loss[0] += s;
    }
    if (a.counter) {
        // every thread of the CTA has used its read of counter[0] before this
        // barrier, and nothing else in the kernel depends on the counter, so
        // the completion count needs no fence
        __syncthreads();
        if (threadIdx.x == 0) {
            if (atomicAdd(a.counter + 1, 1) == (int)gridDim.x - 1) {   // all CTAs have read it
                a.counter[0] += 1;
                a.counter[1] = 0;
            }
        }
    }
}

constexpr size_t kMaxSmem = 200 * 1024;
constexpr int kTvParts = 4096;    // per-CTA TV partials the TV workspace holds


constexpr int kRayLanes = 1;   // lanes per ray in the forward integrals

enum FwdMode { kFwdGlobal = 0, kFwdShared = 1, kFwdPadded = 2 };

// Staging of the SOS excess for the forward integrals: padded (no clamps) when
// every sample inside the mask disk has node coordinates in [-1, G] and the
// padded grid fits, else the plain shared grid, else global memory.
// Every sample inside the mask disk has node coordinates in [-1, G] (padded
// coordinates in [1, G + 2]).
bool hull_ok(const pact_geometry* g) { return g->mask_radius <= (0.5f * g->sos_g + 0.5f) * g->sos_dx; }

int fwd_mode(const pact_geometry* g, size_t* bytes) {
    const int G = g->sos_g;
    if (hull_ok(g) && pad_bytes(G) <= kMaxSmem) {
        *bytes = pad_bytes(G);
        return kFwdPadded;
    }
    const size_t plain = (size_t)G * smem_pitch(G) * sizeof(float);
    if (plain <= kMaxSmem) {
        *bytes = plain;
        return kFwdShared;
    }
    *bytes = 0;
    return kFwdGlobal;
}

const void* fwd_fn(int mode) {
    return mode == kFwdPadded   ? (const void*)rays_fwd_kernel<kRayLanes, true, true>
           : mode == kFwdShared ? (const void*)rays_fwd_kernel<kRayLanes, true, false>
                                : (const void*)rays_fwd_kernel<kRayLanes, false, false>;
}

// Persistent grid: as many CTAs of `threads` as fit on the device at once.
int persistent_grid(const void* fn, int threads, size_t smem) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return num_sms() * per_sm;
}

struct Plan {
    int fwd_mode, nb_fwd;
    int R, nbands, nb_adj, nparts;
    bool narrow;
    size_t smem_fwd, smem_adj, ws;
};

Plan make_plan(const pact_geometry* g, const pact_patches* pt) {
    Plan p;
    const int G = g->sos_g;
    p.fwd_mode = fwd_mode(g, &p.smem_fwd);
    {
        constexpr int RB = 32 / kRayLanes;
        const int items = pt->n * ((g->n_t + RB - 1) / RB);          // warp work items
        p.nb_fwd = std::max(1, std::min(persistent_grid(fwd_fn(p.fwd_mode), 512, p.smem_fwd), (items + 15) / 16));
    }
    // adjoint: bands of R cell rows of the padded grid (G + 3 cell rows, row pitch
    // pad_pitch(G)); excess rows, accumulator and the two edge rows in shared memory
    const int pp = pad_pitch(G);
    const size_t edge = 2 * sizeof(int) * (size_t)G + 2 * sizeof(int) * (size_t)kOrder;   // + claim order
    p.R = std::max(1, std::min(G + 3, (int)((kMaxSmem - edge) / (2 * sizeof(float) * (size_t)pp)) - 1));
    p.nbands = (G + 3 + p.R - 1) / p.R;
    p.smem_adj = 2 * sizeof(float) * (size_t)(p.R + 1) * pp + edge;
    p.narrow = hull_ok(g);
    const int nrays = pt->n * g->n_t;
    const int want = std::max(1, std::min(num_sms(), (nrays + 31) / 32));   // one persistent CTA per SM
    p.nb_adj = want;
    p.nparts = p.nb_adj;
    p.ws = align_up((size_t)p.nparts * G * G * sizeof(float), 256);
    return p;
}

RayArgs make_args(const pact_geometry* g, const pact_patches* pt, const Plan& pl, const float* sos) {
    RayArgs a = {};
    a.g = make_geo(g);
    a.N = pt->n;
    a.centres = reinterpret_cast<const int2*>(pt->centres);
    a.sos = sos;
    a.w = nullptr;
    a.dLdw = nullptr;
    a.part = nullptr;
    a.out = nullptr;
    a.use_smem = pl.fwd_mode != kFwdGlobal;
    return a;
}

}  // namespace

pact_status launch_pixel_rays(const pact_geometry* g, const float* sos, const float* p0, int pix0, int npix,
                              float* wT, int ld, cudaStream_t st) {
    if (npix <= 0) return PACT_OK;
    PACT_TRY(require_sms());
    size_t smem = 0;
    const int mode = fwd_mode(g, &smem);
    const void* fn = mode == kFwdPadded   ? (const void*)rays_pix_kernel<kRayLanes, true, true>
                     : mode == kFwdShared ? (const void*)rays_pix_kernel<kRayLanes, true, false>
                                          : (const void*)rays_pix_kernel<kRayLanes, false, false>;
    if (smem) PACT_TRY(ensure_smem(fn, smem, "rf_synth: shared memory attribute"));
    const int grid = std::min(npix, persistent_grid(fn, 512, smem));
    RayArgs a = {};
    a.g = make_geo(g);
    a.N = 0;
    a.sos = sos;
    a.use_smem = mode != kFwdGlobal;
    if (mode == kFwdPadded)
        rays_pix_kernel<kRayLanes, true, true><<<grid, 512, smem, st>>>(a, p0, pix0, npix, wT, ld);
    else if (mode == kFwdShared)
        rays_pix_kernel<kRayLanes, true, false><<<grid, 512, smem, st>>>(a, p0, pix0, npix, wT, ld);
    else
        rays_pix_kernel<kRayLanes, false, false><<<grid, 512, 0, st>>>(a, p0, pix0, npix, wT, ld);
    return check_launch("rf_synth: ray kernel");
}

}  // namespace pact

using namespace pact;

static pact_status sos_to_delays(const pact_geometry* g, const pact_patches* pt, const float* sos, float* w,
                                 float* clear, size_t n_clear, void* stream, float tv_lambda = 0.f,
                                 void* tv_ws = nullptr, size_t tv_ws_bytes = 0) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!sos || !w) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays: sos and w must not be NULL");
    if (n_clear && (!clear || reinterpret_cast<uintptr_t>(clear) % 16 || n_clear % 4))
        return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_clear: clear must be 16-byte aligned, n_clear a multiple of 4");
    const size_t GG = (size_t)g->sos_g * g->sos_g;
    if (tv_ws) {
        if (reinterpret_cast<uintptr_t>(tv_ws) % 256) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_tv: tv_ws must be 256-byte aligned");
        if (tv_ws_bytes < (GG + kTvParts) * sizeof(float))
            return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_tv: tv_ws too small: %zu < %zu bytes", tv_ws_bytes,
                        (GG + kTvParts) * sizeof(float));
        if (!std::isfinite(tv_lambda)) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_tv: lambda must be finite");
    }
    PACT_TRY(require_sms());
    const Plan pl = make_plan(g, pt);
    if (tv_ws && pl.nb_fwd > kTvParts) return fail(PACT_ERR_UNSUPPORTED, "sos_to_delays_tv: %d CTAs", pl.nb_fwd);
    RayArgs a = make_args(g, pt, pl, sos);
    a.w = w;
    a.clear = reinterpret_cast<float4*>(clear);
    a.n_clear4 = n_clear / 4;
    if (tv_ws) {
        a.tv_lambda = tv_lambda;
        a.tv_grad = static_cast<float*>(tv_ws);
        a.tv_part = static_cast<float*>(tv_ws) + GG;
    }
    cudaStream_t st = as_stream(stream);
    if (pl.smem_fwd)
        PACT_TRY(ensure_smem(fwd_fn(pl.fwd_mode), pl.smem_fwd, "sos_to_delays: shared memory attribute"));
    if (pl.fwd_mode == kFwdPadded)
        rays_fwd_kernel<kRayLanes, true, true><<<pl.nb_fwd, 512, pl.smem_fwd, st>>>(a);
    else if (pl.fwd_mode == kFwdShared)
        rays_fwd_kernel<kRayLanes, true, false><<<pl.nb_fwd, 512, pl.smem_fwd, st>>>(a);
    else
        rays_fwd_kernel<kRayLanes, false, false><<<pl.nb_fwd, 512, 0, st>>>(a);
    return check_launch("sos_to_delays kernel");
}

extern "C" pact_status pact_sos_to_delays(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                          float* w, void* stream) {
    return sos_to_delays(g, pt, sos, w, nullptr, 0, stream);
}

extern "C" pact_status pact_sos_to_delays_clear(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                                float* w, float* clear, size_t n_clear, void* stream) {
    return sos_to_delays(g, pt, sos, w, clear, n_clear, stream);
}

extern "C" size_t pact_sos_to_delays_tv_workspace_size(const pact_geometry* g, const pact_patches* pt) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK) return 0;
    return align_up(((size_t)g->sos_g * g->sos_g + kTvParts) * sizeof(float), 256);
}

extern "C" pact_status pact_sos_to_delays_tv(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                             float* w, float* clear, size_t n_clear, float lambda, void* tv_ws,
                                             size_t tv_ws_bytes, void* stream) {
    if (!tv_ws) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_tv: tv_ws is NULL");
    return sos_to_delays(g, pt, sos, w, clear, n_clear, stream, lambda, tv_ws, tv_ws_bytes);
}

extern "C" size_t pact_sos_to_delays_adj_workspace_size(const pact_geometry* g, const pact_patches* pt) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK) return 0;
    if (require_sms() != PACT_OK) {              // no device to ask: enough for any GPU of up to 256 SMs
        const int nrays = pt->n * g->n_t;
        const size_t parts = (size_t)std::max(1, std::min(256, (nrays + 31) / 32));
        return align_up(parts * g->sos_g * g->sos_g * sizeof(float), 256);
    }
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
    PACT_TRY(require_sms());                       // the plan's grid (and workspace) follow the SM count
    const Plan pl = make_plan(g, pt);
    if (ws_bytes < pl.ws) return fail(PACT_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, pl.ws);
    cudaStream_t st = as_stream(stream);
    const int GG = g->sos_g * g->sos_g;
    RayArgs a = make_args(g, pt, pl, sos);
    a.dLdw = dL_dw;
    a.part = static_cast<float*>(ws);
    a.out = dL_dsos;
    auto adj = pl.nbands == 1 ? (pl.narrow ? rays_adj_kernel<true, true> : rays_adj_kernel<true, false>)
                              : (pl.narrow ? rays_adj_kernel<false, true> : rays_adj_kernel<false, false>);
    PACT_TRY(ensure_smem((const void*)adj, pl.smem_adj, "sos_to_delays_adj: shared memory attribute"));
    if (launch_pdl(adj, dim3(pl.nb_adj), dim3(1024), pl.smem_adj, st, a, pl.R, pl.nbands) != cudaSuccess)
        return check_launch("sos_to_delays_adj kernel");
    PACT_TRY(check_launch("sos_to_delays_adj kernel"));
    // one partial grid per CTA: a single fixed-order sum
    if (launch_pdl(reduce_parts_kernel, dim3((GG + 31) / 32), dim3(256), 0, st, a.part, pl.nparts, GG, dL_dsos,
                   accumulate) != cudaSuccess)
        return check_launch("sos_to_delays_adj reduction");
    return check_launch("sos_to_delays_adj reduction");
}

extern "C" pact_status pact_sos_to_delays_adj_adam(const pact_geometry* g, const pact_patches* pt, float* sos,
                                                   const float* dL_dw, const void* tv_ws, float* loss, float* dL_dsos,
                                                   float* m, float* v, int step, int* step_counter, float lr,
                                                   float beta1, float beta2, float eps, const unsigned char* mask,
                                                   void* ws, size_t ws_bytes, void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!sos || !dL_dw || !m || !v)
        return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj_adam: sos, dL_dw, m and v must not be NULL");
    if (!step_counter && step < 1) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj_adam: step must be >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f))
        return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj_adam: betas must be in [0, 1)");
    if (!ws) return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj_adam: workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (tv_ws && reinterpret_cast<uintptr_t>(tv_ws) % 256)
        return fail(PACT_ERR_INVALID_ARG, "sos_to_delays_adj_adam: tv_ws must be 256-byte aligned");
    PACT_TRY(require_sms());
    const Plan pl = make_plan(g, pt);
    if (ws_bytes < pl.ws) return fail(PACT_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, pl.ws);
    if (tv_ws && pl.nb_fwd > kTvParts) return fail(PACT_ERR_UNSUPPORTED, "sos_to_delays_adj_adam: %d CTAs", pl.nb_fwd);
    cudaStream_t st = as_stream(stream);
    const int GG = g->sos_g * g->sos_g;
    RayArgs a = make_args(g, pt, pl, sos);
    a.dLdw = dL_dw;
    a.part = static_cast<float*>(ws);
    auto adj = pl.nbands == 1 ? (pl.narrow ? rays_adj_kernel<true, true> : rays_adj_kernel<true, false>)
                              : (pl.narrow ? rays_adj_kernel<false, true> : rays_adj_kernel<false, false>);
    PACT_TRY(ensure_smem((const void*)adj, pl.smem_adj, "sos_to_delays_adj_adam: shared memory attribute"));
    if (launch_pdl(adj, dim3(pl.nb_adj), dim3(1024), pl.smem_adj, st, a, pl.R, pl.nbands) != cudaSuccess)
        return check_launch("sos_to_delays_adj_adam: adjoint kernel");
    PACT_TRY(check_launch("sos_to_delays_adj_adam: adjoint kernel"));
    TailArgs t;
    t.part = a.part;
    t.np = pl.nparts;
    t.GG = GG;
    t.tv_grad = tv_ws ? static_cast<const float*>(tv_ws) : nullptr;
    t.tv_part = tv_ws ? static_cast<const float*>(tv_ws) + GG : nullptr;
    t.ntv = pl.nb_fwd;
    t.loss = loss;
    t.grad_out = dL_dsos;
    t.param = sos;
    t.m = m;
    t.v = v;
    t.lr = lr;
    t.b1 = beta1;
    t.b2 = beta2;
    t.eps = eps;
    const int s1 = step < 1 ? 1 : step;
    t.bc1 = (float)(1.0 - pow((double)beta1, s1));
    t.bc2 = (float)(1.0 - pow((double)beta2, s1));
    t.counter = step_counter;
    t.mask = mask;
    if (launch_pdl(adj_adam_kernel, dim3((GG + 31) / 32), dim3(256), 0, st, t) != cudaSuccess)
        return check_launch("sos_to_delays_adj_adam: tail kernel");
    return check_launch("sos_to_delays_adj_adam: tail kernel");
}
