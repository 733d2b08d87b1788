// Warm-start CNN on the fifth-generation tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in tensor memory).  The paper recovers the SOS by
// test-time optimisation alone (Sec. 3.3); this network is a learned addition
// that predicts a starting SOS map from the delay stack, trained on stacks the
// forward model (Eq. 5) generates from random SOS fields.
//
// Architecture (fixed; M = delay channels, padded to Cp = 16 or 32 or 64):
//   x  = pool4(stack) / rms            [B][R][R][Cp]     R = img / 4
//   h1 = relu(conv3x3(x;  W1, b1))     32 ch at R,   2x2 mean -> R/2
//   h2 = relu(conv3x3(.;  W2, b2))     64 ch at R/2, 2x2 mean -> R/4
//   h3..h5 = relu(conv3x3(.; W3..W5))  64 ch at R/4
//   z  = w6 . h5 + b6,  v32 = v_mid + v_half tanh(z)          [B][R/4][R/4]
//   sos = bilinear x4 (v32) on the mask, v_bg outside         [B][G][G], G = R
// Activations are NHWC BF16; every 3x3 convolution is an implicit GEMM:
//   forward  Z[p][co] = sum_tap sum_ci X[p + off(tap)][ci] W[co][ci][tap]
//   dgrad    dX[p][ci] = sum_tap sum_co dZ[p - off(tap)][co] W[co][ci][tap]
//   wgrad    dW[co][ci][tap] = sum_p X[p + off(tap)][ci] dZ[p][co]
// The first two run in conv_kernel (M = 128 pixels, N = output channels, K =
// input channels per tap, operands K-major); the third in wgrad_kernel with
// both operands MN-major (rows = (tap, ci) or co, K = pixels), so that every
// operand tile is gathered with 16-byte copies straight from NHWC tensors.
#include <cuda_bf16.h>

#include <algorithm>

#include "pact_internal.cuh"
#include "umma.cuh"

namespace pact {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kConvStages = 3;
constexpr int kWgPix = 64;          // pixels (K) per wgrad stage
constexpr int kWgStages = 3;
constexpr int kWgChunk = 4096;      // largest pixel chunk per wgrad CTA
constexpr int kWgMinChunk = 512;    // smallest (a multiple of kWgPix)
constexpr int kWgTargetCtas = 304;  // chunks x tap groups aimed for: two CTAs per SM of a 152-SM GPU
constexpr int kNumConv = 5;
constexpr int kHid = 64;            // channels of h3..h5 (head input)

// -------------------------------------------------------------- small helpers

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

using umma::idesc_bf16_mn;
using umma::mn_slice;
using umma::mnmaj_off;

__device__ __forceinline__ bool wait_or_flag(uint64_t* bar, uint32_t parity, int* status, unsigned long long limit) {
    const bool ok = mbar_wait_bounded(bar, parity, limit);
    if (!ok) atomicExch(status, 1);
    return ok;
}

__device__ __forceinline__ uint32_t tmem_cols(int n) { return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : 256u; }

// -------------------------------------------------------------- 3x3 convolution (forward / dgrad)

struct ConvArgs {
    const bf16* in;        // [P][K] NHWC gathered operand (x for forward, dZ for dgrad)
    const bf16* wpk;       // [9][N][K] packed weights, each tap a K-major N x K tile image
    const float* bias;     // [N] or NULL
    const bf16* mask;      // [P][N] or NULL: output multiplied by (mask > 0) (ReLU backward)
    bf16* out;             // [P][N]
    int B, H, W, K, N;
    int sign;              // +1: tap offset (dy - 1, dx - 1); -1: its negative (dgrad)
    int relu;
    int* status;
    unsigned long long limit_ns;   // bound on every tensor-core wait (pact_set_wait_limit_ns)
};

// CTA: 128 consecutive pixels p = (b H + y) W + x, all N output channels.
// Per tap, the 128 x K input rows (zero outside the image) and the N x K weight
// tile are gathered by cp.async into a stage of a 3-deep ring; one thread
// issues K/16 MMAs per tap and commits them to the stage's mbarrier.
__global__ void __launch_bounds__(128) conv_kernel(const ConvArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int K = a.K, N = a.N;
    const uint32_t a_bytes = 128u * (uint32_t)K * 2u, b_bytes = (uint32_t)N * (uint32_t)K * 2u;
    unsigned char* As[kConvStages];
    unsigned char* Bs[kConvStages];
    for (int s = 0; s < kConvStages; ++s) {
        As[s] = sm + s * (a_bytes + b_bytes);
        Bs[s] = As[s] + a_bytes;
    }
    __shared__ __align__(8) uint64_t done[kConvStages];
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int P = a.B * a.H * a.W;
    const int p = blockIdx.x * 128 + tid;
    const bool pvalid = p < P;
    const uint32_t ncols = tmem_cols(N);
    // Gather mapping: element e = tid + 128 it of the 128 pixels x K/8 16-byte
    // chunks, pixel-fastest in groups of eight (pixel 8 ph + pl, chunk c8): each
    // 8-thread phase writes 128 contiguous bytes of the K-major tile, and each
    // warp reads whole pixel rows.  A thread's pixels and their image
    // coordinates are the same for all nine taps.
    const int K8 = K / 8, nit = K8;                 // 128 * K8 elements, 128 threads
    const int pl = tid & 7, c8 = (tid >> 3) % K8, ph0 = (tid >> 3) / K8, ph_step = 16 / K8;
    int gx[8], gy[8], gp[8];                        // K8 <= 8 (K <= 64)
    const float invW = 1.f / (float)a.W, invH = 1.f / (float)a.H;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        if (it >= nit) break;
        const int q = blockIdx.x * 128 + 8 * (ph0 + it * ph_step) + pl;
        const int r = (int)(((float)q + 0.5f) * invW);      // q / W (exact: q + W < 2^22)
        gx[it] = q - r * a.W;
        gy[it] = r - (int)(((float)r + 0.5f) * invH) * a.H;
        gp[it] = q < P ? q : -1;
    }

    if (warp == 0) umma::tmem_alloc(&tmem_s, ncols);
    if (tid == 0) {
        for (int s = 0; s < kConvStages; ++s) mbar_init(&done[s], 1);
        mbar_init_fence();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tmem_s;

    auto gather = [&](int tap, int s) {
        const int oy = a.sign * (tap / 3 - 1), ox = a.sign * (tap % 3 - 1);
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            if (it >= nit) break;
            const int ys = gy[it] + oy, xs = gx[it] + ox;
            const bool ok = gp[it] >= 0 && ys >= 0 && ys < a.H && xs >= 0 && xs < a.W;
            const bf16* src = a.in + (size_t)(ok ? gp[it] + oy * a.W + ox : 0) * K + 8 * c8;
            const int pix = 8 * (ph0 + it * ph_step) + pl;
            cp_async16(As[s] + umma::kmaj_off(pix, 8 * c8, K), src, ok);
        }
        const bf16* wt = a.wpk + (size_t)tap * N * K;
        for (int c = tid; c < N * K / 8; c += 128) cp_async16(Bs[s] + 16 * c, wt + 8 * c, true);
        cp_async_commit();
    };

    bool ok = true;
    gather(0, 0);
    gather(1, 1);
    const uint32_t idesc = umma::idesc_bf16(128, N);
    for (int t = 0; t < 9; ++t) {
        const int s = t % kConvStages;
        if (t < 8) cp_async_wait<1>(); else cp_async_wait<0>();
        umma::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after();
            for (int kk = 0; kk < K / 16; ++kk)
                umma::mma(tmem, umma::kslice(As[s], K, kk), umma::kslice(Bs[s], K, kk), idesc, t > 0 || kk > 0);
            umma::commit(&done[s]);
        }
        const int tn = t + 2;
        if (tn < 9) {
            const int sn = tn % kConvStages;
            if (tn >= kConvStages)    // the MMAs of tap tn - 3 read stage sn
                ok = wait_or_flag(&done[sn], (uint32_t)(((tn - kConvStages) / kConvStages) & 1), a.status, a.limit_ns) && ok;
            gather(tn, sn);
        }
    }
    ok = wait_or_flag(&done[8 % kConvStages], (uint32_t)((8 / kConvStages) & 1), a.status, a.limit_ns) && ok;
    umma::fence_after();
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < N; c0 += 32) {
        float v[32];
        umma::ld32(tmem + lane_base + c0, v);
        if (!pvalid) continue;
        __align__(16) bf16 o[32];
        const bf16* mk = a.mask ? a.mask + (size_t)p * N + c0 : nullptr;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float h = v[j] + (a.bias ? __ldg(a.bias + c0 + j) : 0.f);
            if (a.relu) h = fmaxf(h, 0.f);
            if (mk && !(__bfloat162float(mk[j]) > 0.f)) h = 0.f;
            o[j] = __float2bfloat16_rn(ok ? h : __int_as_float(0x7fc00000));
        }
        uint4* dst = reinterpret_cast<uint4*>(a.out + (size_t)p * N + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// -------------------------------------------------------------- weight gradient

struct WgradArgs {
    const bf16* x;         // [P][Cin] layer input (NHWC)
    const bf16* dz;        // [P][Cout] gradient at the pre-activation
    float* part;           // [nchunks][groups][128][Cout] partial sums
    int B, H, W, Cin, Cout;
    int taps_per_group;    // 128 / Cin
    int chunk;             // pixels per CTA (a multiple of kWgPix)
    int* status;
    unsigned long long limit_ns;   // bound on every tensor-core wait (pact_set_wait_limit_ns)
};

// CTA (chunk, group): pixels [chunk*4096, +4096), rows r = tl * Cin + ci for the
// taps tap = group * taps_per_group + tl.  D[r][co] += X[p + off(tap)][ci] dZ[p][co].
// Tap slot 9 (always present: 9 is not a multiple of 128 / Cin for Cin = 16, 32
// or 64) holds a row of ones in its first row, so that D there is the bias
// gradient sum_p dZ[p][co].
__global__ void __launch_bounds__(128) wgrad_kernel(const WgradArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int Cin = a.Cin, Cout = a.Cout;
    const uint32_t a_bytes = 128u * kWgPix * 2u, b_bytes = (uint32_t)Cout * kWgPix * 2u;
    unsigned char* As[kWgStages];
    unsigned char* Bs[kWgStages];
    for (int s = 0; s < kWgStages; ++s) {
        As[s] = sm + s * (a_bytes + b_bytes);
        Bs[s] = As[s] + a_bytes;
    }
    __shared__ __align__(8) uint64_t done[kWgStages];
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int P = a.B * a.H * a.W;
    const int p0 = blockIdx.x * a.chunk;
    const int npix = min(a.chunk, P - p0);
    const int nst = (npix + kWgPix - 1) / kWgPix;
    const int group = blockIdx.y;
    const uint32_t ncols = tmem_cols(Cout);

    if (warp == 0) umma::tmem_alloc(&tmem_s, ncols);
    if (tid == 0) {
        for (int s = 0; s < kWgStages; ++s) mbar_init(&done[s], 1);
        mbar_init_fence();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tmem_s;

    // Gather mapping (the same for every stage): element e = tid + 128 it, with
    // k & 7 = e & 7 fastest, so that each 8-thread phase writes 128 contiguous
    // bytes of the MN-major tile and each warp reads whole pixel rows.
    // A (128 rows x 64 pixels): rows 8 (tid >> 3) .. +7, pixels k = 8 it + (tid & 7).
    const int kk = tid & 7, r8 = tid >> 3;
    const int tl = (8 * r8) / Cin, ci = 8 * r8 - tl * Cin;
    const int tap = group * a.taps_per_group + tl;
    const bool bias_row = tap == 9, tap_ok = tap < 9;
    const int oy = tap_ok ? tap / 3 - 1 : 0, ox = tap_ok ? tap % 3 - 1 : 0;
    const uint32_t a_off = (uint32_t)(r8 * 128 + kk * 16);     // mnmaj_off(8 r8, 8 it + kk, 128) - 2048 it
    // B (Cout rows x 64 pixels): rows 8 c8 .. +7, pixels k = 8 (kb0 + it kb_step) + kk
    const int co8 = Cout / 8, c8 = (tid >> 3) % co8, kb0 = (tid >> 3) / co8, kb_step = 16 / co8;
    const float invW = 1.f / (float)a.W, invH = 1.f / (float)a.H;
    // stage j: pixels p0 + 64 j .. +63
    auto gather = [&](int j, int s) {
        const int pbase = p0 + j * kWgPix, lim = npix - j * kWgPix;
#pragma unroll
        for (int it = 0; it < kWgPix / 8; ++it) {
            const int k = 8 * it + kk;
            const uint32_t off = a_off + (uint32_t)it * 2048u;
            const bool inpix = k < lim;
            if (bias_row) {                         // bias row: 1 at ci = 0, pixel in range
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (ci == 0 && inpix) v.x = 0x3F80u;  // bf16 1.0 in the low half
                *reinterpret_cast<uint4*>(As[s] + off) = v;
                continue;
            }
            bool ok = tap_ok && inpix;
            int src = 0;
            if (ok) {
                const int p = pbase + k;
                const int q = (int)(((float)p + 0.5f) * invW);      // p / W (exact: p + W < 2^22)
                const int x = p - q * a.W, y = q - (int)(((float)q + 0.5f) * invH) * a.H;
                ok = y + oy >= 0 && y + oy < a.H && x + ox >= 0 && x + ox < a.W;
                src = ok ? p + oy * a.W + ox : 0;
            }
            cp_async16(As[s] + off, a.x + (size_t)src * Cin + ci, ok);
        }
        for (int it = 0; it < co8 / 2; ++it) {
            const int k = 8 * (kb0 + it * kb_step) + kk;
            const bool ok = k < lim;
            cp_async16(Bs[s] + mnmaj_off(8 * c8, k, Cout), a.dz + (size_t)(ok ? pbase + k : 0) * Cout + 8 * c8, ok);
        }
        cp_async_commit();
    };

    bool ok = true;
    const uint32_t idesc = idesc_bf16_mn(128, Cout);
    gather(0, 0);
    if (nst > 1) gather(1, 1);
    for (int j = 0; j < nst; ++j) {
        const int s = j % kWgStages;
        if (j + 1 < nst) cp_async_wait<1>(); else cp_async_wait<0>();
        umma::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after();
            for (int kk = 0; kk < kWgPix / 16; ++kk)
                umma::mma(tmem, mn_slice(As[s], 128, kk), mn_slice(Bs[s], Cout, kk), idesc, j > 0 || kk > 0);
            umma::commit(&done[s]);
        }
        const int jn = j + 2;
        if (jn < nst) {
            const int sn = jn % kWgStages;
            if (jn >= kWgStages)
                ok = wait_or_flag(&done[sn], (uint32_t)(((jn - kWgStages) / kWgStages) & 1), a.status, a.limit_ns) && ok;
            gather(jn, sn);
        }
    }
    const int last = nst - 1;
    ok = wait_or_flag(&done[last % kWgStages], (uint32_t)((last / kWgStages) & 1), a.status, a.limit_ns) && ok;
    umma::fence_after();
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int groups = gridDim.y;
    float* dst = a.part + (((size_t)blockIdx.x * groups + group) * 128 + tid) * Cout;
    for (int c0 = 0; c0 < Cout; c0 += 32) {
        float v[32];
        umma::ld32(tmem + lane_base + c0, v);
#pragma unroll
        for (int q = 0; q < 32; q += 4)
            *reinterpret_cast<float4*>(dst + c0 + q) =
                ok ? make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]) : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// dW[co][ci][tap] (+)= sum over chunks of part[chunk][group][r][co] and
// db[co] (+)= the same sum at the ones row.  One thread per partial element
// (group, r, co), co fastest so that a warp reads contiguous partials; the
// chunks are summed in a fixed order (four interleaved sums, then their pairs).
// cin: channels of the parameter layout, cin_pad: rows per tap in the partials.
__global__ void wgrad_reduce_kernel(const float* part, int nchunks, int groups, int cin, int cin_pad, int Cout,
                                    int tpg, float* dW, float* db, int accumulate) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= groups * 128 * Cout) return;
    const int co = e % Cout, gr = e / Cout, r = gr % 128, group = gr / 128;
    const int tl = r / cin_pad, ci = r - tl * cin_pad, tap = group * tpg + tl;
    float* dst;
    if (tap < 9 && ci < cin) dst = dW + ((size_t)co * cin + ci) * 9 + tap;
    else if (tap == 9 && ci == 0) dst = db + co;
    else return;
    const size_t stride = (size_t)groups * 128 * Cout;
    const float* src = part + e;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    int c = 0;
    for (; c + 4 <= nchunks; c += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] += src[(size_t)(c + u) * stride];
    for (; c < nchunks; ++c) s[0] += src[(size_t)c * stride];
    const float t = (s[0] + s[1]) + (s[2] + s[3]);
    *dst = accumulate ? *dst + t : t;
}

// -------------------------------------------------------------- elementwise kernels

// pooled[b][y][x][c] = mean of the 4 x 4 block of stack[c]; also sum of squares
// (per-CTA fixed-order sums added in FP64: the result does not depend on the
// order of the atomic additions to within far less than one FP32 unit).
__global__ void pool4_kernel(const float* stack, int m, int H, int W, float* pooled, int cp, double* sumsq) {
    const int R = H / 4, C = W / 4;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    float q = 0.f;
    if (e < R * C * cp) {
        const int c = e % cp, px = (e / cp) % C, py = e / (cp * C);
        float s = 0.f;
        if (c < m)
            for (int dy = 0; dy < 4; ++dy)
                for (int dx = 0; dx < 4; ++dx) s += stack[((size_t)c * H + 4 * py + dy) * W + 4 * px + dx];
        s *= 1.f / 16.f;
        pooled[e] = s;
        q = c < m ? s * s : 0.f;
    }
    __shared__ float red[8];
    q = block_sum(q, red);
    if (threadIdx.x == 0) atomicAdd(sumsq, (double)q);
}

__global__ void scale_cast_kernel(const float* pooled, int n, const double* sumsq, float count, bf16* x) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float rms = sqrtf((float)(*sumsq / (double)count));
    x[e] = __float2bfloat16_rn(pooled[e] / (rms + 1e-12f));
}

// 2 x 2 mean of NHWC [B][H][W][C] -> [B][H/2][W/2][C].
__global__ void avgpool2_kernel(const bf16* in, int B, int H, int W, int C, bf16* out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (e >= B * Ho * Wo * C) return;
    const int c = e % C, xo = (e / C) % Wo, yo = (e / (C * Wo)) % Ho, b = e / (C * Wo * Ho);
    const bf16* s = in + (((size_t)b * H + 2 * yo) * W + 2 * xo) * C + c;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(size_t)W * C]) +
                    __bfloat162float(s[(size_t)W * C + C]);
    out[e] = __float2bfloat16_rn(0.25f * v);
}

// Adjoint of avgpool2 followed by the ReLU derivative of the pooled layer:
// dz[b][y][x][c] = dpool[b][y/2][x/2][c] / 4 * (act[b][y][x][c] > 0).
__global__ void avgpool2_adj_kernel(const bf16* dpool, const bf16* act, int B, int H, int W, int C, bf16* dz) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * H * W * C) return;
    const int c = e % C, x = (e / C) % W, y = (e / (C * W)) % H, b = e / (C * W * H);
    const float g = __bfloat162float(dpool[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]);
    dz[e] = __float2bfloat16_rn(__bfloat162float(act[e]) > 0.f ? 0.25f * g : 0.f);
}

// Bilinear x4 sample position of fine node q (clamped to the coarse grid).
__device__ __forceinline__ void up4(int q, int n, int& i0, int& i1, float& t) {
    float s = (q + 0.5f) * 0.25f - 0.5f;
    s = fminf(fmaxf(s, 0.f), (float)(n - 1));
    i0 = (int)s;
    i1 = min(i0 + 1, n - 1);
    t = s - (float)i0;
}

// Head: z = w6 . h5 + b6, tz = tanh z (kept for the backward pass),
// v32 = v_mid + v_half tz.
__global__ void head_fwd_kernel(const bf16* h5, const float* w6, const float* b6, int npix, float v_mid, float v_half,
                                float* tz, float* v32) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const bf16* h = h5 + (size_t)p * kHid;
    float z = __ldg(b6);
    for (int c = 0; c < kHid; ++c) z = fmaf(__bfloat162float(h[c]), __ldg(w6 + c), z);
    const float t = tanhf(z);
    tz[p] = t;
    v32[p] = fmaf(v_half, t, v_mid);
}

// sos[b][qy][qx] = bilinear x4 of v32 on the mask, v_bg outside.
__global__ void upsample4_kernel(const float* v32, int B, int n, const unsigned char* mask, float v_bg, float* sos) {
    const int G = 4 * n;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * G * G) return;
    const int qx = e % G, qy = (e / G) % G, b = e / (G * G);
    if (mask && !mask[qy * G + qx]) {
        sos[e] = v_bg;
        return;
    }
    int y0, y1, x0, x1;
    float ty, tx;
    up4(qy, n, y0, y1, ty);
    up4(qx, n, x0, x1, tx);
    const float* v = v32 + (size_t)b * n * n;
    const float top = fmaf(tx, v[y0 * n + x1] - v[y0 * n + x0], v[y0 * n + x0]);
    const float bot = fmaf(tx, v[y1 * n + x1] - v[y1 * n + x0], v[y1 * n + x0]);
    sos[e] = fmaf(ty, bot - top, top);
}

// Training loss mean ((v - v_true) / scale)^2 over samples and mask nodes, and
// dL/dsos (0 outside the mask).  One CTA per sample, partial sums per sample.
__global__ void mse_kernel(const float* sos, const float* sos_true, const unsigned char* mask, int GG, float inv_count,
                           float inv_scale2, float* part, float* dsos) {
    const int b = blockIdx.x;
    float acc = 0.f;
    for (int q = threadIdx.x; q < GG; q += blockDim.x) {
        const size_t e = (size_t)b * GG + q;
        const bool in = mask ? mask[q] != 0 : true;
        const float r = in ? sos[e] - sos_true[e] : 0.f;
        acc = fmaf(r * r, inv_scale2, acc);
        if (dsos) dsos[e] = 2.f * r * inv_scale2 * inv_count;
    }
    __shared__ float red[8];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[b] = acc * inv_count;
}

__global__ void sum_kernel(const float* part, int n, float* out) {
    __shared__ float red[8];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[0] = acc;
}

// Head backward: dv32 = upsample4^T (dsos on the mask) (gathered per coarse
// node), dz = dv32 v_half (1 - tz^2); dh5[p][c] = dz w6[c] (h5 > 0); per-pixel
// products dz h5[p][c] and dz for dw6, db6 go to `hp` [npix][kHid + 1].
__global__ void head_bwd_kernel(const float* dsos, const unsigned char* mask, const float* tz, const bf16* h5,
                                const float* w6, int B, int n, float v_half, bf16* dh5, float* hp) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * n * n) return;
    const int ix = e % n, iy = (e / n) % n, b = e / (n * n);
    const int G = 4 * n;
    float g = 0.f;
    // fine nodes whose bilinear stencil touches coarse row iy lie in 4 iy - 2 .. 4 iy + 5
    for (int qy = max(0, 4 * iy - 2); qy <= min(G - 1, 4 * iy + 5); ++qy) {
        int y0, y1;
        float ty;
        up4(qy, n, y0, y1, ty);
        const float wy = (y0 == iy ? 1.f - ty : 0.f) + (y1 == iy ? ty : 0.f);
        if (wy == 0.f) continue;
        for (int qx = max(0, 4 * ix - 2); qx <= min(G - 1, 4 * ix + 5); ++qx) {
            if (mask && !mask[qy * G + qx]) continue;
            int x0, x1;
            float tx;
            up4(qx, n, x0, x1, tx);
            const float wx = (x0 == ix ? 1.f - tx : 0.f) + (x1 == ix ? tx : 0.f);
            g = fmaf(wy * wx, dsos[((size_t)b * G + qy) * G + qx], g);
        }
    }
    const float t = tz[e];
    const float dz = g * v_half * (1.f - t * t);
    const bf16* h = h5 + (size_t)e * kHid;
    bf16* dh = dh5 + (size_t)e * kHid;
    float* o = hp + (size_t)e * (kHid + 1);
    for (int c = 0; c < kHid; ++c) {
        const float hv = __bfloat162float(h[c]);
        dh[c] = __float2bfloat16_rn(hv > 0.f ? dz * __ldg(w6 + c) : 0.f);
        o[c] = dz * hv;
    }
    o[kHid] = dz;
}

constexpr int kColRows = 512;    // rows per block of the first column-sum stage

// Column sums of hp [npix][cols] in two fixed-order stages:
// part[blk][c] = sum of rows blk*512 .. +511, then out[c] (+)= sum over blocks.
__global__ void colsum1_kernel(const float* hp, int npix, int cols, float* part) {
    const int c = threadIdx.x;
    if (c >= cols) return;
    const int r0 = blockIdx.x * kColRows, r1 = min(npix, r0 + kColRows);
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += hp[(size_t)r * cols + c];
    part[(size_t)blockIdx.x * cols + c] = s;
}

__global__ void colsum2_kernel(const float* part, int nblk, int cols, float* out, int accumulate) {
    const int c = threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * cols + c];
    out[c] = accumulate ? out[c] + s : s;
}

// Packed BF16 weights of one 3x3 layer: forward taps [9][Cout][Cin] and dgrad
// taps [9][Cin][Cout], each tap a K-major tile image.  Input channels beyond
// cin (padding of the first layer) are zero.
__global__ void pack_kernel(const float* W, int cout, int cin, int cin_pad, bf16* fwd, bf16* bwd) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 9 * cout * cin_pad) return;
    const int tap = e / (cout * cin_pad), rem = e - tap * cout * cin_pad, co = rem / cin_pad, ci = rem % cin_pad;
    const float w = ci < cin ? W[((size_t)co * cin + ci) * 9 + tap] : 0.f;
    const bf16 v = __float2bfloat16_rn(w);
    unsigned char* f = reinterpret_cast<unsigned char*>(fwd + (size_t)tap * cout * cin_pad);
    *reinterpret_cast<bf16*>(f + umma::kmaj_off(co, ci, cin_pad)) = v;
    if (bwd) {
        unsigned char* g = reinterpret_cast<unsigned char*>(bwd + (size_t)tap * cout * cin_pad);
        *reinterpret_cast<bf16*>(g + umma::kmaj_off(ci, co, cout)) = v;
    }
}

// -------------------------------------------------------------- host plan

struct Layer {
    int cin, cin_pad, cout, res;   // res: side of the layer's input and output
    bool pool;
    size_t off_w, off_b;           // in the flat parameter vector
};

struct Net {
    int m, cp, R, B;
    Layer L[kNumConv];
    size_t off_w6, off_b6, nparam;
};

int pad_channels(int m) { return m <= 16 ? 16 : m <= 32 ? 32 : 64; }

Net make_net(int m, int R, int B) {
    Net n;
    n.m = m;
    n.cp = pad_channels(m);
    n.R = R;
    n.B = B;
    const int cins[kNumConv] = {m, 32, 64, 64, 64}, couts[kNumConv] = {32, 64, 64, 64, 64};
    const bool pools[kNumConv] = {true, true, false, false, false};
    size_t o = 0;
    int res = R;
    for (int l = 0; l < kNumConv; ++l) {
        Layer& y = n.L[l];
        y.cin = cins[l];
        y.cin_pad = l == 0 ? n.cp : cins[l];
        y.cout = couts[l];
        y.res = res;
        y.pool = pools[l];
        y.off_w = o;
        o += (size_t)y.cout * y.cin * 9;
        y.off_b = o;
        o += y.cout;
        if (y.pool) res /= 2;
    }
    n.off_w6 = o;
    o += kHid;
    n.off_b6 = o;
    o += 1;
    n.nparam = o;
    return n;
}

// Workspace layout (all offsets 256-byte aligned).
struct CnnPlan {
    Net net;
    size_t off_wf[kNumConv], off_wb[kNumConv];   // packed weights
    size_t off_act[kNumConv];      // layer outputs before pooling [B][res][res][cout]
    size_t off_pool[2];            // pooled outputs of layers 1, 2
    size_t off_tz, off_v32;        // head
    size_t off_g1, off_g2;         // gradient buffers (max activation size), bf16
    size_t off_hp;                 // head products [npix][65] fp32
    size_t off_part;               // wgrad partials
    size_t off_status;
    size_t total;
};

// Pixels per weight-gradient CTA: halved from kWgChunk (down to kWgMinChunk)
// while the layer would give fewer than kWgTargetCtas CTAs, so that the
// small-resolution layers fill the GPU (a fixed target keeps the workspace
// size independent of the device).
int wgrad_chunk(const Layer& y, int B) {
    const long long P = (long long)B * y.res * y.res;
    const int tpg = 128 / y.cin_pad, groups = (9 + tpg - 1) / tpg;
    int chunk = kWgChunk;
    while (chunk > kWgMinChunk && ((P + chunk - 1) / chunk) * groups < kWgTargetCtas) chunk /= 2;
    return chunk;
}

size_t wgrad_part_elems(const Layer& y, int B) {
    const size_t P = (size_t)B * y.res * y.res;
    const int tpg = 128 / y.cin_pad, groups = (9 + tpg - 1) / tpg;
    const size_t chunk = (size_t)wgrad_chunk(y, B);
    return ((P + chunk - 1) / chunk) * groups * 128 * (size_t)y.cout;
}

CnnPlan make_cnn_plan(int m, int R, int B) {
    CnnPlan p;
    p.net = make_net(m, R, B);
    const Net& n = p.net;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes, 256);
        return at;
    };
    size_t maxact = 0, maxpart = 0;
    for (int l = 0; l < kNumConv; ++l) {
        const Layer& y = n.L[l];
        p.off_wf[l] = take((size_t)9 * y.cout * y.cin_pad * 2);
        p.off_wb[l] = take((size_t)9 * y.cout * y.cin_pad * 2);
        const size_t act = (size_t)B * y.res * y.res * y.cout;
        p.off_act[l] = take(act * 2);
        maxact = std::max(maxact, std::max(act, (size_t)B * y.res * y.res * y.cin_pad));
        maxpart = std::max(maxpart, wgrad_part_elems(y, B));
    }
    p.off_pool[0] = take((size_t)B * (R / 2) * (R / 2) * 32 * 2);
    p.off_pool[1] = take((size_t)B * (R / 4) * (R / 4) * 64 * 2);
    const size_t npix = (size_t)B * (R / 4) * (R / 4);
    p.off_tz = take(npix * 4);
    p.off_v32 = take(npix * 4);
    p.off_g1 = take(maxact * 2);
    p.off_g2 = take(maxact * 2);
    p.off_hp = take(npix * (kHid + 1) * 4);
    p.off_part = take(maxpart * 4);
    p.off_status = take(4);
    p.total = o;
    return p;
}

pact_status check_cnn(const pact_geometry* g, int m, int B) {
    PACT_TRY(check_geometry(g));
    if (m < 1 || m > PACT_MAX_CHANNELS) return fail(PACT_ERR_SHAPE, "cnn: channel count %d outside 1..%d", m, PACT_MAX_CHANNELS);
    if (B < 1) return fail(PACT_ERR_INVALID_ARG, "cnn: batch must be >= 1");
    if (g->img_h != g->img_w || g->img_h != 4 * g->sos_g || g->sos_g % 8 != 0)
        return fail(PACT_ERR_SHAPE, "cnn: needs a square image of 4 G pixels per side with G a multiple of 8");
    // the convolution kernels divide pixel indices by a float reciprocal, exact below 2^22
    if ((long long)B * g->sos_g * g->sos_g + g->sos_g >= (1ll << 22))
        return fail(PACT_ERR_SHAPE, "cnn: batch x G^2 = %lld pixels, must be below 2^22 - G",
                    (long long)B * g->sos_g * g->sos_g);
    return PACT_OK;
}

struct Ctx {
    CnnPlan pl;
    char* ws;
    cudaStream_t st;
    int* status;
    template <typename T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

pact_status launch_conv(const Ctx& c, const bf16* in, const bf16* wpk, const float* bias, const bf16* mask, bf16* out,
                        int B, int res, int K, int N, int sign, int relu) {
    ConvArgs a;
    a.in = in;
    a.wpk = wpk;
    a.bias = bias;
    a.mask = mask;
    a.out = out;
    a.B = B;
    a.H = res;
    a.W = res;
    a.K = K;
    a.N = N;
    a.sign = sign;
    a.relu = relu;
    a.status = c.status;
    a.limit_ns = wait_limit_ns();
    if (K % 8 || K > 64 || 16 % (K / 8)) return fail(PACT_ERR_SHAPE, "cnn: conv K = %d unsupported", K);
    const size_t smem = (size_t)kConvStages * (128 * K * 2 + (size_t)N * K * 2);
    PACT_TRY(ensure_smem((const void*)conv_kernel, smem, "cnn: conv shared memory attribute"));
    const int P = B * res * res;
    conv_kernel<<<(P + 127) / 128, 128, smem, c.st>>>(a);
    return check_launch("cnn conv kernel");
}

pact_status launch_wgrad(const Ctx& c, const Layer& y, const bf16* x, const bf16* dz, float* dW, float* db,
                         int accumulate) {
    const int B = c.pl.net.B;
    const int P = B * y.res * y.res;
    WgradArgs a;
    a.x = x;
    a.dz = dz;
    a.part = c.at<float>(c.pl.off_part);
    a.B = B;
    a.H = y.res;
    a.W = y.res;
    a.Cin = y.cin_pad;
    a.Cout = y.cout;
    a.taps_per_group = 128 / y.cin_pad;
    a.status = c.status;
    a.limit_ns = wait_limit_ns();
    const int groups = (9 + a.taps_per_group - 1) / a.taps_per_group;
    a.chunk = wgrad_chunk(y, B);
    const int nchunks = (P + a.chunk - 1) / a.chunk;
    const size_t smem = (size_t)kWgStages * (128 * kWgPix * 2 + (size_t)y.cout * kWgPix * 2);
    PACT_TRY(ensure_smem((const void*)wgrad_kernel, smem, "cnn: wgrad shared memory attribute"));
    wgrad_kernel<<<dim3(nchunks, groups), 128, smem, c.st>>>(a);
    PACT_TRY(check_launch("cnn wgrad kernel"));
    const int ne = groups * 128 * y.cout;
    wgrad_reduce_kernel<<<(ne + 255) / 256, 256, 0, c.st>>>(a.part, nchunks, groups, y.cin, y.cin_pad, y.cout,
                                                           a.taps_per_group, dW, db, accumulate);
    return check_launch("cnn wgrad reduction");
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" int pact_cnn_param_count(int m) {
    if (m < 1 || m > PACT_MAX_CHANNELS) return 0;
    return (int)make_net(m, 32, 1).nparam;
}

extern "C" size_t pact_cnn_workspace_size(const pact_geometry* g, int m, int batch) {
    if (check_cnn(g, m, batch) != PACT_OK) return 0;
    return make_cnn_plan(m, g->sos_g, batch).total;
}

extern "C" int pact_cnn_input_channels(int m) { return m < 1 || m > PACT_MAX_CHANNELS ? 0 : pad_channels(m); }

extern "C" size_t pact_cnn_pool_workspace_size(const pact_geometry* g, int m) {
    if (check_cnn(g, m, 1) != PACT_OK) return 0;
    return align_up((size_t)g->sos_g * g->sos_g * pad_channels(m) * sizeof(float), 16) + sizeof(double);
}

extern "C" pact_status pact_cnn_pool_stack(const pact_geometry* g, const float* stack, int m, void* x, void* ws,
                                           size_t ws_bytes, void* stream) {
    PACT_TRY(check_cnn(g, m, 1));
    if (!stack || !x || !ws) return fail(PACT_ERR_INVALID_ARG, "cnn_pool_stack: null pointer");
    if (reinterpret_cast<uintptr_t>(x) % 16) return fail(PACT_ERR_INVALID_ARG, "cnn_pool_stack: x must be 16-byte aligned");
    const size_t need = pact_cnn_pool_workspace_size(g, m);
    if (ws_bytes < need) return fail(PACT_ERR_INVALID_ARG, "cnn_pool_stack: workspace too small: %zu < %zu", ws_bytes, need);
    cudaStream_t st = as_stream(stream);
    const int R = g->sos_g, cp = pad_channels(m);
    const int n = R * R * cp;
    float* pooled = static_cast<float*>(ws);
    double* sumsq = reinterpret_cast<double*>(static_cast<char*>(ws) + align_up((size_t)n * sizeof(float), 16));
    if (cudaMemsetAsync(sumsq, 0, sizeof(double), st) != cudaSuccess) return check_launch("cnn_pool_stack: memset");
    pool4_kernel<<<(n + 255) / 256, 256, 0, st>>>(stack, m, g->img_h, g->img_w, pooled, cp, sumsq);
    PACT_TRY(check_launch("cnn pool kernel"));
    scale_cast_kernel<<<(n + 255) / 256, 256, 0, st>>>(pooled, n, sumsq, (float)R * R * m, static_cast<bf16*>(x));
    return check_launch("cnn scale kernel");
}

extern "C" pact_status pact_cnn_forward(const pact_geometry* g, int m, int batch, const float* params,
                                        const void* x, const unsigned char* mask, float v_mid, float v_half,
                                        float* sos, void* ws, size_t ws_bytes, void* stream) {
    PACT_TRY(check_cnn(g, m, batch));
    if (!params || !x || !sos || !ws) return fail(PACT_ERR_INVALID_ARG, "cnn_forward: null pointer");
    if (reinterpret_cast<uintptr_t>(x) % 16) return fail(PACT_ERR_INVALID_ARG, "cnn_forward: x must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "cnn: workspace must be 256-byte aligned");
    Ctx c;
    c.pl = make_cnn_plan(m, g->sos_g, batch);
    if (ws_bytes < c.pl.total) return fail(PACT_ERR_INVALID_ARG, "cnn: workspace too small: %zu < %zu", ws_bytes, c.pl.total);
    c.ws = static_cast<char*>(ws);
    c.st = as_stream(stream);
    c.status = c.at<int>(c.pl.off_status);
    const Net& n = c.pl.net;
    const int B = batch, R = n.R;
    if (cudaMemsetAsync(c.status, 0, sizeof(int), c.st) != cudaSuccess) return check_launch("cnn: memset");
    for (int l = 0; l < kNumConv; ++l) {
        const Layer& y = n.L[l];
        const int ne = 9 * y.cout * y.cin_pad;
        pack_kernel<<<(ne + 255) / 256, 256, 0, c.st>>>(params + y.off_w, y.cout, y.cin, y.cin_pad,
                                                        c.at<bf16>(c.pl.off_wf[l]), c.at<bf16>(c.pl.off_wb[l]));
        PACT_TRY(check_launch("cnn pack kernel"));
    }
    const bf16* in = static_cast<const bf16*>(x);
    for (int l = 0; l < kNumConv; ++l) {
        const Layer& y = n.L[l];
        bf16* act = c.at<bf16>(c.pl.off_act[l]);
        PACT_TRY(launch_conv(c, in, c.at<bf16>(c.pl.off_wf[l]), params + y.off_b, nullptr, act, B, y.res, y.cin_pad,
                             y.cout, 1, 1));
        if (y.pool) {
            bf16* po = c.at<bf16>(c.pl.off_pool[l]);
            const int ne = B * (y.res / 2) * (y.res / 2) * y.cout;
            avgpool2_kernel<<<(ne + 255) / 256, 256, 0, c.st>>>(act, B, y.res, y.res, y.cout, po);
            PACT_TRY(check_launch("cnn pool kernel"));
            in = po;
        } else {
            in = act;
        }
    }
    const int n4 = R / 4, npix = B * n4 * n4;
    head_fwd_kernel<<<(npix + 255) / 256, 256, 0, c.st>>>(c.at<bf16>(c.pl.off_act[kNumConv - 1]), params + n.off_w6,
                                                          params + n.off_b6, npix, v_mid, v_half,
                                                          c.at<float>(c.pl.off_tz), c.at<float>(c.pl.off_v32));
    PACT_TRY(check_launch("cnn head kernel"));
    const int ns = B * R * R;
    upsample4_kernel<<<(ns + 255) / 256, 256, 0, c.st>>>(c.at<float>(c.pl.off_v32), B, n4, mask, g->v_bg, sos);
    return check_launch("cnn upsample kernel");
}

extern "C" pact_status pact_cnn_mse(const pact_geometry* g, int batch, const float* sos, const float* sos_true,
                                    const unsigned char* mask, int mask_count, float scale, float* loss,
                                    float* dL_dsos, float* scratch, void* stream) {
    PACT_TRY(check_geometry(g));
    if (!sos || !sos_true || !loss || !scratch) return fail(PACT_ERR_INVALID_ARG, "cnn_mse: null pointer");
    const int GG = g->sos_g * g->sos_g;
    const int count = mask ? mask_count : GG;
    if (batch < 1 || !(scale > 0.f) || count < 1 || count > GG)
        return fail(PACT_ERR_INVALID_ARG, "cnn_mse: batch >= 1, scale > 0 and 1 <= mask_count <= G^2 required");
    cudaStream_t st = as_stream(stream);
    mse_kernel<<<batch, 256, 0, st>>>(sos, sos_true, mask, GG, 1.f / ((float)count * batch), 1.f / (scale * scale),
                                      scratch, dL_dsos);
    PACT_TRY(check_launch("cnn mse kernel"));
    sum_kernel<<<1, 256, 0, st>>>(scratch, batch, loss);
    return check_launch("cnn mse sum");
}

extern "C" pact_status pact_cnn_backward(const pact_geometry* g, int m, int batch, const float* params,
                                         const void* x, const unsigned char* mask, float v_half,
                                         const float* dL_dsos, float* dL_dparams, int accumulate, void* ws,
                                         size_t ws_bytes, void* stream) {
    PACT_TRY(check_cnn(g, m, batch));
    if (!params || !x || !dL_dsos || !dL_dparams || !ws) return fail(PACT_ERR_INVALID_ARG, "cnn_backward: null pointer");
    Ctx c;
    c.pl = make_cnn_plan(m, g->sos_g, batch);
    if (ws_bytes < c.pl.total) return fail(PACT_ERR_INVALID_ARG, "cnn: workspace too small: %zu < %zu", ws_bytes, c.pl.total);
    c.ws = static_cast<char*>(ws);
    c.st = as_stream(stream);
    c.status = c.at<int>(c.pl.off_status);
    const Net& n = c.pl.net;
    const int B = batch, R = n.R, n4 = R / 4, npix = B * n4 * n4;
    // head
    bf16* g1 = c.at<bf16>(c.pl.off_g1);
    bf16* g2 = c.at<bf16>(c.pl.off_g2);
    float* hp = c.at<float>(c.pl.off_hp);
    head_bwd_kernel<<<(npix + 255) / 256, 256, 0, c.st>>>(dL_dsos, mask, c.at<float>(c.pl.off_tz),
                                                          c.at<bf16>(c.pl.off_act[kNumConv - 1]), params + n.off_w6, B,
                                                          n4, v_half, g1, hp);
    PACT_TRY(check_launch("cnn head backward"));
    {
        const int nblk = (npix + kColRows - 1) / kColRows;
        float* part = c.at<float>(c.pl.off_part);
        colsum1_kernel<<<nblk, 128, 0, c.st>>>(hp, npix, kHid + 1, part);
        colsum2_kernel<<<1, 128, 0, c.st>>>(part, nblk, kHid + 1, dL_dparams + n.off_w6, accumulate);
        PACT_TRY(check_launch("cnn head reduction"));
    }
    // g1 holds dZ of layer 5 (gradient at its pre-activation); walk back.  Stream
    // order makes each kernel see the previous one's writes.
    bf16* dz = g1;       // dZ of layer l
    bf16* tmp = g2;
    const bf16* xin = static_cast<const bf16*>(x);
    for (int l = kNumConv - 1; l >= 0; --l) {
        const Layer& y = n.L[l];
        const bf16* lin = l == 0 ? xin
                          : n.L[l - 1].pool ? c.at<bf16>(c.pl.off_pool[l - 1]) : c.at<bf16>(c.pl.off_act[l - 1]);
        PACT_TRY(launch_wgrad(c, y, lin, dz, dL_dparams + y.off_w, dL_dparams + y.off_b, accumulate));
        if (l == 0) break;
        const Layer& yp = n.L[l - 1];
        const bf16* act_prev = c.at<bf16>(c.pl.off_act[l - 1]);
        if (!yp.pool) {
            // dZ_{l-1} = (dZ_l conv^T W_l) * (act_{l-1} > 0)
            PACT_TRY(launch_conv(c, dz, c.at<bf16>(c.pl.off_wb[l]), nullptr, act_prev, tmp, B, y.res, y.cout,
                                 y.cin, -1, 0));
            std::swap(dz, tmp);
        } else {
            // d(pooled_{l-1}) = dZ_l conv^T W_l into tmp; pool adjoint and ReLU mask back into dz
            PACT_TRY(launch_conv(c, dz, c.at<bf16>(c.pl.off_wb[l]), nullptr, nullptr, tmp, B, y.res, y.cout, y.cin,
                                 -1, 0));
            const int ne = B * yp.res * yp.res * yp.cout;
            avgpool2_adj_kernel<<<(ne + 255) / 256, 256, 0, c.st>>>(tmp, act_prev, B, yp.res, yp.res, yp.cout, dz);
            PACT_TRY(check_launch("cnn pool adjoint"));
        }
    }
    return PACT_OK;
}

extern "C" pact_status pact_cnn_status(const pact_geometry* g, int m, int batch, const void* ws, size_t ws_bytes,
                                       int* host_status, void* stream) {
    PACT_TRY(check_cnn(g, m, batch));
    if (!ws || !host_status) return fail(PACT_ERR_INVALID_ARG, "cnn_status: null pointer");
    const CnnPlan pl = make_cnn_plan(m, g->sos_g, batch);
    if (ws_bytes < pl.total) return fail(PACT_ERR_INVALID_ARG, "cnn_status: workspace too small");
    cudaStream_t st = as_stream(stream);
    if (cudaMemcpyAsync(host_status, static_cast<const char*>(ws) + pl.off_status, sizeof(int), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return check_launch("cnn_status: copy");
    return *host_status ? fail(PACT_ERR_TIMEOUT, "cnn: a tensor-core completion wait gave up") : PACT_OK;
}
