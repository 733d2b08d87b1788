// Sec. S1.5 on the GPU: Gaussian-windowed patch spectra (pact_patch_fft) and
// stitching of deconvolved patches (pact_stitch).
//
// Both run once per recovery, so they use a direct separable DFT from shared
// memory (one CTA per patch and channel): P x P real samples, a twiddle table
// exp(-2 pi j t / P), a row pass to the P/2+1 half-spectrum columns and a
// column pass, in FP32 (error ~ sqrt(P) ulp).  The forward transform gives
// each thread a register tile of outputs and pairs samples t and P - t.
#include <algorithm>

#include "pact_internal.cuh"

namespace pact {
namespace {

// Shared-memory layout of patch_fft_kernel for patch size P.  xT holds the
// windowed patch transposed (xT[b][a] = sample at row a, column b) with a row
// stride PS: a multiple of 4 (float4 reads of four rows) whose quarter is odd,
// so the transposing float4 stores of eight consecutive columns hit distinct
// banks.  R holds the row spectra with an even stride HS (float4 reads of two
// columns), tw the twiddles exp(-2 pi j t / P).
__host__ __device__ inline int fft_ps(int P) {
    const int p4 = (P + 3) & ~3;
    return ((p4 / 4) & 1) ? p4 : p4 + 4;
}
__host__ __device__ inline int fft_hs(int P) { return ((P / 2 + 1) + 1) & ~1; }
inline size_t fft_smem(int P) {
    return (size_t)P * fft_ps(P) * sizeof(float) + ((size_t)P * fft_hs(P) + P) * sizeof(float2);
}

// Register tiles: the row pass gives a thread 4 patch rows x 4 half-spectrum
// columns, the column pass 8 frequency rows x 2 columns.
constexpr int kRA = 4, kRV = 4, kCU = 8, kCV = 2;

// Windowed half-spectrum DFT of patch i = blockIdx.y, channel j = blockIdx.x.
// Both passes pair sample t with P - t: for a real row, x_t e^{-j phi} +
// x_{P-t} e^{j phi} = (x_t + x_{P-t}) cos phi - j (x_t - x_{P-t}) sin phi, and
// for the complex column pass the same with R_t +- R_{P-t}, which halves the
// multiply-adds; t = 0 and t = P/2 enter once with phase 1 and (-1)^k.
__global__ void __launch_bounds__(256, 3) patch_fft_kernel(Geo g, int P, int M, const int2* centres,
                                                        float inv_2s2, const float* stack, float2* Y) {
    extern __shared__ float4 sm4[];
    const int half = P / 2 + 1, h2 = P / 2, PS = fft_ps(P), HS = fft_hs(P);
    float* xT = reinterpret_cast<float*>(sm4);
    float2* R = reinterpret_cast<float2*>(xT + (size_t)P * PS);
    float2* tw = R + (size_t)P * HS;
    const int i = blockIdx.y, j = blockIdx.x;
    const int2 c = centres[i];
    const int r0 = c.x - P / 2, c0 = c.y - P / 2;
    for (int t = threadIdx.x; t < P; t += blockDim.x) tw[t] = cis_pi(-2.f * t / P);
    const float* img = stack + (size_t)j * g.H * g.W;
    // column b fastest: coalesced reads of the image, one float4 of four rows per store
    for (int q = threadIdx.x; q < (PS / 4) * P; q += blockDim.x) {
        const int ag = q / P, b = q - ag * P;
        const int col = c0 + b;
        const float ob = (b - P / 2) * g.dx;
        float v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int a = ag * 4 + r, row = r0 + a;
            float val = 0.f;
            if (a < P && row >= 0 && row < g.H && col >= 0 && col < g.W) val = img[(size_t)row * g.W + col];
            const float oa = (a - P / 2) * g.dx;
            v[r] = val * expf(-(oa * oa + ob * ob) * inv_2s2);
        }
        *reinterpret_cast<float4*>(xT + (size_t)b * PS + ag * 4) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __syncthreads();
    // row pass: R[a][v] = sum_b x[a][b] exp(-2 pi j b v / P); neighbouring lanes
    // take neighbouring row groups, so a warp's twiddle loads are broadcasts
    const int na1 = (P + kRA - 1) / kRA;
    for (int t = threadIdx.x; t < na1 * ((half + kRV - 1) / kRV); t += blockDim.x) {
        const int v0 = (t / na1) * kRV, a0 = (t - (t / na1) * na1) * kRA;
        int vv[kRV], id[kRV];
        float re[kRA][kRV], im[kRA][kRV];
        const float4 x0 = *reinterpret_cast<const float4*>(xT + a0);
        const float4 xh = *reinterpret_cast<const float4*>(xT + (size_t)h2 * PS + a0);
        const float xa[4] = {x0.x, x0.y, x0.z, x0.w}, xb[4] = {xh.x, xh.y, xh.z, xh.w};
#pragma unroll
        for (int k = 0; k < kRV; ++k) {
            vv[k] = min(v0 + k, half - 1);
            id[k] = vv[k];
#pragma unroll
            for (int r = 0; r < kRA; ++r) {
                re[r][k] = (vv[k] & 1) ? xa[r] - xb[r] : xa[r] + xb[r];
                im[r][k] = 0.f;
            }
        }
        for (int b = 1; b < h2; ++b) {
            const float4 p = *reinterpret_cast<const float4*>(xT + (size_t)b * PS + a0);
            const float4 m = *reinterpret_cast<const float4*>(xT + (size_t)(P - b) * PS + a0);
            const float s[4] = {p.x + m.x, p.y + m.y, p.z + m.z, p.w + m.w};
            const float d[4] = {p.x - m.x, p.y - m.y, p.z - m.z, p.w - m.w};
#pragma unroll
            for (int k = 0; k < kRV; ++k) {
                const float2 w = tw[id[k]];
#pragma unroll
                for (int r = 0; r < kRA; ++r) {
                    re[r][k] = fmaf(s[r], w.x, re[r][k]);
                    im[r][k] = fmaf(d[r], w.y, im[r][k]);
                }
                id[k] += vv[k];
                if (id[k] >= P) id[k] -= P;
            }
        }
#pragma unroll
        for (int r = 0; r < kRA; ++r)
#pragma unroll
            for (int k = 0; k < kRV; ++k)
                if (a0 + r < P && v0 + k < half) R[(size_t)(a0 + r) * HS + v0 + k] = make_float2(re[r][k], im[r][k]);
    }
    __syncthreads();
    // column pass: Y[u][v] = sum_a R[a][v] exp(-2 pi j u a / P) / P
    const float inv_p = 1.f / P;
    float2* out = Y + ((size_t)i * M + j) * P * half;
    const int nv2 = (half + kCV - 1) / kCV;
    for (int t = threadIdx.x; t < ((P + kCU - 1) / kCU) * nv2; t += blockDim.x) {
        const int u0 = (t / nv2) * kCU, v0 = (t - (t / nv2) * nv2) * kCV;
        int uu[kCU], id[kCU];
        float re[kCU][2], im[kCU][2];
        const float4 q0 = *reinterpret_cast<const float4*>(R + v0);
        const float4 qh = *reinterpret_cast<const float4*>(R + (size_t)h2 * HS + v0);
#pragma unroll
        for (int k = 0; k < kCU; ++k) {
            uu[k] = min(u0 + k, P - 1);
            id[k] = uu[k];
            const float sg = (uu[k] & 1) ? -1.f : 1.f;
            re[k][0] = fmaf(sg, qh.x, q0.x);
            im[k][0] = fmaf(sg, qh.y, q0.y);
            re[k][1] = fmaf(sg, qh.z, q0.z);
            im[k][1] = fmaf(sg, qh.w, q0.w);
        }
        for (int a = 1; a < h2; ++a) {
            const float4 p = *reinterpret_cast<const float4*>(R + (size_t)a * HS + v0);
            const float4 m = *reinterpret_cast<const float4*>(R + (size_t)(P - a) * HS + v0);
            const float sr0 = p.x + m.x, si0 = p.y + m.y, dr0 = p.x - m.x, di0 = p.y - m.y;
            const float sr1 = p.z + m.z, si1 = p.w + m.w, dr1 = p.z - m.z, di1 = p.w - m.w;
#pragma unroll
            for (int k = 0; k < kCU; ++k) {
                const float2 w = tw[id[k]];
                re[k][0] = fmaf(-di0, w.y, fmaf(sr0, w.x, re[k][0]));
                im[k][0] = fmaf(dr0, w.y, fmaf(si0, w.x, im[k][0]));
                re[k][1] = fmaf(-di1, w.y, fmaf(sr1, w.x, re[k][1]));
                im[k][1] = fmaf(dr1, w.y, fmaf(si1, w.x, im[k][1]));
                id[k] += uu[k];
                if (id[k] >= P) id[k] -= P;
            }
        }
#pragma unroll
        for (int k = 0; k < kCU; ++k)
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2)
                if (u0 + k < P && v0 + c2 < half)
                    out[(size_t)(u0 + k) * half + v0 + c2] = make_float2(re[k][c2] * inv_p, im[k][c2] * inv_p);
    }
}

// Shared memory of stitch_kernel: the patch's half spectrum X and the column
// pass output Z, both [P][HS] float2 (HS = fft_hs(P): float4 reads of two
// columns), and the twiddles exp(+2 pi j t / P).
inline size_t stitch_smem(int P) { return ((size_t)2 * P * fft_hs(P) + P) * sizeof(float2); }

// Register tiles of the inverse: the column pass gives a thread 8 rows x 2
// half-spectrum columns (as the forward column pass), the row pass 4 rows x 4
// column pairs (b, P - b).
constexpr int kSA = 4, kSB = 4;

// Inverse half-spectrum DFT of patch i = blockIdx.x, channel j = blockIdx.y
// (X [N][m][P][P/2+1]), then scatter-add into the channel's numerator image
// and, for channel 0, into the window-sum image.  Both images are FP64: a pixel
// sums a few FP32 terms (one per overlapping patch), which FP64 holds exactly,
// so the order of the atomic additions cannot change the result (the stitched
// image is the same in every run).
// Column pass: Z[a][v] = sum_u X[u][v] exp(+2 pi j a u / P), pairing u with
// P - u as the forward column pass does.  Row pass: every row of Z is the
// half of a Hermitian row spectrum, so with C = sum_v c_v Re Z[a][v] cos(2 pi v b / P)
// and S = sum_v c_v Im Z[a][v] sin(2 pi v b / P) (c_v = 1 at v = 0, P/2, else 2)
// the pixel pair is x[a][b] = (C - S) / P, x[a][P - b] = (C + S) / P: one set
// of sums gives both.
__global__ void __launch_bounds__(256) stitch_kernel(Geo g, int P, const int2* centres, float inv_2s2,
                                                     const float2* X, double* num, double* den) {
    extern __shared__ float4 sm4[];
    const int half = P / 2 + 1, h2 = P / 2, HS = fft_hs(P);
    float2* Xs = reinterpret_cast<float2*>(sm4);   // [P][HS]
    float2* Z = Xs + (size_t)P * HS;               // [P][HS]
    float2* tw = Z + (size_t)P * HS;               // [P]: exp(+2 pi j t / P)
    const int i = blockIdx.x, j = blockIdx.y, m = gridDim.y;
    const int2 c = centres[i];
    const int r0 = c.x - P / 2, c0 = c.y - P / 2;
    const float2* Xi = X + ((size_t)i * m + j) * P * half;
    for (int t = threadIdx.x; t < P; t += blockDim.x) tw[t] = cis_pi(2.f * t / P);
    for (int q = threadIdx.x; q < P * half; q += blockDim.x) {
        const int u = q / half, v = q - (q / half) * half;
        Xs[(size_t)u * HS + v] = Xi[q];
    }
    if (HS > half)
        for (int u = threadIdx.x; u < P; u += blockDim.x) Xs[(size_t)u * HS + half] = make_float2(0.f, 0.f);
    __syncthreads();
    // column pass
    const int nv2 = (half + kCV - 1) / kCV;
    for (int t = threadIdx.x; t < ((P + kCU - 1) / kCU) * nv2; t += blockDim.x) {
        const int a0 = (t / nv2) * kCU, v0 = (t - (t / nv2) * nv2) * kCV;
        int aa[kCU], id[kCU];
        float re[kCU][2], im[kCU][2];
        const float4 q0 = *reinterpret_cast<const float4*>(Xs + v0);
        const float4 qh = *reinterpret_cast<const float4*>(Xs + (size_t)h2 * HS + v0);
#pragma unroll
        for (int k = 0; k < kCU; ++k) {
            aa[k] = min(a0 + k, P - 1);
            id[k] = aa[k];
            const float sg = (aa[k] & 1) ? -1.f : 1.f;
            re[k][0] = fmaf(sg, qh.x, q0.x);
            im[k][0] = fmaf(sg, qh.y, q0.y);
            re[k][1] = fmaf(sg, qh.z, q0.z);
            im[k][1] = fmaf(sg, qh.w, q0.w);
        }
        for (int u = 1; u < h2; ++u) {
            const float4 p = *reinterpret_cast<const float4*>(Xs + (size_t)u * HS + v0);
            const float4 mm = *reinterpret_cast<const float4*>(Xs + (size_t)(P - u) * HS + v0);
            const float sr0 = p.x + mm.x, si0 = p.y + mm.y, dr0 = p.x - mm.x, di0 = p.y - mm.y;
            const float sr1 = p.z + mm.z, si1 = p.w + mm.w, dr1 = p.z - mm.z, di1 = p.w - mm.w;
#pragma unroll
            for (int k = 0; k < kCU; ++k) {
                const float2 w = tw[id[k]];
                re[k][0] = fmaf(-di0, w.y, fmaf(sr0, w.x, re[k][0]));
                im[k][0] = fmaf(dr0, w.y, fmaf(si0, w.x, im[k][0]));
                re[k][1] = fmaf(-di1, w.y, fmaf(sr1, w.x, re[k][1]));
                im[k][1] = fmaf(dr1, w.y, fmaf(si1, w.x, im[k][1]));
                id[k] += aa[k];
                if (id[k] >= P) id[k] -= P;
            }
        }
#pragma unroll
        for (int k = 0; k < kCU; ++k)
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2)
                if (a0 + k < P && v0 + c2 < half) Z[(size_t)(a0 + k) * HS + v0 + c2] = make_float2(re[k][c2], im[k][c2]);
    }
    __syncthreads();
    // row pass and scatter: rows a0 .. a0 + 3, columns b0 .. b0 + 3 (<= P/2) and their mirrors
    const float inv_p = 1.f / P;
    num += (size_t)j * g.H * g.W;
    const int nb4 = (h2 + 1 + kSB - 1) / kSB, na4 = (P + kSA - 1) / kSA;
    for (int t = threadIdx.x; t < na4 * nb4; t += blockDim.x) {
        const int a0 = (t / nb4) * kSA, b0 = (t - (t / nb4) * nb4) * kSB;
        int bb[kSB], id[kSB];
        float C[kSA][kSB], S[kSA][kSB];
#pragma unroll
        for (int k = 0; k < kSB; ++k) {
            bb[k] = min(b0 + k, h2);
            id[k] = bb[k];
        }
#pragma unroll
        for (int r = 0; r < kSA; ++r) {
            const int a = min(a0 + r, P - 1);
            const float z0 = Z[(size_t)a * HS].x, zh = Z[(size_t)a * HS + h2].x;
#pragma unroll
            for (int k = 0; k < kSB; ++k) {
                C[r][k] = (bb[k] & 1) ? z0 - zh : z0 + zh;
                S[r][k] = 0.f;
            }
        }
        for (int v = 1; v < h2; ++v) {
            float2 w[kSB];
#pragma unroll
            for (int k = 0; k < kSB; ++k) {
                w[k] = tw[id[k]];
                id[k] += bb[k];
                if (id[k] >= P) id[k] -= P;
            }
#pragma unroll
            for (int r = 0; r < kSA; ++r) {
                const float2 zv = Z[(size_t)min(a0 + r, P - 1) * HS + v];
#pragma unroll
                for (int k = 0; k < kSB; ++k) {
                    C[r][k] = fmaf(2.f * zv.x, w[k].x, C[r][k]);
                    S[r][k] = fmaf(2.f * zv.y, w[k].y, S[r][k]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kSA; ++r) {
            const int a = a0 + r, row = r0 + a;
            if (a >= P || row < 0 || row >= g.H) continue;
            const float oa = (a - P / 2) * g.dx;
#pragma unroll
            for (int k = 0; k < kSB; ++k) {
                const int b = b0 + k;
                if (b > h2) continue;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int bc = side ? P - b : b;
                    if (side && (b == 0 || b == h2)) continue;
                    const int col = c0 + bc;
                    if (col < 0 || col >= g.W) continue;
                    const float val = (side ? C[r][k] + S[r][k] : C[r][k] - S[r][k]) * inv_p;
                    atomicAdd(num + (size_t)row * g.W + col, (double)val);
                    if (j == 0) {
                        const float ob = (bc - P / 2) * g.dx;
                        atomicAdd(den + (size_t)row * g.W + col, (double)expf(-(oa * oa + ob * ob) * inv_2s2));
                    }
                }
            }
        }
    }
}

// out[j][q] = num[j][q] / den[q] (0 where no window reaches), j = blockIdx.y.
__global__ void stitch_divide_kernel(int n, const double* num, const double* den, float* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const size_t o = (size_t)blockIdx.y * n + q;
    const float d = (float)den[q];
    out[o] = d > 0.f ? (float)num[o] / d : 0.f;
}

float inv_two_sigma2(float fwhm) {
    const double sig = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    return (float)(1.0 / (2.0 * sig * sig));
}



}  // namespace
}  // namespace pact

using namespace pact;

extern "C" pact_status pact_patch_fft(const pact_geometry* g, const pact_patches* pt, const float* stack, int m,
                                      float* Y, void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!stack || !Y) return fail(PACT_ERR_INVALID_ARG, "patch_fft: stack and Y must not be NULL");
    if (m < 1 || m > 65535) return fail(PACT_ERR_INVALID_ARG, "patch_fft: channel count %d out of range", m);
    const int P = pt->p;
    const size_t shm = fft_smem(P);
    PACT_TRY(ensure_smem((const void*)patch_fft_kernel, shm, "patch_fft: shared memory attribute"));
    dim3 grid(m, pt->n);
    // one thread per register tile of the larger pass (at most 256): fewer idle
    // warps at the barriers and more CTAs per SM for small patches
    const int half = P / 2 + 1;
    const int tiles = std::max(((P + kRA - 1) / kRA) * ((half + kRV - 1) / kRV),
                               ((P + kCU - 1) / kCU) * ((half + kCV - 1) / kCV));
    const int threads = std::min(256, (tiles + 31) / 32 * 32);
    patch_fft_kernel<<<grid, threads, shm, as_stream(stream)>>>(make_geo(g), P, m,
                                                           reinterpret_cast<const int2*>(pt->centres),
                                                           inv_two_sigma2(pt->window_fwhm), stack,
                                                           reinterpret_cast<float2*>(Y));
    return check_launch("patch_fft kernel");
}

namespace pact {
namespace {

pact_status run_stitch(const pact_geometry* g, const pact_patches* pt, int m, const float* Xhat, float* image,
                       void* ws, size_t ws_bytes, void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    if (!Xhat || !image || !ws) return fail(PACT_ERR_INVALID_ARG, "stitch: Xhat, image and ws must not be NULL");
    if (m < 1 || m > 65535) return fail(PACT_ERR_INVALID_ARG, "stitch: channel count %d out of range", m);
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const size_t plane = (size_t)g->img_h * g->img_w * sizeof(double);
    const size_t need = align_up((size_t)(m + 1) * plane, 256);
    if (ws_bytes < need) return fail(PACT_ERR_INVALID_ARG, "stitch: workspace too small: %zu < %zu", ws_bytes, need);
    cudaStream_t st = as_stream(stream);
    double* num = static_cast<double*>(ws);
    double* den = num + (size_t)m * g->img_h * g->img_w;
    if (cudaMemsetAsync(ws, 0, (size_t)(m + 1) * plane, st) != cudaSuccess) return check_launch("stitch: memset");
    const int P = pt->p;
    const size_t shm = stitch_smem(P);
    PACT_TRY(ensure_smem((const void*)stitch_kernel, shm, "stitch: shared memory attribute"));
    stitch_kernel<<<dim3(pt->n, m), 256, shm, st>>>(make_geo(g), P, reinterpret_cast<const int2*>(pt->centres),
                                                    inv_two_sigma2(pt->window_fwhm),
                                                    reinterpret_cast<const float2*>(Xhat), num, den);
    PACT_TRY(check_launch("stitch kernel"));
    const int n = g->img_h * g->img_w;
    stitch_divide_kernel<<<dim3((n + 255) / 256, m), 256, 0, st>>>(n, num, den, image);
    return check_launch("stitch divide");
}

}  // namespace
}  // namespace pact

extern "C" size_t pact_stitch_workspace_size(const pact_geometry* g, const pact_patches* pt) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK) return 0;
    return align_up(2 * (size_t)g->img_h * g->img_w * sizeof(double), 256);
}

extern "C" pact_status pact_stitch(const pact_geometry* g, const pact_patches* pt, const float* Xhat,
                                   float* image, void* ws, size_t ws_bytes, void* stream) {
    return run_stitch(g, pt, 1, Xhat, image, ws, ws_bytes, stream);
}

extern "C" size_t pact_stitch_channels_workspace_size(const pact_geometry* g, const pact_patches* pt, int m) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK || m < 1) return 0;
    return align_up((size_t)(m + 1) * g->img_h * g->img_w * sizeof(double), 256);
}

extern "C" pact_status pact_stitch_channels(const pact_geometry* g, const pact_patches* pt, int m, const float* Y,
                                            float* stack, void* ws, size_t ws_bytes, void* stream) {
    return run_stitch(g, pt, m, Y, stack, ws, ws_bytes, stream);
}
