// Sec. S1.4 on the GPU: Gaussian-windowed patch spectra (pact_patch_fft) and
// stitching of deconvolved patches (pact_stitch).
//
// Both run once per recovery, so they use a direct separable DFT from shared
// memory (one CTA per patch and channel): P x P real samples, a twiddle table
// exp(-2 pi j t / P), a row pass to the P/2+1 half-spectrum columns and a
// column pass, in FP32 (error ~ sqrt(P) ulp).
#include <algorithm>

#include "pact_internal.cuh"

namespace pact {
namespace {

__global__ void __launch_bounds__(256) patch_fft_kernel(Geo g, int P, int M, const int2* centres,
                                                        float inv_2s2, const float* stack, float2* Y) {
    extern __shared__ float sm[];
    const int half = P / 2 + 1;
    float* x = sm;                                          // [P*P]
    float2* R = reinterpret_cast<float2*>(sm + P * P);      // [P*half]
    float2* tw = R + P * half;                              // [P]
    const int i = blockIdx.y, j = blockIdx.x;
    const int2 c = centres[i];
    const int r0 = c.x - P / 2, c0 = c.y - P / 2;
    for (int t = threadIdx.x; t < P; t += blockDim.x) tw[t] = cis_pi(-2.f * t / P);
    const float* img = stack + (size_t)j * g.H * g.W;
    for (int q = threadIdx.x; q < P * P; q += blockDim.x) {
        const int a = q / P, b = q - (q / P) * P;
        const int row = r0 + a, col = c0 + b;
        float val = 0.f;
        if (row >= 0 && row < g.H && col >= 0 && col < g.W) val = img[(size_t)row * g.W + col];
        const float oa = (a - P / 2) * g.dx, ob = (b - P / 2) * g.dx;
        x[q] = val * expf(-(oa * oa + ob * ob) * inv_2s2);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < P * half; q += blockDim.x) {
        const int a = q / half, v = q - (q / half) * half;
        const float* xr = x + a * P;
        float re = 0.f, im = 0.f;
        int idx = 0;
        for (int b = 0; b < P; ++b) {
            const float2 t = tw[idx];
            re = fmaf(xr[b], t.x, re);
            im = fmaf(xr[b], t.y, im);
            idx += v;
            if (idx >= P) idx -= P;
        }
        R[q] = make_float2(re, im);
    }
    __syncthreads();
    const float inv_p = 1.f / P;
    float2* out = Y + ((size_t)i * M + j) * P * half;
    for (int q = threadIdx.x; q < P * half; q += blockDim.x) {
        const int u = q / half, v = q - (q / half) * half;
        float re = 0.f, im = 0.f;
        int idx = 0;
        for (int a = 0; a < P; ++a) {
            const float2 r = R[a * half + v];
            const float2 t = tw[idx];
            re = fmaf(r.x, t.x, fmaf(-r.y, t.y, re));
            im = fmaf(r.x, t.y, fmaf(r.y, t.x, im));
            idx += u;
            if (idx >= P) idx -= P;
        }
        out[q] = make_float2(re * inv_p, im * inv_p);
    }
}

// Inverse half-spectrum DFT of patch i = blockIdx.x, channel j = blockIdx.y
// (X [N][m][P][P/2+1]), then scatter-add into the channel's numerator image
// and, for channel 0, into the window-sum image.
__global__ void __launch_bounds__(256) stitch_kernel(Geo g, int P, const int2* centres, float inv_2s2,
                                                     const float2* X, float* num, float* den) {
    extern __shared__ float sm[];
    const int half = P / 2 + 1;
    float2* Z = reinterpret_cast<float2*>(sm);     // [P*half]
    float2* tw = Z + P * half;                     // [P]: exp(+2 pi j t / P)
    const int i = blockIdx.x;
    const int2 c = centres[i];
    const int r0 = c.x - P / 2, c0 = c.y - P / 2;
    for (int t = threadIdx.x; t < P; t += blockDim.x) tw[t] = cis_pi(2.f * t / P);
    __syncthreads();
    const int j = blockIdx.y, m = gridDim.y;
    const float2* Xi = X + ((size_t)i * m + j) * P * half;
    num += (size_t)j * g.H * g.W;
    for (int q = threadIdx.x; q < P * half; q += blockDim.x) {
        const int a = q / half, v = q - (q / half) * half;
        float re = 0.f, im = 0.f;
        int idx = 0;
        for (int u = 0; u < P; ++u) {
            const float2 xv = Xi[u * half + v];
            const float2 t = tw[idx];
            re = fmaf(xv.x, t.x, fmaf(-xv.y, t.y, re));
            im = fmaf(xv.x, t.y, fmaf(xv.y, t.x, im));
            idx += a;
            if (idx >= P) idx -= P;
        }
        Z[q] = make_float2(re, im);
    }
    __syncthreads();
    const float inv_p = 1.f / P;
    for (int q = threadIdx.x; q < P * P; q += blockDim.x) {
        const int a = q / P, b = q - (q / P) * P;
        const int row = r0 + a, col = c0 + b;
        if (row < 0 || row >= g.H || col < 0 || col >= g.W) continue;
        const float2* za = Z + a * half;
        float s = za[0].x + ((b & 1) ? -za[P / 2].x : za[P / 2].x);
        int idx = b;
        float acc = 0.f;
        for (int v = 1; v < P / 2; ++v) {
            const float2 t = tw[idx];
            acc = fmaf(za[v].x, t.x, fmaf(-za[v].y, t.y, acc));
            idx += b;
            if (idx >= P) idx -= P;
        }
        s = fmaf(2.f, acc, s);
        const float oa = (a - P / 2) * g.dx, ob = (b - P / 2) * g.dx;
        atomicAdd(num + (size_t)row * g.W + col, s * inv_p);
        if (j == 0) atomicAdd(den + (size_t)row * g.W + col, expf(-(oa * oa + ob * ob) * inv_2s2));
    }
}

// out[j][q] = num[j][q] / den[q] (0 where no window reaches), j = blockIdx.y.
__global__ void stitch_divide_kernel(int n, const float* num, const float* den, float* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const size_t o = (size_t)blockIdx.y * n + q;
    const float d = den[q];
    out[o] = d > 0.f ? num[o] / d : 0.f;
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
    const int P = pt->p, half = P / 2 + 1;
    const size_t shm = (size_t)P * P * sizeof(float) + (size_t)(P * half + P) * sizeof(float2);
    PACT_TRY(ensure_smem((const void*)patch_fft_kernel, shm, "patch_fft: shared memory attribute"));
    dim3 grid(m, pt->n);
    patch_fft_kernel<<<grid, 256, shm, as_stream(stream)>>>(make_geo(g), P, m,
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
    const size_t plane = (size_t)g->img_h * g->img_w * sizeof(float);
    const size_t need = align_up((size_t)(m + 1) * plane, 256);
    if (ws_bytes < need) return fail(PACT_ERR_INVALID_ARG, "stitch: workspace too small: %zu < %zu", ws_bytes, need);
    cudaStream_t st = as_stream(stream);
    float* num = static_cast<float*>(ws);
    float* den = num + (size_t)m * g->img_h * g->img_w;
    if (cudaMemsetAsync(ws, 0, (size_t)(m + 1) * plane, st) != cudaSuccess) return check_launch("stitch: memset");
    const int P = pt->p, half = P / 2 + 1;
    const size_t shm = (size_t)(P * half + P) * sizeof(float2);
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
    return align_up(2 * (size_t)g->img_h * g->img_w * sizeof(float), 256);
}

extern "C" pact_status pact_stitch(const pact_geometry* g, const pact_patches* pt, const float* Xhat,
                                   float* image, void* ws, size_t ws_bytes, void* stream) {
    return run_stitch(g, pt, 1, Xhat, image, ws, ws_bytes, stream);
}

extern "C" size_t pact_stitch_channels_workspace_size(const pact_geometry* g, const pact_patches* pt, int m) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK || m < 1) return 0;
    return align_up((size_t)(m + 1) * g->img_h * g->img_w * sizeof(float), 256);
}

extern "C" pact_status pact_stitch_channels(const pact_geometry* g, const pact_patches* pt, int m, const float* Y,
                                            float* stack, void* ws, size_t ws_bytes, void* stream) {
    return run_stitch(g, pt, m, Y, stack, ws, ws_bytes, stream);
}
