// Synthetic ring channel data (pact_rf_synth): the input of Eq. 1 for
// end-to-end runs, with straight-ray times of flight through the SOS grid
// (Eq. 2-3) and the differentiated pulse of Sec. S1.1.
//
// The pixels are taken in passes of B (B set by the workspace).  Per pass:
//   1. the ray kernel of rays.cu integrates w(p, n) for every emitting pixel p
//      of the pass and every transducer n, transposed to wT[n][p];
//   2. one CTA per transducer n holds its record rf[n][0 .. n_s) in shared
//      memory; each warp sets up 32 pixels at once (one per lane: time of
//      flight in FP64, amplitude), then adds their pulses one pixel at a time,
//      the lanes covering consecutive samples around the arrival, and the CTA
//      writes the record back (first pass: from zero).
#include <algorithm>
#include <cmath>

#include "pact_internal.cuh"

namespace pact {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxSamples = 49152;     // 192 KB of shared memory per record
constexpr int kMaxHalf = 1024;         // pulse support half-width [samples]

struct RfArgs {
    int n_t, W, H;
    double R, phase, dx;   // receiving ring radius (R + ring_dr), phase, pixel pitch
    double a;              // fs / v0 [samples per metre]
    double qoff;           // t0 fs
    float inv_sig;         // 1 / (sigma fs)
    float spread;
    int half;              // ceil(6 sigma fs)
    int n_s;
    const float* p0;
    const float* wT;
    int ld, pix0, npix;
    float* rf;
    int first;
};

__global__ void __launch_bounds__(kThreads) rf_scatter_kernel(const RfArgs a) {
    extern __shared__ float rec[];
    const int n = blockIdx.x;
    float* row = a.rf + (size_t)n * a.n_s;
    for (int q = threadIdx.x; q < a.n_s; q += blockDim.x) rec[q] = a.first ? 0.f : row[q];
    double sn, cs;
    sincospi(2.0 * n / a.n_t + a.phase * 0.31830988618379067, &sn, &cs);
    const double rx = a.R * cs, ry = a.R * sn;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* w = a.wT + (size_t)n * a.ld;
    const int span = 2 * a.half + 2;           // samples floor(q_c) - half .. floor(q_c) + half + 1
    for (int base = warp * 32; base < a.npix; base += nw * 32) {
        const int q = base + lane;
        float amp = 0.f, fr = 0.f;
        int k0 = 0;
        if (q < a.npix) {
            const int pix = a.pix0 + q;
            const float p = a.p0[pix];
            if (p != 0.f) {
                const int prow = pix / a.W, pcol = pix - (pix / a.W) * a.W;
                const double x = (pcol - 0.5 * (a.W - 1)) * a.dx, y = (prow - 0.5 * (a.H - 1)) * a.dx;
                const double ex = rx - x, ey = ry - y;
                const double L = sqrt(ex * ex + ey * ey);
                // sample position of the arrival: (tau - t0) fs, tau = (L - w) / v0
                double qc = (L - (double)w[q]) * a.a - a.qoff;
                qc = fmin(fmax(qc, -1.0e9), 1.0e9);
                const double fl = floor(qc);
                k0 = (int)fl - a.half;
                fr = (float)(qc - fl);
                amp = a.spread != 0.f ? p * powf((float)(a.R / L), a.spread) : p;
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, amp != 0.f);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const float am = __shfl_sync(0xffffffffu, amp, src);
            const float f = __shfl_sync(0xffffffffu, fr, src);
            const int kk = __shfl_sync(0xffffffffu, k0, src);
            for (int j = lane; j < span; j += 32) {
                const int k = kk + j;
                if (k >= 0 && k < a.n_s) {
                    const float u = ((float)(j - a.half) - f) * a.inv_sig;
                    atomicAdd(rec + k, am * (1.f - u * u) * __expf(-0.5f * u * u));
                }
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.n_s; q += blockDim.x) row[q] = rec[q];
}

// Transducer band-limit (a model mismatch for robustness studies): every
// channel filtered along time by the zero-phase impulse response
//   h_k = (2 / Z) exp(-tau_k^2 / (2 s_t^2)) cos(2 pi fc tau_k),  tau_k = k / fs,
// |k| <= K, Z the sum of the window, s_t = 1 / (2 pi s_f) and s_f = frac_bw fc
// / (2 sqrt(2 ln 2)) (full width at half amplitude frac_bw fc); samples
// outside the record are zero.  CTA (tile of kBpTile samples, channel): the
// taps (computed per CTA, the window sum in a fixed order) and the tile with
// its K-sample halos in shared memory; one thread per output sample.
constexpr int kBpTile = 256;
constexpr int kBpMaxK = 512;

__global__ void __launch_bounds__(kBpTile) rf_bandpass_kernel(const float* in, float* out, int n_s, float inv_fs,
                                                              float fc, float s_t, int K) {
    extern __shared__ float sm_bp[];
    float* taps = sm_bp;                     // [2K + 1]
    float* x = sm_bp + 2 * K + 1;            // [kBpTile + 2K]
    __shared__ float red[kBpTile / 32];
    const int n = blockIdx.y, q0 = blockIdx.x * kBpTile, tid = threadIdx.x;
    float zs = 0.f;
    for (int j = tid; j <= 2 * K; j += blockDim.x) {
        const float tau = (float)(j - K) * inv_fs, u = tau / s_t;
        const float env = expf(-0.5f * u * u);
        taps[j] = env * cospif(2.f * fc * tau);
        zs += env;
    }
    const float z = block_sum(zs, red);      // valid in thread 0
    if (tid == 0) red[0] = 2.f / z;
    const float* row = in + (size_t)n * n_s;
    for (int j = tid; j < kBpTile + 2 * K; j += blockDim.x) {
        const int q = q0 - K + j;
        x[j] = q >= 0 && q < n_s ? row[q] : 0.f;
    }
    __syncthreads();
    const float scale = red[0];
    const int q = q0 + tid;
    if (q >= n_s) return;
    // out[q] = sum_k h_k in[q - k]: x[tid + K - k] with k = j - K
    float acc = 0.f;
    for (int j = 0; j <= 2 * K; ++j) acc = fmaf(taps[j], x[tid + 2 * K - j], acc);
    out[(size_t)n * n_s + q] = scale * acc;
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" pact_status pact_rf_bandpass(const float* rf_in, float* rf_out, int n_t, int n_s, float fs, float fc,
                                        float frac_bw, void* stream) {
    if (!rf_in || !rf_out) return fail(PACT_ERR_INVALID_ARG, "rf_bandpass: rf_in and rf_out must not be NULL");
    if (rf_in == rf_out) return fail(PACT_ERR_INVALID_ARG, "rf_bandpass: rf_in and rf_out must be different buffers");
    if (n_t < 1 || n_s < 1) return fail(PACT_ERR_INVALID_ARG, "rf_bandpass: n_t and n_s must be >= 1");
    if (n_t > 65535) return fail(PACT_ERR_SHAPE, "rf_bandpass: n_t must be <= 65535");
    if (!(fs > 0.f) || !isfinite(fs)) return fail(PACT_ERR_INVALID_ARG, "rf_bandpass: fs must be finite and > 0");
    if (!(fc > 0.f) || !(fc < 0.5f * fs)) return fail(PACT_ERR_INVALID_ARG, "rf_bandpass: fc must be in (0, fs / 2)");
    if (!(frac_bw > 0.f) || !(frac_bw <= 2.f)) return fail(PACT_ERR_INVALID_ARG, "rf_bandpass: frac_bw must be in (0, 2]");
    const double s_f = (double)frac_bw * fc / (2.0 * sqrt(2.0 * log(2.0)));
    const double s_t = 1.0 / (2.0 * 3.141592653589793 * s_f);
    const double Kd = ceil(4.0 * s_t * fs);
    if (Kd > kBpMaxK) return fail(PACT_ERR_SHAPE, "rf_bandpass: %g taps per side, at most %d", Kd, kBpMaxK);
    const int K = (int)Kd;
    const size_t smem = (size_t)(2 * K + 1 + kBpTile + 2 * K) * sizeof(float);
    PACT_TRY(ensure_smem((const void*)rf_bandpass_kernel, smem, "rf_bandpass: shared memory attribute"));
    const dim3 grid((n_s + kBpTile - 1) / kBpTile, n_t);
    rf_bandpass_kernel<<<grid, kBpTile, smem, as_stream(stream)>>>(rf_in, rf_out, n_s, (float)(1.0 / fs), fc,
                                                                  (float)s_t, K);
    return check_launch("rf_bandpass kernel");
}

extern "C" size_t pact_rf_synth_workspace_size(const pact_geometry* g, int pixels_per_pass) {
    if (check_geometry(g) != PACT_OK || pixels_per_pass < 1) return 0;
    return align_up((size_t)g->n_t * (size_t)pixels_per_pass * sizeof(float), 256);
}

extern "C" pact_status pact_rf_synth(const pact_geometry* g, const float* p0, const float* sos,
                                     const pact_rf_params* rp, float* rf, void* ws, size_t ws_bytes, void* stream) {
    PACT_TRY(check_geometry(g));
    if (!p0 || !sos || !rp || !rf) return fail(PACT_ERR_INVALID_ARG, "rf_synth: p0, sos, rp and rf must not be NULL");
    if (!ws) return fail(PACT_ERR_INVALID_ARG, "rf_synth: workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (!(rp->fs > 0.f) || !isfinite(rp->fs)) return fail(PACT_ERR_INVALID_ARG, "rf_synth: fs must be finite and > 0");
    if (!isfinite(rp->t0)) return fail(PACT_ERR_INVALID_ARG, "rf_synth: t0 must be finite");
    if (!(rp->sigma > 0.f) || !isfinite(rp->sigma))
        return fail(PACT_ERR_INVALID_ARG, "rf_synth: sigma must be finite and > 0");
    if (!isfinite(rp->spread)) return fail(PACT_ERR_INVALID_ARG, "rf_synth: spread must be finite");
    if (!isfinite(rp->ring_dr) || !(g->ring_radius + rp->ring_dr > 0.f))
        return fail(PACT_ERR_INVALID_ARG, "rf_synth: ring_radius + ring_dr must be > 0");
    if (rp->n_s < 1 || rp->n_s > kMaxSamples)
        return fail(PACT_ERR_SHAPE, "rf_synth: n_s must be in [1, %d]", kMaxSamples);
    const double sig_s = (double)rp->sigma * (double)rp->fs;
    if (6.0 * sig_s > kMaxHalf) return fail(PACT_ERR_SHAPE, "rf_synth: 6 sigma fs must be <= %d samples", kMaxHalf);
    const size_t per_pix = (size_t)g->n_t * sizeof(float);
    if (ws_bytes < per_pix) return fail(PACT_ERR_INVALID_ARG, "rf_synth: workspace too small: %zu < %zu", ws_bytes, per_pix);
    const int npix_all = g->img_h * g->img_w;
    const int B = (int)std::min<size_t>((size_t)npix_all, ws_bytes / per_pix);
    float* wT = static_cast<float*>(ws);
    cudaStream_t st = as_stream(stream);

    pact_geometry gs = *g;                      // the receiving ring of the synthesis
    gs.ring_radius = g->ring_radius + rp->ring_dr;
    const size_t smem = (size_t)rp->n_s * sizeof(float);
    PACT_TRY(ensure_smem((const void*)rf_scatter_kernel, smem, "rf_synth: shared memory attribute"));

    RfArgs a;
    a.n_t = g->n_t;
    a.W = g->img_w;
    a.H = g->img_h;
    a.R = (double)gs.ring_radius;
    a.phase = (double)g->ring_phase;
    a.dx = (double)g->dx;
    a.a = (double)rp->fs / (double)g->v0;
    a.qoff = (double)rp->t0 * (double)rp->fs;
    a.inv_sig = (float)(1.0 / sig_s);
    a.spread = rp->spread;
    a.half = (int)ceil(6.0 * sig_s);
    a.n_s = rp->n_s;
    a.p0 = p0;
    a.wT = wT;
    a.ld = B;
    a.rf = rf;
    for (int pix0 = 0; pix0 < npix_all; pix0 += B) {
        const int npix = std::min(B, npix_all - pix0);
        PACT_TRY(launch_pixel_rays(&gs, sos, p0, pix0, npix, wT, B, st));
        a.pix0 = pix0;
        a.npix = npix;
        a.first = pix0 == 0;
        rf_scatter_kernel<<<g->n_t, kThreads, smem, st>>>(a);
        PACT_TRY(check_launch("rf_synth: pulse kernel"));
    }
    return PACT_OK;
}
