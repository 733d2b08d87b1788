// Eq. 1 on the GPU: delay-and-sum stack for M extra delays (pact_das_stack).
//
// One thread per pixel; every thread walks the ring, taking M linearly
// interpolated taps of S(., n) per transducer:
//     q_j = |r' - r_n| fs/v0 - (d_j/v0 + t0) fs.
// Tiled kernel (das_tile_kernel): a CTA is a 32 x 8 pixel tile.  For each
// transducer the samples its pixels can touch form one short window (the
// spread of |r' - r_n| over the tile plus the spread of the delays); the CTA
// stages the windows of kChunk transducers at a time in shared memory (zero
// outside the record) as linear pieces a_k + q b_k, so that a tap is one
// 64-bit shared load and one FMA, and neighbouring pixels read neighbouring
// addresses.  Problems whose window would not fit take das_kernel, which
// reads S from global memory.
#include <algorithm>
#include <cmath>

#include "pact_internal.cuh"

namespace pact {
namespace {

constexpr float kTwoPi = 6.283185307179586f;

struct DasArgs {
    Geo g;
    const float* rf;
    int n_s;
    float a;                           // fs / v0 [samples per metre]
    float qoff[PACT_MAX_CHANNELS];     // (d_j / v0 + t0) fs
    int M;
    float* stack;
};

template <int MMAX>
__global__ void __launch_bounds__(256) das_kernel(const DasArgs a) {
    extern __shared__ float2 rn[];
    const int n_t = a.g.n_t;
    for (int n = threadIdx.x; n < n_t; n += blockDim.x) {
        float sn, cs;
        sincosf(kTwoPi * ((float)n / (float)n_t) + a.g.phase, &sn, &cs);
        rn[n] = make_float2(a.g.R * cs, a.g.R * sn);
    }
    __syncthreads();
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    const int npix = a.g.H * a.g.W;
    if (pix >= npix) return;
    const int row = pix / a.g.W, col = pix - (pix / a.g.W) * a.g.W;
    const float2 p = pixel_xy(a.g, row, col);
    float acc[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) acc[j] = 0.f;
    for (int n = 0; n < n_t; ++n) {
        const float ddx = p.x - rn[n].x, ddy = p.y - rn[n].y;
        const float base = sqrtf(ddx * ddx + ddy * ddy) * a.a;
        const float* s = a.rf + (size_t)n * a.n_s;
#pragma unroll
        for (int j = 0; j < MMAX; ++j) {
            if (j < a.M) {
                const float q = base - a.qoff[j];
                const float q0 = floorf(q);
                const float f = q - q0;
                const int i0 = (int)q0;
                const float s0 = (i0 >= 0 && i0 < a.n_s) ? __ldg(s + i0) : 0.f;
                const float s1 = (i0 + 1 >= 0 && i0 + 1 < a.n_s) ? __ldg(s + i0 + 1) : 0.f;
                acc[j] += fmaf(f, s1 - s0, s0);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MMAX; ++j)
        if (j < a.M) a.stack[(size_t)j * npix + pix] = acc[j];
}

constexpr int kTX = 32, kTY = 8;       // tile: 4 x 2 warps of 8 x 4 pixels
constexpr int kWin = 128;               // samples per staged window
constexpr int kChunk = 32;              // transducers staged at a time

struct DasTileArgs {
    DasArgs d;
    float qmax;                         // max_j qoff_j
    float dmarg;                        // margin on the tile's distance range [m]
};

// Distance range from r to the pixel centres of the tile [x0, x1] x [y0, y1].
__device__ __forceinline__ float2 rect_range(float rx, float ry, float x0, float x1, float y0, float y1) {
    const float cx = fminf(fmaxf(rx, x0), x1), cy = fminf(fmaxf(ry, y0), y1);
    const float fx = fmaxf(fabsf(rx - x0), fabsf(rx - x1)), fy = fmaxf(fabsf(ry - y0), fabsf(ry - y1));
    return make_float2(sqrtf((rx - cx) * (rx - cx) + (ry - cy) * (ry - cy)), sqrtf(fx * fx + fy * fy));
}

template <int MMAX, bool EXACT>   // EXACT: M == MMAX
__global__ void __launch_bounds__(kTX * kTY) das_tile_kernel(const DasTileArgs t) {
    // win[n][k] = (a_k, b_k): the linear piece of S(., n) on [ws + k, ws + k + 1]
    // written as S(ws + q) = a_k + q b_k, q measured from the window start
    __shared__ float2 win[kChunk][kWin];
    __shared__ float2 rn_s[kChunk];
    __shared__ int ws_s[kChunk];
    const DasArgs& a = t.d;
    const int n_t = a.g.n_t, W = a.g.W, H = a.g.H;
    const int c0 = blockIdx.x * kTX, r0 = blockIdx.y * kTY;
    // a warp covers an 8 x 4 pixel block: its taps of one transducer fall within
    // about ten consecutive window entries, so its shared loads do not conflict
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = c0 + (wid & (kTX / 8 - 1)) * 8 + (lane & 7);
    const int row = r0 + (wid / (kTX / 8)) * 4 + (lane >> 3);
    const bool inside = col < W && row < H;
    const float2 p = pixel_xy(a.g, min(row, H - 1), min(col, W - 1));
    const float2 lo = pixel_xy(a.g, r0, c0), hi = pixel_xy(a.g, min(r0 + kTY, H) - 1, min(c0 + kTX, W) - 1);
    float acc[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) acc[j] = 0.f;
    for (int nc = 0; nc < n_t; nc += kChunk) {
        const int cn = min(kChunk, n_t - nc);
        __syncthreads();                                  // the previous chunk is consumed
        if (threadIdx.x < cn) {
            const int n = nc + threadIdx.x;
            float sn, cs;
            sincosf(kTwoPi * ((float)n / (float)n_t) + a.g.phase, &sn, &cs);
            const float rx = a.g.R * cs, ry = a.g.R * sn;
            rn_s[threadIdx.x] = make_float2(rx, ry);
            const float2 dr = rect_range(rx, ry, lo.x, hi.x, lo.y, hi.y);
            // first sample any pixel of the tile can touch, with a margin of two
            ws_s[threadIdx.x] = (int)floorf((dr.x - t.dmarg) * a.a - t.qmax) - 2;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < cn * kWin; e += blockDim.x) {
            const int nl = e / kWin, k = e - nl * kWin, q = ws_s[nl] + k;
            const float* s = a.rf + (size_t)(nc + nl) * a.n_s;
            const float s0 = (q >= 0 && q < a.n_s) ? __ldg(s + q) : 0.f;
            const float s1 = (q + 1 >= 0 && q + 1 < a.n_s) ? __ldg(s + q + 1) : 0.f;
            const float b = s1 - s0;
            win[nl][k] = make_float2(fmaf(-(float)k, b, s0), b);
        }
        __syncthreads();
        for (int nl = 0; nl < cn; ++nl) {
            const float2 r = rn_s[nl];
            const float ddx = p.x - r.x, ddy = p.y - r.y;
            // sample position relative to the window start: q_j - ws (ws exact in FP32)
            const float base = sqrtf(ddx * ddx + ddy * ddy) * a.a - (float)ws_s[nl];
            // shared address of entry floor(q) = bits(q + 2^23 - 1/2) * 8 + this offset
            // (32-bit wrap-around)
            const unsigned off = (unsigned)__cvta_generic_to_shared(win[nl]) - 0x4B000000u * 8u;
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (EXACT || j < a.M) {
                    const float q = base - a.qoff[j];                  // in [2, kWin - 2] by the window
                    const float tq = q + 8388607.5f;                   // floor without conversions
                    const unsigned addr = (unsigned)__float_as_int(tq) * 8u + off;
                    float pa, pb;
                    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(pa), "=f"(pb) : "r"(addr));
                    acc[j] += fmaf(q, pb, pa);
                }
            }
        }
    }
    if (!inside) return;
    const int npix = H * W, pix = row * W + col;
#pragma unroll
    for (int j = 0; j < MMAX; ++j)
        if (EXACT || j < a.M) a.stack[(size_t)j * npix + pix] = acc[j];
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" pact_status pact_das_stack(const pact_geometry* g, const float* rf, int n_s, float fs, float t0,
                                      const float* d, int m, float* stack, void* stream) {
    PACT_TRY(check_geometry(g));
    if (!rf || !d || !stack) return fail(PACT_ERR_INVALID_ARG, "das_stack: null pointer");
    if (n_s < 1) return fail(PACT_ERR_INVALID_ARG, "das_stack: n_s must be >= 1");
    if (!(fs > 0.f)) return fail(PACT_ERR_INVALID_ARG, "das_stack: fs must be > 0");
    if (m < 1) return fail(PACT_ERR_INVALID_ARG, "das_stack: m must be >= 1");
    if (m > PACT_MAX_CHANNELS) return fail(PACT_ERR_SHAPE, "das_stack: m must be <= %d", PACT_MAX_CHANNELS);
    DasArgs a;
    a.g = make_geo(g);
    a.rf = rf;
    a.n_s = n_s;
    a.a = (float)((double)fs / (double)g->v0);
    for (int j = 0; j < PACT_MAX_CHANNELS; ++j)
        a.qoff[j] = j < m ? (float)(((double)d[j] / (double)g->v0 + (double)t0) * (double)fs) : 0.f;
    a.M = m;
    a.stack = stack;
    const size_t shm = (size_t)g->n_t * sizeof(float2);
    const int npix = g->img_h * g->img_w;
    const int blocks = (npix + 255) / 256;
    cudaStream_t st = as_stream(stream);
    // tiled path when a tile's window fits: distance spread over the tile (its
    // diagonal) + delay spread, in samples, plus the margins
    double qmin = 1e300, qmax = -1e300;
    for (int j = 0; j < m; ++j) {
        qmin = std::min(qmin, (double)a.qoff[j]);
        qmax = std::max(qmax, (double)a.qoff[j]);
    }
    const double diag = (double)g->dx * std::sqrt((double)(kTX - 1) * (kTX - 1) + (double)(kTY - 1) * (kTY - 1));
    const double marg = 1e-3 * diag + 1e-9;        // FP32 rounding of the distances, generously
    const double need = (diag + 2.0 * marg) * (double)a.a + (qmax - qmin) + 8.0;
    if (need <= kWin && std::fabs(qmax) < 1e6 && std::fabs(qmin) < 1e6 && g->n_t < (1 << 24)) {
        DasTileArgs t;
        t.d = a;
        t.qmax = (float)qmax;
        t.dmarg = (float)marg;
        const dim3 grid((g->img_w + kTX - 1) / kTX, (g->img_h + kTY - 1) / kTY);
        if (m == 8) das_tile_kernel<8, true><<<grid, kTX * kTY, 0, st>>>(t);
        else if (m == 16) das_tile_kernel<16, true><<<grid, kTX * kTY, 0, st>>>(t);
        else if (m == 32) das_tile_kernel<32, true><<<grid, kTX * kTY, 0, st>>>(t);
        else if (m == 64) das_tile_kernel<64, true><<<grid, kTX * kTY, 0, st>>>(t);
        else if (m < 8) das_tile_kernel<8, false><<<grid, kTX * kTY, 0, st>>>(t);
        else if (m < 16) das_tile_kernel<16, false><<<grid, kTX * kTY, 0, st>>>(t);
        else if (m < 32) das_tile_kernel<32, false><<<grid, kTX * kTY, 0, st>>>(t);
        else das_tile_kernel<64, false><<<grid, kTX * kTY, 0, st>>>(t);
        return check_launch("das_stack kernel");
    }
#define PACT_DAS(MM)                                                                                 \
    do {                                                                                             \
        PACT_TRY(ensure_smem((const void*)das_kernel<MM>, shm, "das_stack: shared memory attribute")); \
        das_kernel<MM><<<blocks, 256, shm, st>>>(a);                                                 \
    } while (0)
    if (m <= 8) PACT_DAS(8);
    else if (m <= 16) PACT_DAS(16);
    else if (m <= 32) PACT_DAS(32);
    else PACT_DAS(64);
#undef PACT_DAS
    return check_launch("das_stack kernel");
}
