// Eq. 1 on the GPU: delay-and-sum stack for M extra delays (pact_das_stack).
//
// One thread per pixel; the CTA stages the transducer positions in shared
// memory and every thread walks the ring, taking M linearly interpolated
// taps of S(., n) per transducer:  q_j = |r' - r_n| fs/v0 - (d_j/v0 + t0) fs.
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
