// TV regulariser of Eq. 7 (pact_tv) and the Adam update of Sec. 3.3
// (pact_adam_step) on the GPU.
#include <math.h>

#include "pact_internal.cuh"

namespace pact {
namespace {

__device__ __forceinline__ float sgn(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// One thread per node: subgradient; the value is reduced per CTA and added
// to *value with one atomic per CTA.
__global__ void __launch_bounds__(256) tv_kernel(int G, const float* sos, float lambda, float* value,
                                                 float* grad, int accumulate) {
    __shared__ float red[8];
    pdl_trigger();
    pdl_wait();
    const int GG = G * G;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    float part = 0.f;
    if (q < GG) {
        const int p = q / G, c = q - (q / G) * G;
        const float v = sos[q];
        float gq = 0.f;
        if (p + 1 < G) {
            const float dn = sos[q + G] - v;
            part += fabsf(dn);
            gq -= sgn(dn);
        }
        if (c + 1 < G) {
            const float rt = sos[q + 1] - v;
            part += fabsf(rt);
            gq -= sgn(rt);
        }
        if (p > 0) gq += sgn(v - sos[q - G]);
        if (c > 0) gq += sgn(v - sos[q - 1]);
        if (grad) grad[q] = accumulate ? fmaf(lambda, gq, grad[q]) : lambda * gq;
    }
    if (value) {
        const float tot = block_sum(part, red);
        if (threadIdx.x == 0) atomicAdd(value, lambda * tot);
    }
}

// counter (optional): [0] steps taken so far, [1] CTAs done with this step.
// Every thread reads [0] first; the last CTA to finish advances it, so the
// update needs no second kernel.
__global__ void adam_kernel(int n, float* param, const float* grad, float* m, float* v, float lr, float b1,
                            float b2, float eps, float bc1, float bc2, int* counter, const unsigned char* mask) {
    pdl_trigger();
    pdl_wait();
    if (counter) {  // t = steps so far + 1
        const float t = (float)(counter[0] + 1);
        bc1 = 1.f - powf(b1, t);
        bc2 = 1.f - powf(b2, t);
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        if (mask && !mask[q]) continue;
        const float g = grad[q];
        const float mq = fmaf(b1, m[q], (1.f - b1) * g);
        const float vq = fmaf(b2, v[q], (1.f - b2) * g * g);
        m[q] = mq;
        v[q] = vq;
        param[q] -= lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
    }
    if (counter) {
        // every thread of the CTA has used its read of counter[0] before this
        // barrier, and nothing else in the kernel depends on the counter, so
        // the completion count needs no fence
        __syncthreads();
        if (threadIdx.x == 0) {
            if (atomicAdd(counter + 1, 1) == (int)gridDim.x - 1) {   // all CTAs have read it
                counter[0] += 1;
                counter[1] = 0;
            }
        }
    }
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" pact_status pact_tv(const pact_geometry* g, const float* sos, float lambda, float* value,
                               float* dL_dsos, int accumulate, void* stream) {
    PACT_TRY(check_geometry(g));
    if (!sos) return fail(PACT_ERR_INVALID_ARG, "tv: sos is NULL");
    if (!value && !dL_dsos) return PACT_OK;
    cudaStream_t st = as_stream(stream);
    if (value && !accumulate && cudaMemsetAsync(value, 0, sizeof(float), st) != cudaSuccess)
        return check_launch("tv: memset");
    const int GG = g->sos_g * g->sos_g;
    if (launch_pdl(tv_kernel, dim3((GG + 255) / 256), dim3(256), 0, st, g->sos_g, sos, lambda, value, dL_dsos,
                   accumulate) != cudaSuccess)
        return check_launch("tv kernel");
    return check_launch("tv kernel");
}

extern "C" pact_status pact_adam_step(int n, float* param, const float* grad, float* m, float* v, int step,
                                      int* step_counter, float lr, float beta1, float beta2, float eps,
                                      const unsigned char* mask, void* stream) {
    if (n < 0) return fail(PACT_ERR_INVALID_ARG, "adam: n must be >= 0");
    if (n == 0) return PACT_OK;
    if (!param || !grad || !m || !v) return fail(PACT_ERR_INVALID_ARG, "adam: null pointer");
    if (!step_counter && step < 1) return fail(PACT_ERR_INVALID_ARG, "adam: step must be >= 1");
    if (step < 1) step = 1;
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f))
        return fail(PACT_ERR_INVALID_ARG, "adam: betas must be in [0, 1)");
    PACT_TRY(require_sms());
    const float bc1 = (float)(1.0 - pow((double)beta1, step));
    const float bc2 = (float)(1.0 - pow((double)beta2, step));
    const int blocks = (n + 255) / 256 < 4 * num_sms() ? (n + 255) / 256 : 4 * num_sms();
    if (launch_pdl(adam_kernel, dim3(blocks), dim3(256), 0, as_stream(stream), n, param, grad, m, v, lr, beta1, beta2,
                   eps, bc1, bc2, step_counter, mask) != cudaSuccess)
        return check_launch("adam kernel");
    return check_launch("adam kernel");
}
