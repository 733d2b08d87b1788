// The paper's neural field (Sec. 3.3): a SIREN without hidden layers -- 256
// sine features of the node coordinates and a linear output -- plus an output
// scale and offset (1027 parameters):
//     v(x) = offset + scale (sum_f w2_f sin(omega0 (W1_f . x + b1_f)) + b2)
// on the SOS mask (v_bg outside), x the node position scaled to [-1, 1] per axis.
// With K = 2 inputs there is no matrix product worth a tensor core: both passes
// are FP32 on the CUDA cores.
//   forward : one thread per node, parameters in shared memory; z saved for the
//             backward pass.
//   backward: one thread per feature over a chunk of 64 nodes (dL/dv scaled by
//             the output scale staged in shared memory; enough chunks to fill
//             the SMs), per-chunk partial sums in the workspace, then a
//             fixed-order reduction (deterministic).
#include "pact_internal.cuh"

namespace pact {
namespace {

constexpr int kF = 256;                    // sine features
constexpr int kNP = 2 * kF + kF + kF + 3;  // 1027 parameters
constexpr int kOffB1 = 2 * kF, kOffW2 = 3 * kF, kOffB2 = 4 * kF, kOffScale = 4 * kF + 1, kOffOffset = 4 * kF + 2;
constexpr int kChunk = 64;                 // nodes per backward CTA (G = 128: 256 CTAs)
constexpr int kStride = 1088;              // partial-row stride (>= kNP + 2, multiple of 64)

struct SirenArgs {
    int G;
    float omega0, v_bg;
    const float* params;
    const unsigned char* mask;
    float* sos;
    float* z;               // [G*G] network output before scale/offset
    const float* dL_dsos;
    float* part;            // [chunks][kStride]
    float* dL_dparams;
    int accumulate;
};

__device__ __forceinline__ float coord(int q, int G) { return (q - 0.5f * (G - 1)) / (0.5f * (G - 1)); }

// kFwdLanes threads per node, lane l taking features l, l + kFwdLanes, ...
// (neighbouring lanes read neighbouring parameters, every node of a warp the
// same ones), the lanes' sums combined by a fixed butterfly.
constexpr int kFwdLanes = 4;

__global__ void __launch_bounds__(256) siren_fwd_kernel(const SirenArgs a) {
    __shared__ float p_s[kNP];
    for (int e = threadIdx.x; e < kNP; e += blockDim.x) p_s[e] = a.params[e];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int node = t / kFwdLanes, part = t % kFwdLanes;
    const int GG = a.G * a.G;
    const bool valid = node < GG;
    const int nd = valid ? node : 0;
    const float x = coord(nd % a.G, a.G), y = coord(nd / a.G, a.G);
    // sin(omega0 t) as sinpi((omega0 / pi) t): the argument reduction is exact in units of pi
    const float om_pi = a.omega0 * 0.3183098861837907f;
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 4
    for (int f = part; f < kF; f += 2 * kFwdLanes) {
        const int f1 = f + kFwdLanes;
        const float s0 = sinpif(om_pi * fmaf(p_s[2 * f], x, fmaf(p_s[2 * f + 1], y, p_s[kOffB1 + f])));
        const float s1 = sinpif(om_pi * fmaf(p_s[2 * f1], x, fmaf(p_s[2 * f1 + 1], y, p_s[kOffB1 + f1])));
        acc0 = fmaf(p_s[kOffW2 + f], s0, acc0);
        acc1 = fmaf(p_s[kOffW2 + f1], s1, acc1);
    }
    float acc = acc0 + acc1;
#pragma unroll
    for (int o = 1; o < kFwdLanes; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!valid || part != 0) return;
    const float z = acc + p_s[kOffB2];
    a.z[node] = z;
    const bool inside = a.mask ? a.mask[node] != 0 : true;
    a.sos[node] = inside ? fmaf(p_s[kOffScale], z, p_s[kOffOffset]) : a.v_bg;
}

// CTA c: nodes [c * kChunk, +kChunk); thread f accumulates, over those nodes with
// g = dL/dv (0 outside the mask) and dz = scale g,
//   dW1_f = sum dz w2_f omega0 cos(a_f) x,  db1_f = sum dz w2_f omega0 cos(a_f),  dw2_f = sum dz sin(a_f);
// threads 0..2 also form sum dz (b2), sum g z (scale) and sum g (offset).
__global__ void __launch_bounds__(kF) siren_bwd_kernel(const SirenArgs a) {
    __shared__ float gx_s[kChunk], gy_s[kChunk], dz_s[kChunk], gz_s[kChunk], g_s[kChunk];
    const int GG = a.G * a.G;
    const int n0 = blockIdx.x * kChunk, nn = min(kChunk, GG - n0);
    const float scale = a.params[kOffScale];
    for (int e = threadIdx.x; e < kChunk; e += blockDim.x) {
        const int node = n0 + e;
        float g = 0.f, zz = 0.f;
        if (e < nn) {
            const bool inside = a.mask ? a.mask[node] != 0 : true;
            g = inside ? a.dL_dsos[node] : 0.f;
            zz = a.z[node];
        }
        gx_s[e] = coord(node % a.G, a.G);
        gy_s[e] = coord(node / a.G, a.G);
        g_s[e] = g;
        dz_s[e] = g * scale;
        gz_s[e] = g * zz;
    }
    __syncthreads();
    const int f = threadIdx.x;
    const float w1x = a.params[2 * f], w1y = a.params[2 * f + 1], b1 = a.params[kOffB1 + f];
    const float w2 = a.params[kOffW2 + f], om = a.omega0, om_pi = om * 0.3183098861837907f;
    float sx = 0.f, sy = 0.f, sb = 0.f, sw = 0.f;
    for (int e = 0; e < nn; ++e) {
        const float dz = dz_s[e];
        float sn, cs;
        sincospif(om_pi * fmaf(w1x, gx_s[e], fmaf(w1y, gy_s[e], b1)), &sn, &cs);
        const float t = dz * cs;
        sx = fmaf(t, gx_s[e], sx);
        sy = fmaf(t, gy_s[e], sy);
        sb += t;
        sw = fmaf(dz, sn, sw);
    }
    float* row = a.part + (size_t)blockIdx.x * kStride;
    const float k = w2 * om;
    row[2 * f] = k * sx;
    row[2 * f + 1] = k * sy;
    row[kOffB1 + f] = k * sb;
    row[kOffW2 + f] = sw;
    if (f < 3) {
        float s = 0.f;
        const float* src = f == 0 ? dz_s : f == 1 ? gz_s : g_s;
        for (int e = 0; e < nn; ++e) s += src[e];
        row[kOffB2 + f] = s;      // b2, scale, offset
    }
}

// Parameters e = 32 b + lane of block b: warp w adds the partial rows of its
// chunk [chunks w / 8, chunks (w + 1) / 8) in order, warp 0 the eight chunk
// sums in order (fixed order, eight times the loads in flight).
__global__ void __launch_bounds__(256) siren_reduce_kernel(const float* part, int chunks, float* out,
                                                           int accumulate) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    const int c0 = chunks * w / 8, c1 = chunks * (w + 1) / 8;
    float s = 0.f;
    if (e < kNP) {
#pragma unroll 8
        for (int c = c0; c < c1; ++c) s += part[(size_t)c * kStride + e];     // in order; loads run ahead
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < kNP) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        out[e] = accumulate ? out[e] + t : t;
    }
}

struct SirenPlan {
    int chunks;
    size_t off_z, off_part, total;
};

SirenPlan siren_plan(const pact_geometry* g) {
    SirenPlan p;
    const int GG = g->sos_g * g->sos_g;
    p.chunks = (GG + kChunk - 1) / kChunk;
    p.off_z = 0;
    p.off_part = align_up((size_t)GG * sizeof(float), 256);
    p.total = p.off_part + align_up((size_t)p.chunks * kStride * sizeof(float), 256);
    return p;
}

pact_status siren_args(const pact_geometry* g, const float* params, const unsigned char* mask, float omega0,
                       void* ws, size_t ws_bytes, SirenArgs& a) {
    PACT_TRY(check_geometry(g));
    if (!params || !ws) return fail(PACT_ERR_INVALID_ARG, "siren: params and workspace must not be NULL");
    if (!(omega0 > 0.f) || !isfinite(omega0)) return fail(PACT_ERR_INVALID_ARG, "siren: omega0 must be finite and > 0");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const SirenPlan pl = siren_plan(g);
    if (ws_bytes < pl.total) return fail(PACT_ERR_INVALID_ARG, "siren: workspace too small: %zu < %zu", ws_bytes, pl.total);
    char* base = static_cast<char*>(ws);
    a.G = g->sos_g;
    a.omega0 = omega0;
    a.v_bg = g->v_bg;
    a.params = params;
    a.mask = mask;
    a.z = reinterpret_cast<float*>(base + pl.off_z);
    a.part = reinterpret_cast<float*>(base + pl.off_part);
    a.sos = nullptr;
    a.dL_dsos = nullptr;
    a.dL_dparams = nullptr;
    a.accumulate = 0;
    return PACT_OK;
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" int pact_siren_param_count(void) { return kNP; }

extern "C" size_t pact_siren_workspace_size(const pact_geometry* g) {
    if (check_geometry(g) != PACT_OK) return 0;
    return siren_plan(g).total;
}

extern "C" pact_status pact_siren_forward(const pact_geometry* g, const float* params, const unsigned char* mask,
                                          float omega0, float* sos, void* ws, size_t ws_bytes, void* stream) {
    SirenArgs a;
    PACT_TRY(siren_args(g, params, mask, omega0, ws, ws_bytes, a));
    if (!sos) return fail(PACT_ERR_INVALID_ARG, "siren_forward: sos is NULL");
    a.sos = sos;
    const int GG = g->sos_g * g->sos_g;
    siren_fwd_kernel<<<(GG * kFwdLanes + 255) / 256, 256, 0, as_stream(stream)>>>(a);
    return check_launch("siren forward kernel");
}

extern "C" pact_status pact_siren_backward(const pact_geometry* g, const float* params, const unsigned char* mask,
                                           float omega0, const float* dL_dsos, float* dL_dparams, int accumulate,
                                           void* ws, size_t ws_bytes, void* stream) {
    SirenArgs a;
    PACT_TRY(siren_args(g, params, mask, omega0, ws, ws_bytes, a));
    if (!dL_dsos || !dL_dparams) return fail(PACT_ERR_INVALID_ARG, "siren_backward: dL_dsos and dL_dparams must not be NULL");
    a.dL_dsos = dL_dsos;
    a.dL_dparams = dL_dparams;
    a.accumulate = accumulate;
    const SirenPlan pl = siren_plan(g);
    cudaStream_t st = as_stream(stream);
    siren_bwd_kernel<<<pl.chunks, kF, 0, st>>>(a);
    PACT_TRY(check_launch("siren backward kernel"));
    siren_reduce_kernel<<<(kNP + 31) / 32, 256, 0, st>>>(a.part, pl.chunks, dL_dparams, accumulate);
    return check_launch("siren reduction");
}
