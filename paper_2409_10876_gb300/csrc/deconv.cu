// Eq. 4-7 on the GPU: transfer-function synthesis (pact_psf_synth and its
// adjoint, pact_forward_model) and the fused multi-channel deconvolution +
// loss + adjoint pass (pact_mc_deconv_loss).
//
// Algebra of the fused pass (per patch i and half-spectrum bin k; M channels).
// With E_j = exp(j|k|d_j), a = exp(-j|k|W(ang k)), b = exp(+j|k|W(ang k + pi)):
//     H_j = (E_j a + conj(E_j) b) / 2                                   (Eq. 4)
// so every channel sum of Eq. 6 reduces to sums over the data alone:
//     S1 = sum_j cos(|k|d_j) Y_j,  S2 = sum_j sin(|k|d_j) Y_j,  C2 = sum_j E_j^2
//     A  = sum_j conj(H_j) Y_j = (conj(a) (S1 - jS2) + conj(b) (S1 + jS2)) / 2
//     B  = sum_j |H_j|^2       = (M + Re(a conj(b) C2)) / 2
//     X  = A / (B + eps)                                                  (Eq. 6)
// The residual R_j = Y_j - H_j X = Y_j - cos(|k|d_j) p - sin(|k|d_j) q with
// p = (a + b) X / 2, q = j (a - b) X / 2 is formed explicitly in a second
// pass over the shared-memory copy of Y (no E - |A|^2/B cancellation), giving
// the loss term w_k sum_j |R_j|^2 (Eq. 7, w_k = c_k |k|_mm).
// Adjoint: dL/dconj(H_j) = -(w_k conj(X)/D) ((B + 2 eps) R_j - eps X H_j),
// D = B + eps, and with T1 = sum_j cos(|k|d_j) conj(R_j),
// T2 = sum_j sin(|k|d_j) conj(R_j):
//     dL/dW(ang k)      =  |k| Im(conj(K) ((B+2eps) a (T1 + jT2) - eps conj(X) (M + a conj(b) C2)/2))
//     dL/dW(ang k + pi) = -|k| Im(conj(K) ((B+2eps) b (T1 - jT2) - eps conj(X) (M + conj(a) b conj(C2))/2))
// with K = -w_k conj(X)/D; these are scattered to the two transducers each
// lookup interpolates (shared-memory accumulation per CTA, then a
// deterministic reduction over the CTAs of a patch).
#include <algorithm>
#include <mutex>

#include "pact_internal.cuh"

namespace pact {
namespace {

constexpr int kTPB = 256;
constexpr float kTwoPi = 6.283185307179586f;

struct Tf {  // per (patch, bin) quantities of Eq. 4
    float fm;          // |f| [cycles/m]; |k| = 2 pi fm
    float2 a, b;       // exp(-j|k|W1), exp(+j|k|W2)
    int n1a, n1b;
    float fa, fb;
    float W1, W2;
};

__device__ __forceinline__ Tf make_tf(const Geo& g, int P, float inv_pdx, float n_over_2pi,
                                      float2 c, const float* w_row, int k, int& u, int& v) {
    Tf t;
    const float2 f = bin_freq(k, P, inv_pdx, u, v);
    t.fm = sqrtf(f.x * f.x + f.y * f.y);
    float ex = 1.f, ey = 0.f;
    if (t.fm > 0.f) {
        ex = f.x / t.fm;
        ey = f.y / t.fm;
    }
    const Hits h = ring_hits(c.x, c.y, ex, ey, g, n_over_2pi);
    t.n1a = h.n1a;
    t.n1b = h.n1b;
    t.fa = h.fa;
    t.fb = h.fb;
    const int n2a = t.n1a + 1 == g.n_t ? 0 : t.n1a + 1;
    const int n2b = t.n1b + 1 == g.n_t ? 0 : t.n1b + 1;
    t.W1 = fmaf(t.fa, w_row[n2a] - w_row[t.n1a], w_row[t.n1a]);
    t.W2 = fmaf(t.fb, w_row[n2b] - w_row[t.n1b], w_row[t.n1b]);
    t.a = cis_pi(-2.f * t.fm * t.W1);
    t.b = cis_pi(2.f * t.fm * t.W2);
    return t;
}

struct McdArgs {
    Geo g;
    int N, P, F, M;
    const int2* centres;
    const float* w;
    const float2* Y;
    float eps;
    Delays dl;
    float2* Xhat;
    int want_grad;
    int fp64;
    float* part_loss;      // [N][KT]
    float* part_dw;        // [N][KT][n_t]
    const float2* lut;     // [N][F] ring coordinates (t_a, t_b)
    const float2* etab;    // [M][F] exp(j|k|d_j)
    const float4* btab;    // [F] (|k|/2pi, c_k |k|_mm, Re C2, Im C2)
    const double2* c2d;    // [F] C2 in FP64 (eps < 1e-6 only)
    int KT;                // 256-bin tiles
};

// Ring coordinate t = alpha N_t / (2 pi) in [0, N_t) of the point where the ray
// from c in direction (dx, dy) meets the ring (same arithmetic as ring_hit).
__device__ __forceinline__ float ring_coord(float cx, float cy, float dx, float dy, const Geo& g,
                                            float n_over_2pi) {
    const float ce = cx * dx + cy * dy;
    const float disc = fmaxf(ce * ce - (cx * cx + cy * cy) + g.R * g.R, 0.f);
    const float s = sqrtf(disc) - ce;
    float t = (atan2f(fmaf(s, dy, cy), fmaf(s, dx, cx)) - g.phase) * n_over_2pi;
    t -= floorf(t / (float)g.n_t) * (float)g.n_t;
    return t;
}

// Per-call tables of the fused pass, one launch:
//  * blockIdx.y < N: geometry-only part of Eq. 4 for patch i = blockIdx.y, the
//    ring coordinates of the directions ang k and ang k + pi,
//    lut[i][k] = (t_a, t_b);
//  * blockIdx.y == N: per-bin tables etab[j][k] = exp(j|k|d_j) and
//    btab[k] = (|k|/2pi, c_k |k|_mm, Re C2, Im C2) with C2 = sum_j exp(2j|k|d_j).
__global__ void mcd_tables_kernel(Geo g, int N, int P, int F, int M, Delays dl, const int2* centres, float2* lut,
                                  float2* etab, float4* btab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F) return;
    int u, v;
    const float2 f = bin_freq(k, P, 1.f / (P * g.dx), u, v);
    const float fm = sqrtf(f.x * f.x + f.y * f.y);
    if ((int)blockIdx.y < N) {
        const float ex = fm > 0.f ? f.x / fm : 1.f, ey = fm > 0.f ? f.y / fm : 0.f;
        const int2 cc = centres[blockIdx.y];
        const float2 c = pixel_xy(g, cc.x, cc.y);
        const float nop = g.n_t / kTwoPi;
        lut[(size_t)blockIdx.y * F + k] =
            make_float2(ring_coord(c.x, c.y, ex, ey, g, nop), ring_coord(c.x, c.y, -ex, -ey, g, nop));
        return;
    }
    float c2x = 0.f, c2y = 0.f;
    for (int j = 0; j < M; ++j) {
        const float2 e = cis_pi(2.f * fm * dl.d[j]);
        etab[(size_t)j * F + k] = e;
        c2x = fmaf(e.x, e.x, fmaf(-e.y, e.y, c2x));
        c2y = fmaf(2.f * e.x, e.y, c2y);
    }
    const float om = ((v == 0 || v == P / 2) ? 1.f : 2.f) * kTwoPi * fm * 1e-3f;
    btab[k] = make_float4(fm, om, c2x, c2y);
}

// FP64 C2(k) = sum_j exp(2j|k|d_j) for the eps < 1e-6 path.
__global__ void mcd_c2d_kernel(int P, int F, double dx, Delays dl, double2* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F) return;
    const int half = P / 2 + 1;
    const int u = k / half, v = k - (k / half) * half;
    const int us = u < P / 2 ? u : u - P;
    const double fx = v / (P * dx), fy = us / (P * dx);
    const double fm = sqrt(fx * fx + fy * fy);
    double re = 0.0, im = 0.0;
    for (int j = 0; j < dl.m; ++j) {
        double sn, cs;
        sincospi(4.0 * fm * (double)dl.d[j], &sn, &cs);
        re += cs;
        im += sn;
    }
    out[k] = make_double2(re, im);
}

// Sum over the two threads of a bin (lanes b and b + 16).
__device__ __forceinline__ float pair_sum(float x) { return x + __shfl_xor_sync(0xffffffffu, x, 16); }

// CTA (kt, i): bins kt*256 .. kt*256+255 of patch i, 512 threads.  Two
// threads share a bin (lanes b and b+16 of a warp; warp w owns bins
// 16w .. 16w+15): half h owns channels j = h, h+2, ..., loads Y_ij(k) and
// exp(j|k|d_j) for them straight into registers (Y streamed once from HBM,
// the exp table from L2) and completes every channel sum with one shuffle.
// Half 0 evaluates the lookup of w at ang k, half 1 at ang k + pi.  With
// S1 = sum cos(|k|d_j) Y_j and S2 = sum sin(|k|d_j) Y_j the residual sums of
// the adjoint follow in closed form, T1 = conj(S1) - conj(p) Scc - conj(q) Scs,
// T2 = conj(S2) - conj(p) Scs - conj(q) Sss; only sum |R_j|^2 needs the explicit
// second pass over the registers.  CPH channels per half; EXACT: M == 2 CPH.
template <int CPH, bool EXACT>
__global__ void __launch_bounds__(512, 1) mcd_kernel(const McdArgs a) {
    extern __shared__ float dw_s[];                          // [n_t]
    __shared__ float lsum_s;
    const int n_t = a.g.n_t, M = EXACT ? 2 * CPH : a.M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hf = lane >> 4;
    const int kt = blockIdx.x, i = blockIdx.y;
    const int k = kt * 256 + warp * 16 + (lane & 15);
    const bool valid = k < a.F;
    for (int n = tid; n < n_t; n += 512) dw_s[n] = 0.f;
    if (tid == 0) lsum_s = 0.f;

    float2 y[CPH], E[CPH];
    const float2* yp = a.Y + ((size_t)i * M + hf) * a.F + k;
    const float2* ep = a.etab + (size_t)hf * a.F + k;
    float4 bt = make_float4(0.f, 0.f, 0.f, 0.f);
    float tr = 0.f;
    if (valid) {
#pragma unroll
        for (int m = 0; m < CPH; ++m) {
            if (EXACT || 2 * m + hf < M) {
                y[m] = __ldcs(yp + (size_t)(2 * m) * a.F);
                E[m] = __ldg(ep + (size_t)(2 * m) * a.F);
            } else {
                y[m] = make_float2(0.f, 0.f);
                E[m] = make_float2(0.f, 0.f);
            }
        }
        bt = __ldg(a.btab + k);
        tr = __ldg(reinterpret_cast<const float*>(a.lut) + 2 * ((size_t)i * a.F + k) + hf);
    }
    const float fm = bt.x, om = bt.y;
    const float2 C2 = make_float2(bt.z, bt.w);
    const float Mf = (float)M;
    const float eps = a.eps;

    // w at this thread's direction (Eq. 4): linear in ring angle between two transducers
    const float* wr = a.w + (size_t)i * n_t;
    const float fl = floorf(tr);
    const float fr = tr - fl;
    int n1 = (int)fl;
    n1 = n1 >= n_t ? n1 - n_t : n1;
    const int n2 = n1 + 1 == n_t ? 0 : n1 + 1;
    const float w1 = __ldg(wr + n1), w2 = __ldg(wr + n2);
    const float Wd = fmaf(fr, w2 - w1, w1);
    const float dsgn = hf ? -1.f : 1.f;
    const float2 ph = cis_pi(-dsgn * 2.f * fm * Wd);   // half 0: exp(-j|k|W1), half 1: exp(+j|k|W2)
    const float2 oth = make_float2(__shfl_xor_sync(0xffffffffu, ph.x, 16), __shfl_xor_sync(0xffffffffu, ph.y, 16));
    const float Wo = __shfl_xor_sync(0xffffffffu, Wd, 16);
    const float2 al = hf ? oth : ph, be = hf ? ph : oth;
    const float W1 = hf ? Wo : Wd, W2 = hf ? Wd : Wo;

    // pass 1 (own channels), completed across the pair
    float s1x = 0.f, s1y = 0.f, s2x = 0.f, s2y = 0.f;
#pragma unroll
    for (int m = 0; m < CPH; ++m) {
        s1x = fmaf(E[m].x, y[m].x, s1x);
        s1y = fmaf(E[m].x, y[m].y, s1y);
        s2x = fmaf(E[m].y, y[m].x, s2x);
        s2y = fmaf(E[m].y, y[m].y, s2y);
    }
    const float2 S1 = make_float2(pair_sum(s1x), pair_sum(s1y));
    const float2 S2 = make_float2(pair_sum(s2x), pair_sum(s2y));
    const float2 U = make_float2(S1.x + S2.y, S1.y - S2.x);   // sum conj(E_j) Y_j
    const float2 V = make_float2(S1.x - S2.y, S1.y + S2.x);   // sum E_j Y_j
    const float2 ca = cmulc(al, U), cb = cmulc(be, V);
    const float2 A = make_float2(0.5f * (ca.x + cb.x), 0.5f * (ca.y + cb.y));
    const float2 ab = cmulc(be, al);                           // a conj(b)
    float B, D;
    float2 X;
    if (a.fp64) {
        double sn, cs;
        sincospi(-2.0 * (double)fm * ((double)W1 + (double)W2), &sn, &cs);
        const double2 C2d = valid ? a.c2d[k] : make_double2(0.0, 0.0);
        const double Bd = 0.5 * ((double)M + (cs * C2d.x - sn * C2d.y));
        const double Dd = Bd + (double)eps;
        B = (float)Bd;
        D = (float)Dd;
        X = Dd != 0.0 ? make_float2((float)(A.x / Dd), (float)(A.y / Dd)) : make_float2(0.f, 0.f);
    } else {
        B = 0.5f * (Mf + (ab.x * C2.x - ab.y * C2.y));
        D = B + eps;
        const float iD = D != 0.f ? __frcp_rn(D) : 0.f;
        X = make_float2(A.x * iD, A.y * iD);
    }

    // pass 2: explicit residual energy of the own channels
    const float2 pp = make_float2(0.5f * (al.x + be.x), 0.5f * (al.y + be.y));
    const float2 qm = make_float2(0.5f * (al.x - be.x), 0.5f * (al.y - be.y));
    const float2 p = cmul(pp, X);
    const float2 q0v = cmul(qm, X);
    const float2 qv = make_float2(-q0v.y, q0v.x);
    float e2 = 0.f;
#pragma unroll
    for (int m = 0; m < CPH; ++m) {
        const float rx = y[m].x - fmaf(E[m].x, p.x, E[m].y * qv.x);
        const float ry = y[m].y - fmaf(E[m].x, p.y, E[m].y * qv.y);
        e2 = fmaf(rx, rx, fmaf(ry, ry, e2));
    }
    e2 = pair_sum(e2);
    float contrib = 0.f;
    __syncthreads();                                    // dw_s cleared
    if (valid) {
        if (hf == 0) {
            contrib = om * e2;
            if (a.Xhat) a.Xhat[(size_t)i * a.F + k] = X;
        }
        if (a.want_grad && fm > 0.f && D != 0.f) {
            const float Scc = 0.5f * (Mf + C2.x), Sss = 0.5f * (Mf - C2.x), Scs = 0.5f * C2.y;
            const float iD = __frcp_rn(D);
            const float kmag = kTwoPi * fm;
            const float2 Kc = make_float2(-om * X.x * iD, -om * X.y * iD);   // conj(K)
            const float b2 = B + 2.f * eps;
            const float2 abC2 = cmul(ab, C2);
            const float2 xc = make_float2(X.x, -X.y);
            // T1 = sum cos conj(R), T2 = sum sin conj(R)
            const float2 T1 = make_float2(S1.x - p.x * Scc - qv.x * Scs, -S1.y + p.y * Scc + qv.y * Scs);
            const float2 T2 = make_float2(S2.x - p.x * Scs - qv.x * Sss, -S2.y + p.y * Scs + qv.y * Sss);
            float gW;
            if (hf == 0) {
                const float2 hp = make_float2(0.5f * (Mf + abC2.x), 0.5f * abC2.y);
                const float2 tp = make_float2(T1.x - T2.y, T1.y + T2.x);
                const float2 ap = cmul(al, tp), xhp = cmul(xc, hp);
                const float2 SP = make_float2(b2 * ap.x - eps * xhp.x, b2 * ap.y - eps * xhp.y);
                gW = kmag * (Kc.x * SP.y + Kc.y * SP.x);
            } else {
                const float2 hq = make_float2(0.5f * (Mf + abC2.x), -0.5f * abC2.y);
                const float2 tq = make_float2(T1.x + T2.y, T1.y - T2.x);
                const float2 bq = cmul(be, tq), xhq = cmul(xc, hq);
                const float2 SQ = make_float2(b2 * bq.x - eps * xhq.x, b2 * bq.y - eps * xhq.y);
                gW = -kmag * (Kc.x * SQ.y + Kc.y * SQ.x);
            }
            atomicAdd(dw_s + n1, (1.f - fr) * gW);
            atomicAdd(dw_s + n2, fr * gW);
        }
    }
    contrib = warp_sum(contrib);
    if (lane == 0) atomicAdd(&lsum_s, contrib);
    __syncthreads();
    if (a.want_grad) {
        float* dst = a.part_dw + ((size_t)i * a.KT + kt) * n_t;
        for (int n = tid; n < n_t; n += 512) dst[n] = dw_s[n];
    }
    if (tid == 0) a.part_loss[(size_t)i * a.KT + kt] = lsum_s;
}

struct FinArgs {
    int N, S, n_t;
    const float* part_loss;
    const float* part_dw;
    float* loss;
    float* loss_pp;
    float* dL_dw;
    const float* scale;   // device scalar or NULL
    int accumulate;
    int want_grad;
};

__global__ void __launch_bounds__(kTPB) mcd_finalize_kernel(const FinArgs a) {
    __shared__ float red[kTPB / 32];
    const int i = blockIdx.x;
    const float sc = a.scale ? *a.scale : 1.f;
    if (a.want_grad && a.dL_dw) {
        for (int n = threadIdx.x; n < a.n_t; n += kTPB) {
            float acc = 0.f;
            for (int s = 0; s < a.S; ++s) acc += a.part_dw[((size_t)i * a.S + s) * a.n_t + n];
            acc *= sc;
            float* o = a.dL_dw + (size_t)i * a.n_t + n;
            *o = a.accumulate ? *o + acc : acc;
        }
    }
    if (a.loss_pp && threadIdx.x == 0) {
        float acc = 0.f;
        for (int s = 0; s < a.S; ++s) acc += a.part_loss[(size_t)i * a.S + s];
        a.loss_pp[i] = acc;
    }
    if (i == 0 && a.loss) {
        float acc = 0.f;
        const int tot = a.N * a.S;
        for (int q = threadIdx.x; q < tot; q += kTPB) acc += a.part_loss[q];
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) a.loss[0] = acc;
    }
}

struct Plan {
    int KT;
    size_t off_dw, off_lut, off_etab, off_btab, off_c2d, total;
};

Plan make_plan(const pact_geometry* g, const pact_patches* pt, int m) {
    Plan p;
    const int F = pt->p * (pt->p / 2 + 1);
    p.KT = (F + 255) / 256;
    size_t o = align_up((size_t)pt->n * p.KT * sizeof(float), 256);
    p.off_dw = o;
    o += align_up((size_t)pt->n * p.KT * g->n_t * sizeof(float), 256);
    p.off_lut = o;
    o += align_up((size_t)pt->n * F * sizeof(float2), 256);
    p.off_etab = o;
    o += align_up((size_t)m * F * sizeof(float2), 256);
    p.off_btab = o;
    o += align_up((size_t)F * sizeof(float4), 256);
    p.off_c2d = o;
    o += align_up((size_t)F * sizeof(double2), 256);
    p.total = o;
    return p;
}

pact_status check_delays(const float* d, int m) {
    if (!d) return fail(PACT_ERR_INVALID_ARG, "delay list is NULL");
    if (m < 1) return fail(PACT_ERR_INVALID_ARG, "channel count must be >= 1 (got %d)", m);
    if (m > PACT_MAX_CHANNELS)
        return fail(PACT_ERR_SHAPE, "channel count must be <= %d (got %d)", PACT_MAX_CHANNELS, m);
    for (int j = 0; j < m; ++j)
        if (!isfinite(d[j])) return fail(PACT_ERR_INVALID_ARG, "delay %d is not finite", j);
    return PACT_OK;
}

template <int CPH, bool EXACT>
pact_status launch_mcd(const McdArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)a.g.n_t * sizeof(float);
    PACT_TRY(ensure_smem((const void*)mcd_kernel<CPH, EXACT>, smem, "mc_deconv_loss: shared memory attribute"));
    dim3 grid(a.KT, a.N);
    mcd_kernel<CPH, EXACT><<<grid, 512, smem, st>>>(a);
    return check_launch("mc_deconv_loss kernel");
}

pact_status run_mcd(const pact_geometry* g, const pact_patches* pt, const float* w, const float* Y,
                    const float* d, int m, float eps, float* loss, float* loss_pp, float* Xhat,
                    float* dL_dw, const float* scale, int accumulate, void* ws, size_t ws_bytes,
                    void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    PACT_TRY(check_delays(d, m));
    if (!w || !Y) return fail(PACT_ERR_INVALID_ARG, "mc_deconv_loss: w and Y must not be NULL");
    if (!(eps >= 0.f) || !isfinite(eps)) return fail(PACT_ERR_INVALID_ARG, "eps must be finite and >= 0");
    if (!ws) return fail(PACT_ERR_INVALID_ARG, "mc_deconv_loss: workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(Y) % 16) return fail(PACT_ERR_INVALID_ARG, "Y must be 16-byte aligned");
    const Plan pl = make_plan(g, pt, m);
    if ((size_t)g->n_t * sizeof(float) > 200 * 1024) return fail(PACT_ERR_SHAPE, "mc_deconv_loss: n_t too large");
    if (ws_bytes < pl.total)
        return fail(PACT_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, pl.total);
    cudaStream_t st = as_stream(stream);
    char* base = static_cast<char*>(ws);
    McdArgs a;
    a.g = make_geo(g);
    a.N = pt->n;
    a.P = pt->p;
    a.F = pt->p * (pt->p / 2 + 1);
    a.M = m;
    a.centres = reinterpret_cast<const int2*>(pt->centres);
    a.w = w;
    a.Y = reinterpret_cast<const float2*>(Y);
    a.eps = eps;
    a.dl = make_delays(d, m);
    a.Xhat = reinterpret_cast<float2*>(Xhat);
    a.want_grad = dL_dw != nullptr;
    a.fp64 = eps < 1e-6f;
    a.part_loss = reinterpret_cast<float*>(base);
    a.part_dw = reinterpret_cast<float*>(base + pl.off_dw);
    a.lut = reinterpret_cast<const float2*>(base + pl.off_lut);
    a.etab = reinterpret_cast<const float2*>(base + pl.off_etab);
    a.btab = reinterpret_cast<const float4*>(base + pl.off_btab);
    a.c2d = reinterpret_cast<const double2*>(base + pl.off_c2d);
    a.KT = pl.KT;
    dim3 tg((a.F + 255) / 256, a.N + 1);
    mcd_tables_kernel<<<tg, 256, 0, st>>>(a.g, a.N, a.P, a.F, m, a.dl, a.centres,
                                         reinterpret_cast<float2*>(base + pl.off_lut),
                                         reinterpret_cast<float2*>(base + pl.off_etab),
                                         reinterpret_cast<float4*>(base + pl.off_btab));
    PACT_TRY(check_launch("mc_deconv_loss: tables"));
    if (a.fp64) {
        mcd_c2d_kernel<<<(a.F + 255) / 256, 256, 0, st>>>(a.P, a.F, (double)g->dx, a.dl,
                                                          reinterpret_cast<double2*>(base + pl.off_c2d));
        PACT_TRY(check_launch("mc_deconv_loss: FP64 table"));
    }
    pact_status s;
    if (m == 8) s = launch_mcd<4, true>(a, st);
    else if (m == 16) s = launch_mcd<8, true>(a, st);
    else if (m == 32) s = launch_mcd<16, true>(a, st);
    else if (m == 64) s = launch_mcd<32, true>(a, st);
    else if (m < 8) s = launch_mcd<4, false>(a, st);
    else if (m < 16) s = launch_mcd<8, false>(a, st);
    else if (m < 32) s = launch_mcd<16, false>(a, st);
    else s = launch_mcd<32, false>(a, st);
    if (s != PACT_OK) return s;
    FinArgs f;
    f.N = a.N;
    f.S = a.KT;
    f.n_t = g->n_t;
    f.part_loss = a.part_loss;
    f.part_dw = a.part_dw;
    f.loss = loss;
    f.loss_pp = loss_pp;
    f.dL_dw = dL_dw;
    f.scale = scale;
    f.accumulate = accumulate;
    f.want_grad = a.want_grad;
    mcd_finalize_kernel<<<a.N, kTPB, 0, st>>>(f);
    return check_launch("mc_deconv_loss finalize");
}

// ---------------------------------------------------------------- psf synthesis

struct PsfArgs {
    Geo g;
    int N, P, F, M;
    const int2* centres;
    const float* w;
    Delays dl;
    int mode;            // 0: H, 1: Y (+)= H X, 2: adjoint
    const float2* in;    // X (mode 1) or dL_dH (mode 2)
    float2* out;         // H or Y
    float* dL_dw;        // mode 2
    int accumulate;
};

__global__ void __launch_bounds__(kTPB) psf_kernel(const PsfArgs a) {
    const int i = blockIdx.y;
    const int k = blockIdx.x * kTPB + threadIdx.x;
    if (k >= a.F) return;
    const int n_t = a.g.n_t;
    const int2 cc = a.centres[i];
    const float2 c = pixel_xy(a.g, cc.x, cc.y);
    int u, v;
    const Tf t = make_tf(a.g, a.P, 1.f / (a.P * a.g.dx), n_t / kTwoPi, c, a.w + (size_t)i * n_t, k, u, v);
    const float two_fm = 2.f * t.fm;
    if (a.mode == 2) {
        float g1 = 0.f, g2 = 0.f;
        for (int j = 0; j < a.M; ++j) {
            const float2 e = cis_pi(two_fm * a.dl.d[j]);
            const float2 P_ = cmul(e, t.a);
            const float2 Q_ = cmulc(e, t.b);
            const float2 gj = a.in[((size_t)i * a.M + j) * a.F + k];
            const float2 gp = cmulc(gj, P_), gq = cmulc(gj, Q_);
            g1 += gp.y;
            g2 += gq.y;
        }
        const float kmag = kTwoPi * t.fm;
        g1 *= 0.5f * kmag;
        g2 *= -0.5f * kmag;
        const int n2a = t.n1a + 1 == n_t ? 0 : t.n1a + 1;
        const int n2b = t.n1b + 1 == n_t ? 0 : t.n1b + 1;
        float* row = a.dL_dw + (size_t)i * n_t;
        atomicAdd(row + t.n1a, (1.f - t.fa) * g1);
        atomicAdd(row + n2a, t.fa * g1);
        atomicAdd(row + t.n1b, (1.f - t.fb) * g2);
        atomicAdd(row + n2b, t.fb * g2);
        return;
    }
    float2 x = make_float2(0.f, 0.f);
    if (a.mode == 1) x = a.in[(size_t)i * a.F + k];
    for (int j = 0; j < a.M; ++j) {
        const float2 e = cis_pi(two_fm * a.dl.d[j]);
        const float2 P_ = cmul(e, t.a);
        const float2 Q_ = cmulc(e, t.b);
        const float2 H = make_float2(0.5f * (P_.x + Q_.x), 0.5f * (P_.y + Q_.y));
        float2* o = a.out + ((size_t)i * a.M + j) * a.F + k;
        if (a.mode == 0) {
            *o = H;
        } else {
            float2 val = cmul(H, x);
            if (a.accumulate) {
                const float2 old = *o;
                val.x += old.x;
                val.y += old.y;
            }
            *o = val;
        }
    }
}

pact_status run_psf(const pact_geometry* g, const pact_patches* pt, const float* w, const float* d,
                    int m, int mode, const float* in, float* out, float* dL_dw, int accumulate,
                    void* stream) {
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    PACT_TRY(check_delays(d, m));
    if (!w) return fail(PACT_ERR_INVALID_ARG, "w is NULL");
    if (mode == 0 && !out) return fail(PACT_ERR_INVALID_ARG, "H is NULL");
    if (mode == 1 && (!in || !out)) return fail(PACT_ERR_INVALID_ARG, "X and Y must not be NULL");
    if (mode == 2 && (!in || !dL_dw)) return fail(PACT_ERR_INVALID_ARG, "dL_dH and dL_dw must not be NULL");
    cudaStream_t st = as_stream(stream);
    PsfArgs a;
    a.g = make_geo(g);
    a.N = pt->n;
    a.P = pt->p;
    a.F = pt->p * (pt->p / 2 + 1);
    a.M = m;
    a.centres = reinterpret_cast<const int2*>(pt->centres);
    a.w = w;
    a.dl = make_delays(d, m);
    a.mode = mode;
    a.in = reinterpret_cast<const float2*>(in);
    a.out = reinterpret_cast<float2*>(out);
    a.dL_dw = dL_dw;
    a.accumulate = accumulate;
    if (mode == 2 && !accumulate) {
        if (cudaMemsetAsync(dL_dw, 0, (size_t)pt->n * g->n_t * sizeof(float), st) != cudaSuccess)
            return check_launch("psf_synth_adj: memset");
    }
    dim3 grid((a.F + kTPB - 1) / kTPB, a.N);
    psf_kernel<<<grid, kTPB, 0, st>>>(a);
    return check_launch("psf kernel");
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" size_t pact_mc_deconv_loss_workspace_size(const pact_geometry* g, const pact_patches* pt, int m) {
    if (check_geometry(g) != PACT_OK || check_patches(pt) != PACT_OK) return 0;
    return make_plan(g, pt, m).total;
}

extern "C" pact_status pact_mc_deconv_loss(const pact_geometry* g, const pact_patches* pt, const float* w,
                                           const float* Y, const float* d, int m, float eps, float* loss,
                                           float* loss_pp, float* Xhat, float* dL_dw, void* ws,
                                           size_t ws_bytes, void* stream) {
    if (!loss) return fail(PACT_ERR_INVALID_ARG, "mc_deconv_loss: loss is NULL");
    return run_mcd(g, pt, w, Y, d, m, eps, loss, loss_pp, Xhat, dL_dw, nullptr, 0, ws, ws_bytes, stream);
}

extern "C" pact_status pact_mc_deconv_loss_adj(const pact_geometry* g, const pact_patches* pt, const float* w,
                                               const float* Y, const float* d, int m, float eps,
                                               const float* dL_dloss, float* dL_dw, int accumulate, void* ws,
                                               size_t ws_bytes, void* stream) {
    if (!dL_dw) return fail(PACT_ERR_INVALID_ARG, "mc_deconv_loss_adj: dL_dw is NULL");
    return run_mcd(g, pt, w, Y, d, m, eps, nullptr, nullptr, nullptr, dL_dw, dL_dloss, accumulate, ws,
                   ws_bytes, stream);
}

extern "C" pact_status pact_psf_synth(const pact_geometry* g, const pact_patches* pt, const float* w,
                                      const float* d, int m, float* H, void* stream) {
    return run_psf(g, pt, w, d, m, 0, nullptr, H, nullptr, 0, stream);
}

extern "C" pact_status pact_forward_model(const pact_geometry* g, const pact_patches* pt, const float* w,
                                          const float* d, int m, const float* X, float* Y, int accumulate,
                                          void* stream) {
    return run_psf(g, pt, w, d, m, 1, X, Y, nullptr, accumulate, stream);
}

extern "C" pact_status pact_psf_synth_adj(const pact_geometry* g, const pact_patches* pt, const float* w,
                                          const float* d, int m, const float* dL_dH, float* dL_dw,
                                          int accumulate, void* stream) {
    return run_psf(g, pt, w, d, m, 2, dL_dH, nullptr, dL_dw, accumulate, stream);
}

// ---------------------------------------------------------------------------
// pact_mc_deconv_loss_noalloc: the fused pass with its scratch taken from a
// fixed device array instead of a caller-provided workspace, for callers that
// cannot allocate device memory.  The array lives for the life of the process
// on every device that loads the library.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[PACT_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol itself is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
pact_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PACT_ERR_CUDA, "mc_deconv_loss_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(PACT_ERR_UNSUPPORTED, "mc_deconv_loss_noalloc: device index %d", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(PACT_ERR_CUDA, "mc_deconv_loss_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PACT_OK;
}
}  // namespace

extern "C" pact_status pact_mc_deconv_loss_noalloc(const pact_geometry* g, const pact_patches* pt, const float* w,
                                                   const float* Y, const float* d, int m, float eps, float* loss,
                                                   float* loss_pp, float* Xhat, float* dL_dw, void* stream) {
    if (!loss) return fail(PACT_ERR_INVALID_ARG, "mc_deconv_loss_noalloc: loss is NULL");
    PACT_TRY(check_geometry(g));
    PACT_TRY(check_patches(pt));
    PACT_TRY(check_delays(d, m));
    const size_t need = make_plan(g, pt, m).total;
    if (need > (size_t)PACT_NOALLOC_SCRATCH_BYTES)
        return fail(PACT_ERR_SHAPE,
                    "mc_deconv_loss_noalloc: this problem needs %zu bytes of scratch; the built-in scratch array "
                    "holds %zu bytes (use pact_mc_deconv_loss with a workspace instead)",
                    need, (size_t)PACT_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    PACT_TRY(noalloc_scratch(&scratch));
    return run_mcd(g, pt, w, Y, d, m, eps, loss, loss_pp, Xhat, dL_dw, nullptr, 0, scratch,
                   (size_t)PACT_NOALLOC_SCRATCH_BYTES, stream);
}
