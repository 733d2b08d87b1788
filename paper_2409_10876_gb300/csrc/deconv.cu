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
// pass over the register-resident Y (no E - |A|^2/B cancellation), giving
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
    int KT, NG;            // bin tiles, patches per CTA
};

// CTA (kt, grp): bins k = kt*kTPB + threadIdx.x of the patches grp*NG .. grp*NG+NG-1.
// Shared memory: E[j][t] = exp(j|k_t|d_j) for the CTA's bins (each thread reads
// only its own column), then w and dL/dw of the NG patches.
template <int MMAX>
__global__ void __launch_bounds__(kTPB, 2) mcd_kernel(const McdArgs a) {
    extern __shared__ float4 smem4[];
    float2* E = reinterpret_cast<float2*>(smem4);                    // [M][kTPB]
    float* w_s = reinterpret_cast<float*>(E + (size_t)a.M * kTPB);   // [NG][n_t]
    float* dw_s = w_s + (size_t)a.NG * a.g.n_t;                      // [NG][n_t]
    __shared__ float lsum_s[8];
    const int n_t = a.g.n_t;
    const int M = a.M;
    const int kt = blockIdx.x, grp = blockIdx.y;
    const int i0 = grp * a.NG;
    const int ng = min(a.NG, a.N - i0);
    const int tid = threadIdx.x;
    const int k = kt * kTPB + tid;
    const bool valid = k < a.F;

    // ---- per-bin constants (shared by every patch of the group)
    const int half = a.P / 2 + 1;
    const int u = valid ? k / half : 0;
    const int v = valid ? k - u * half : 0;
    const float inv_pdx = 1.f / (a.P * a.g.dx);
    const float fx = v * inv_pdx, fy = (u < a.P / 2 ? u : u - a.P) * inv_pdx;
    const float fm = sqrtf(fx * fx + fy * fy);                  // |k| / 2 pi  [cycles/m]
    const float ex = fm > 0.f ? fx / fm : 1.f, ey = fm > 0.f ? fy / fm : 0.f;
    const float kmag = kTwoPi * fm;
    const float om = ((v == 0 || v == a.P / 2) ? 1.f : 2.f) * kmag * 1e-3f;
    float2 C2 = make_float2(0.f, 0.f);
    for (int j = 0; j < M; ++j) {
        const float2 e = cis_pi(2.f * fm * a.dl.d[j]);
        E[(size_t)j * kTPB + tid] = e;
        C2.x = fmaf(e.x, e.x, fmaf(-e.y, e.y, C2.x));
        C2.y = fmaf(2.f * e.x, e.y, C2.y);
    }
    double2 C2d = make_double2(0.0, 0.0);
    if (a.fp64) {
        const double fxd = v / ((double)a.P * a.g.dx), fyd = (u < a.P / 2 ? u : u - a.P) / ((double)a.P * a.g.dx);
        const double fmd = sqrt(fxd * fxd + fyd * fyd);
        for (int j = 0; j < M; ++j) {
            double sn, cs;
            sincospi(4.0 * fmd * (double)a.dl.d[j], &sn, &cs);
            C2d.x += cs;
            C2d.y += sn;
        }
    }
    for (int q = tid; q < ng * n_t; q += kTPB) {
        w_s[q] = a.w[(size_t)i0 * n_t + q];
        dw_s[q] = 0.f;
    }
    if (tid < 8) lsum_s[tid] = 0.f;
    __syncthreads();

    const float n_over_2pi = n_t / kTwoPi;
    const float Mf = (float)M;
    const float eps = a.eps;
    for (int g = 0; g < ng; ++g) {
        const int i = i0 + g;
        float contrib = 0.f;
        if (valid) {
            const int2 cc = a.centres[i];
            const float2 c = pixel_xy(a.g, cc.x, cc.y);
            const float* wr = w_s + (size_t)g * n_t;
            const Hits h = ring_hits(c.x, c.y, ex, ey, a.g, n_over_2pi);
            const int n2a = h.n1a + 1 == n_t ? 0 : h.n1a + 1;
            const int n2b = h.n1b + 1 == n_t ? 0 : h.n1b + 1;
            const float W1 = fmaf(h.fa, wr[n2a] - wr[h.n1a], wr[h.n1a]);
            const float W2 = fmaf(h.fb, wr[n2b] - wr[h.n1b], wr[h.n1b]);
            const float2 al = cis_pi(-2.f * fm * W1);     // exp(-j|k| W(ang k))
            const float2 be = cis_pi(2.f * fm * W2);      // exp(+j|k| W(ang k + pi))

            const float2* yp = a.Y + (size_t)i * M * a.F + k;
            float2 y[MMAX];
#pragma unroll
            for (int j = 0; j < MMAX; ++j)
                if (j < M) y[j] = __ldcs(yp + (size_t)j * a.F);

            // pass 1: S1 = sum cos(|k|d_j) Y_j, S2 = sum sin(|k|d_j) Y_j
            float2 S1 = make_float2(0.f, 0.f), S2 = S1;
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < M) {
                    const float2 e = E[(size_t)j * kTPB + tid];
                    S1.x = fmaf(e.x, y[j].x, S1.x);
                    S1.y = fmaf(e.x, y[j].y, S1.y);
                    S2.x = fmaf(e.y, y[j].x, S2.x);
                    S2.y = fmaf(e.y, y[j].y, S2.y);
                }
            }
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
                const double Bd = 0.5 * ((double)M + (cs * C2d.x - sn * C2d.y));
                const double Dd = Bd + (double)eps;
                B = (float)Bd;
                D = (float)Dd;
                X = Dd != 0.0 ? make_float2((float)(A.x / Dd), (float)(A.y / Dd)) : make_float2(0.f, 0.f);
            } else {
                B = 0.5f * (Mf + (ab.x * C2.x - ab.y * C2.y));
                D = B + eps;
                const float iD = D != 0.f ? 1.f / D : 0.f;
                X = make_float2(A.x * iD, A.y * iD);
            }

            // pass 2: explicit residual R_j = Y_j - cos(|k|d_j) p - sin(|k|d_j) q
            const float2 pp = make_float2(0.5f * (al.x + be.x), 0.5f * (al.y + be.y));
            const float2 qm = make_float2(0.5f * (al.x - be.x), 0.5f * (al.y - be.y));
            const float2 p = cmul(pp, X);
            const float2 q0 = cmul(qm, X);
            const float2 q = make_float2(-q0.y, q0.x);
            float e2 = 0.f;
            float2 T1 = make_float2(0.f, 0.f), T2 = T1;
#pragma unroll
            for (int j = 0; j < MMAX; ++j) {
                if (j < M) {
                    const float2 e = E[(size_t)j * kTPB + tid];
                    float2 R;
                    R.x = y[j].x - fmaf(e.x, p.x, e.y * q.x);
                    R.y = y[j].y - fmaf(e.x, p.y, e.y * q.y);
                    e2 = fmaf(R.x, R.x, fmaf(R.y, R.y, e2));
                    T1.x = fmaf(e.x, R.x, T1.x);
                    T1.y = fmaf(-e.x, R.y, T1.y);
                    T2.x = fmaf(e.y, R.x, T2.x);
                    T2.y = fmaf(-e.y, R.y, T2.y);
                }
            }
            contrib = om * e2;
            if (a.Xhat) a.Xhat[(size_t)i * a.F + k] = X;

            if (a.want_grad && fm > 0.f && D != 0.f) {
                const float iD = 1.f / D;
                const float2 Kc = make_float2(-om * X.x * iD, -om * X.y * iD);   // conj(K)
                const float b2 = B + 2.f * eps;
                const float2 abC2 = cmul(ab, C2);
                const float2 xc = make_float2(X.x, -X.y);
                const float2 hp = make_float2(0.5f * (Mf + abC2.x), 0.5f * abC2.y);
                const float2 hq = make_float2(0.5f * (Mf + abC2.x), -0.5f * abC2.y);
                const float2 tp = make_float2(T1.x - T2.y, T1.y + T2.x);
                const float2 tq = make_float2(T1.x + T2.y, T1.y - T2.x);
                const float2 ap = cmul(al, tp), bq = cmul(be, tq);
                const float2 xhp = cmul(xc, hp), xhq = cmul(xc, hq);
                const float2 SP = make_float2(b2 * ap.x - eps * xhp.x, b2 * ap.y - eps * xhp.y);
                const float2 SQ = make_float2(b2 * bq.x - eps * xhq.x, b2 * bq.y - eps * xhq.y);
                const float gW1 = kmag * (Kc.x * SP.y + Kc.y * SP.x);
                const float gW2 = -kmag * (Kc.x * SQ.y + Kc.y * SQ.x);
                float* dwr = dw_s + (size_t)g * n_t;
                atomicAdd(dwr + h.n1a, (1.f - h.fa) * gW1);
                atomicAdd(dwr + n2a, h.fa * gW1);
                atomicAdd(dwr + h.n1b, (1.f - h.fb) * gW2);
                atomicAdd(dwr + n2b, h.fb * gW2);
            }
        }
        contrib = warp_sum(contrib);
        if ((tid & 31) == 0) atomicAdd(&lsum_s[g], contrib);
    }
    __syncthreads();
    if (tid < ng) a.part_loss[(size_t)(i0 + tid) * a.KT + kt] = lsum_s[tid];
    if (a.want_grad) {
        for (int q = tid; q < ng * n_t; q += kTPB) {
            const int g = q / n_t, n = q - (q / n_t) * n_t;
            a.part_dw[((size_t)(i0 + g) * a.KT + kt) * n_t + n] = dw_s[q];
        }
    }
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
    int KT, NG;
    size_t smem, off_dw, total;
};

Plan make_plan(const pact_geometry* g, const pact_patches* pt, int m) {
    Plan p;
    const int F = pt->p * (pt->p / 2 + 1);
    p.KT = (F + kTPB - 1) / kTPB;
    const int sms = num_sms();
    int ng = (int)((long long)p.KT * pt->n / (2LL * sms));
    p.NG = std::max(1, std::min(8, ng));
    p.smem = (size_t)m * kTPB * sizeof(float2) + 2 * (size_t)p.NG * g->n_t * sizeof(float);
    const size_t n_loss = (size_t)pt->n * p.KT;
    p.off_dw = align_up(n_loss * sizeof(float), 256);
    p.total = p.off_dw + align_up((size_t)pt->n * p.KT * g->n_t * sizeof(float), 256);
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

template <int MMAX>
pact_status launch_mcd(const McdArgs& a, size_t smem, cudaStream_t st) {
    PACT_TRY(ensure_smem((const void*)mcd_kernel<MMAX>, smem, "mc_deconv_loss: shared memory attribute"));
    dim3 grid(a.KT, (a.N + a.NG - 1) / a.NG);
    mcd_kernel<MMAX><<<grid, kTPB, smem, st>>>(a);
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
    if (reinterpret_cast<uintptr_t>(Y) % 8) return fail(PACT_ERR_INVALID_ARG, "Y must be 8-byte aligned");
    const Plan pl = make_plan(g, pt, m);
    if (pl.smem > 220 * 1024) return fail(PACT_ERR_SHAPE, "mc_deconv_loss: n_t x channels too large for shared memory");
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
    a.KT = pl.KT;
    a.NG = pl.NG;
    pact_status s;
    if (m <= 8) s = launch_mcd<8>(a, pl.smem, st);
    else if (m <= 16) s = launch_mcd<16>(a, pl.smem, st);
    else if (m <= 32) s = launch_mcd<32>(a, pl.smem, st);
    else s = launch_mcd<64>(a, pl.smem, st);
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
