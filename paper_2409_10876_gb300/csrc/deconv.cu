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

#include "pact_internal.cuh"

namespace pact {
namespace {

constexpr int kTPB = 256;
constexpr float kTwoPi = 6.283185307179586f;

struct Phase {
    int uniform;      // delays uniformly spaced: E_j by recurrence
    float d0, dd;
};

Phase make_phase(const float* d, int m) {
    Phase p;
    p.d0 = d[0];
    p.dd = m > 1 ? (d[m - 1] - d[0]) / (float)(m - 1) : 0.f;
    float mx = 0.f;
    for (int j = 0; j < m; ++j) mx = fmaxf(mx, fabsf(d[j]));
    int uni = 1;
    for (int j = 0; j < m; ++j)
        if (fabsf(d[j] - (p.d0 + j * p.dd)) > 1e-6f * mx + 1e-12f) uni = 0;
    p.uniform = uni;
    return p;
}

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

// E_j = exp(j |k| d_j) = exp(j pi 2 fm d_j), generated in channel order.
// Uniform delays use the rotation exp(j |k| dd), re-anchored every 8 channels.
struct PhaseGen {
    float2 e, rot;
    float two_fm;
    __device__ __forceinline__ void start(const Phase& ph, float fm) {
        two_fm = 2.f * fm;
        if (ph.uniform) {
            e = cis_pi(two_fm * ph.d0);
            rot = cis_pi(two_fm * ph.dd);
        }
    }
    __device__ __forceinline__ float2 at(const Phase& ph, const Delays& dl, int j) {
        if (!ph.uniform) return cis_pi(two_fm * dl.d[j]);
        if (j > 0) {
            if ((j & 7) == 0)
                e = cis_pi(two_fm * fmaf((float)j, ph.dd, ph.d0));
            else
                e = cmul(e, rot);
        }
        return e;
    }
};

struct McdArgs {
    Geo g;
    int N, P, F, M;
    const int2* centres;
    const float* w;
    const float2* Y;
    float eps;
    Delays dl;
    Phase ph;
    float2* Xhat;
    int want_grad;
    int fp64;
    const double2* c2tab;  // [F]: sum_j exp(2j|k|d_j) in FP64 (fp64 path)
    float* part_loss;      // [N][S]
    float* part_dw;        // [N][S][n_t]
    int S, chunk;
};

template <int MMAX>
__global__ void __launch_bounds__(kTPB) mcd_kernel(const McdArgs a) {
    extern __shared__ float smem[];
    __shared__ float red[kTPB / 32];
    const int n_t = a.g.n_t;
    float* w_s = smem;
    float* dw_s = smem + n_t;
    const int i = blockIdx.y, s = blockIdx.x;
    for (int n = threadIdx.x; n < n_t; n += kTPB) {
        w_s[n] = a.w[(size_t)i * n_t + n];
        dw_s[n] = 0.f;
    }
    __syncthreads();
    const int2 cc = a.centres[i];
    const float2 c = pixel_xy(a.g, cc.x, cc.y);
    const float inv_pdx = 1.f / (a.P * a.g.dx);
    const float n_over_2pi = n_t / kTwoPi;
    const int k0 = s * a.chunk;
    const int k1 = min(a.F, k0 + a.chunk);
    const int M = a.M;
    const float Mf = (float)M;
    const float eps = a.eps;
    float lsum = 0.f;

    for (int k = k0 + threadIdx.x; k < k1; k += kTPB) {
        int u, v;
        const Tf t = make_tf(a.g, a.P, inv_pdx, n_over_2pi, c, w_s, k, u, v);
        // stream this bin's M channels into registers (read once per pass)
        const float2* yp = a.Y + (size_t)i * M * a.F + k;
        float2 y[MMAX];
#pragma unroll
        for (int j = 0; j < MMAX; ++j)
            if (j < M) y[j] = __ldcs(yp + (size_t)j * a.F);

        // pass 1: channel sums of the data
        PhaseGen pg;
        pg.start(a.ph, t.fm);
        float2 S1 = make_float2(0.f, 0.f), S2 = S1, C2 = S1;
#pragma unroll
        for (int j = 0; j < MMAX; ++j) {
            if (j < M) {
                const float2 e = pg.at(a.ph, a.dl, j);
                S1.x = fmaf(e.x, y[j].x, S1.x);
                S1.y = fmaf(e.x, y[j].y, S1.y);
                S2.x = fmaf(e.y, y[j].x, S2.x);
                S2.y = fmaf(e.y, y[j].y, S2.y);
                C2.x = fmaf(e.x, e.x, fmaf(-e.y, e.y, C2.x));
                C2.y = fmaf(2.f * e.x, e.y, C2.y);
            }
        }
        const float2 U = make_float2(S1.x + S2.y, S1.y - S2.x);   // sum conj(E_j) Y_j
        const float2 V = make_float2(S1.x - S2.y, S1.y + S2.x);   // sum E_j Y_j
        const float2 ca = cmulc(t.a, U), cb = cmulc(t.b, V);
        const float2 A = make_float2(0.5f * (ca.x + cb.x), 0.5f * (ca.y + cb.y));
        const float2 ab = cmulc(t.b, t.a);                          // a conj(b)
        float B, D;
        float2 X;
        if (a.fp64) {
            const double2 c2 = a.c2tab[k];
            double sn, cs;
            sincospi(-2.0 * (double)t.fm * ((double)t.W1 + (double)t.W2), &sn, &cs);
            const double Bd = 0.5 * ((double)M + (cs * c2.x - sn * c2.y));
            const double Dd = Bd + (double)eps;
            B = (float)Bd;
            D = (float)Dd;
            X = Dd != 0.0 ? make_float2((float)(A.x / Dd), (float)(A.y / Dd)) : make_float2(0.f, 0.f);
        } else {
            B = 0.5f * (Mf + (ab.x * C2.x - ab.y * C2.y));
            D = B + eps;
            X = D != 0.f ? make_float2(A.x / D, A.y / D) : make_float2(0.f, 0.f);
        }

        // pass 2: explicit residual, loss, adjoint channel sums
        const float2 pp = make_float2(0.5f * (t.a.x + t.b.x), 0.5f * (t.a.y + t.b.y));
        const float2 qm = make_float2(0.5f * (t.a.x - t.b.x), 0.5f * (t.a.y - t.b.y));
        const float2 p = cmul(pp, X);
        const float2 q0 = cmul(qm, X);
        const float2 q = make_float2(-q0.y, q0.x);                 // j * q0
        pg.start(a.ph, t.fm);
        float e2 = 0.f;
        float2 T1 = make_float2(0.f, 0.f), T2 = T1;
#pragma unroll
        for (int j = 0; j < MMAX; ++j) {
            if (j < M) {
                const float2 e = pg.at(a.ph, a.dl, j);
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
        const float cv = (v == 0 || v == a.P / 2) ? 1.f : 2.f;
        const float kmag = kTwoPi * t.fm;
        const float om = cv * kmag * 1e-3f;
        lsum = fmaf(om, e2, lsum);
        if (a.Xhat) a.Xhat[(size_t)i * a.F + k] = X;

        if (a.want_grad && t.fm > 0.f && D != 0.f) {
            const float2 Kc = make_float2(-om * X.x / D, -om * X.y / D);   // conj(K)
            const float b2 = B + 2.f * eps;
            const float2 abC2 = cmul(ab, C2);
            const float2 xc = make_float2(X.x, -X.y);
            const float2 hp = make_float2(0.5f * (Mf + abC2.x), 0.5f * abC2.y);   // sum conj(H)P
            const float2 hq = make_float2(0.5f * (Mf + abC2.x), -0.5f * abC2.y);  // sum conj(H)Q
            const float2 tp = make_float2(T1.x - T2.y, T1.y + T2.x);              // T1 + jT2
            const float2 tq = make_float2(T1.x + T2.y, T1.y - T2.x);              // T1 - jT2
            const float2 ap = cmul(t.a, tp), bq = cmul(t.b, tq);
            const float2 xhp = cmul(xc, hp), xhq = cmul(xc, hq);
            const float2 SP = make_float2(b2 * ap.x - eps * xhp.x, b2 * ap.y - eps * xhp.y);
            const float2 SQ = make_float2(b2 * bq.x - eps * xhq.x, b2 * bq.y - eps * xhq.y);
            const float gW1 = kmag * (Kc.x * SP.y + Kc.y * SP.x);
            const float gW2 = -kmag * (Kc.x * SQ.y + Kc.y * SQ.x);
            const int n2a = t.n1a + 1 == n_t ? 0 : t.n1a + 1;
            const int n2b = t.n1b + 1 == n_t ? 0 : t.n1b + 1;
            atomicAdd(&dw_s[t.n1a], (1.f - t.fa) * gW1);
            atomicAdd(&dw_s[n2a], t.fa * gW1);
            atomicAdd(&dw_s[t.n1b], (1.f - t.fb) * gW2);
            atomicAdd(&dw_s[n2b], t.fb * gW2);
        }
    }
    const float tot = block_sum(lsum, red);
    if (threadIdx.x == 0) a.part_loss[(size_t)i * a.S + s] = tot;
    if (a.want_grad) {
        __syncthreads();
        float* dst = a.part_dw + ((size_t)i * a.S + s) * n_t;
        for (int n = threadIdx.x; n < n_t; n += kTPB) dst[n] = dw_s[n];
    }
}

// FP64 table C2(k) = sum_j exp(2j|k|d_j) for the eps < 1e-6 path.
__global__ void c2_table_kernel(int P, int F, double dx, Delays dl, double2* out) {
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
    int S, chunk;
    size_t off_dw, off_c2, total;
};

Plan make_plan(const pact_geometry* g, const pact_patches* pt, int m) {
    (void)m;
    Plan p;
    const int F = pt->p * (pt->p / 2 + 1);
    const int sms = num_sms();
    int S = (2 * sms + pt->n - 1) / pt->n;
    S = std::max(1, std::min(S, std::max(1, F / kTPB)));
    p.S = S;
    p.chunk = (F + S - 1) / S;
    const size_t n_loss = (size_t)pt->n * S;
    p.off_dw = align_up(n_loss * sizeof(float), 256);
    p.off_c2 = p.off_dw + align_up((size_t)pt->n * S * g->n_t * sizeof(float), 256);
    p.total = p.off_c2 + align_up((size_t)F * sizeof(double2), 256);
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
pact_status launch_mcd(const McdArgs& a, cudaStream_t st) {
    const size_t shm = 2 * (size_t)a.g.n_t * sizeof(float);
    PACT_TRY(ensure_smem((const void*)mcd_kernel<MMAX>, shm, "mc_deconv_loss: shared memory attribute"));
    dim3 grid(a.S, a.N);
    mcd_kernel<MMAX><<<grid, kTPB, shm, st>>>(a);
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
    if ((size_t)g->n_t * 2 * sizeof(float) > 200 * 1024) return fail(PACT_ERR_SHAPE, "n_t too large");
    const Plan pl = make_plan(g, pt, m);
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
    a.ph = make_phase(d, m);
    a.Xhat = reinterpret_cast<float2*>(Xhat);
    a.want_grad = dL_dw != nullptr;
    a.fp64 = eps < 1e-6f;
    a.c2tab = reinterpret_cast<const double2*>(base + pl.off_c2);
    a.part_loss = reinterpret_cast<float*>(base);
    a.part_dw = reinterpret_cast<float*>(base + pl.off_dw);
    a.S = pl.S;
    a.chunk = pl.chunk;
    if (a.fp64) {
        c2_table_kernel<<<(a.F + 127) / 128, 128, 0, st>>>(a.P, a.F, (double)g->dx, a.dl,
                                                           reinterpret_cast<double2*>(base + pl.off_c2));
        PACT_TRY(check_launch("mc_deconv_loss: c2 table"));
    }
    pact_status s;
    if (m <= 8) s = launch_mcd<8>(a, st);
    else if (m <= 16) s = launch_mcd<16>(a, st);
    else if (m <= 32) s = launch_mcd<32>(a, st);
    else s = launch_mcd<64>(a, st);
    if (s != PACT_OK) return s;
    FinArgs f;
    f.N = a.N;
    f.S = a.S;
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
