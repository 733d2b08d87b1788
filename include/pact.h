/*
 * pact.h -- C ABI of the GB300 (sm_103a) library for the per-iteration hot
 * path of self-supervised joint speed-of-sound (SOS) / image recovery in
 * ring-array photoacoustic computed tomography (Li, Cui, Ma, Alexander,
 * "Coordinate-based Speed of Sound Recovery for Aberration-Corrected
 * Photoacoustic Computed Tomography", arXiv 2409.10876).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - SI units: metres, seconds, m/s.  All arrays are dense and row-major.
 *  - Complex arrays are interleaved float pairs (re, im): a "c64" array of
 *    n complex values is a float array of 2n values, 8-byte aligned.
 *  - Device pointers are caller-owned device memory; the library never
 *    allocates.  Scratch space, where needed, is a caller-provided
 *    workspace whose size the matching *_workspace_size call returns.
 *  - Host pointers (geometry structs, delay lists) are read during the call
 *    only; their values are copied into kernel arguments, so a call
 *    captured into a CUDA graph keeps the values it saw at capture.
 *  - Every call is asynchronous on the given stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream) and never synchronises.
 *  - Outputs are overwritten unless an `accumulate` flag is 1 (then +=).
 *  - Return value: PACT_OK or an error code; pact_last_error_message()
 *    gives a thread-local description of the last failure.  Invalid
 *    arguments are rejected on the host before anything is launched.
 *    No kernel traps; launch failures come back as PACT_ERR_CUDA.
 *
 * Geometry (Sec. 3.1, Sec. S1.1)
 * ------------------------------
 *  Image pixel (row a, col b) sits at x = (b - (W-1)/2) dx,
 *  y = (a - (H-1)/2) dx.  Transducer n sits at
 *  r_n = R (cos(2 pi n / N_t + phase), sin(2 pi n / N_t + phase)).
 *  The SOS pixel grid has G x G nodes at x = (q - (G-1)/2) sos_dx (column q),
 *  y = (p - (G-1)/2) sos_dx (row p), bilinearly interpolated and clamped at
 *  the edge; rays count only inside the mask disk |r| <= mask_radius and
 *  use v_bg outside it (Sec. 3.3: circular mask, fixed background SOS).
 *  Patch i covers rows c_a - P/2 .. c_a + P/2 - 1 (and the same for
 *  columns) around its centre pixel (c_a, c_b) = r'_i, zero outside the
 *  image, and is weighted by a Gaussian window of the given FWHM
 *  (Sec. S1.5).  Spectra are the orthonormal 2-D DFT (kernel
 *  exp(-j k.rho), scale 1/P) on the rfft half-spectrum: [P][P/2+1] with
 *  rows in fftfreq order, F = P (P/2 + 1) bins per patch, k in rad/m.
 */
#ifndef PACT_H
#define PACT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pact_status {
    PACT_OK = 0,
    PACT_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, bad flag */
    PACT_ERR_SHAPE = 2,         /* sizes outside what the kernels support */
    PACT_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    PACT_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (status calls) */
    PACT_ERR_NONFINITE = 5,     /* non-finite values detected (reserved for callers' checks) */
    PACT_ERR_UNSUPPORTED = 6    /* feature not available on this device/build */
} pact_status;

/* Ring array, image grid and SOS grid (all host values). */
typedef struct pact_geometry {
    int   n_t;          /* transducers on the ring, >= 4 */
    float ring_radius;  /* R [m]; every patch centre lies inside the ring */
    float ring_phase;   /* angle of transducer 0 [rad] */
    float v0;           /* SOS assumed by DAS (Eq. 1) [m/s] */
    float v_bg;         /* fixed background SOS outside the mask [m/s] */
    int   img_h;        /* image rows H */
    int   img_w;        /* image columns W */
    float dx;           /* pixel pitch [m] */
    int   sos_g;        /* SOS nodes per side G, 2 <= G <= 512 */
    float sos_dx;       /* node pitch [m] */
    float mask_radius;  /* SOS mask radius [m] */
    float ray_step;     /* midpoint-rule step of the ray integral [m] */
} pact_geometry;

/* Patch set (Sec. S1.5). */
typedef struct pact_patches {
    int        n;            /* number of patches N >= 1 */
    int        p;            /* patch size P, even, 4 <= P <= 128 */
    const int* centres;      /* DEVICE int32 [N][2]: (row, col) of r'_i */
    float      window_fwhm;  /* Gaussian window FWHM [m] */
} pact_patches;

#define PACT_MAX_CHANNELS 64   /* largest delay-channel count M */

/* Library version string (static storage). */
const char* pact_version(void);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* pact_last_error_message(void);

/*
 * Delay-and-sum stack, Eq. 1 (Sec. 3.1, "DAS stack" of Sec. 3.2):
 *   stack[j][a][b] = sum_n S(((|r'_ab - r_n| - d_j) / v0 - t0) * fs, n)
 * with S linearly interpolated between samples and zero outside
 * [0, n_s - 1].
 *   rf     DEVICE float [N_t][n_s]  channel data, sample q at time t0 + q/fs
 *   d      HOST float [m]           extra delay distances d_j [m]
 *   stack  DEVICE float [m][H][W]   output
 * Errors: INVALID_ARG for null pointers or non-positive sizes, SHAPE for
 * m > PACT_MAX_CHANNELS.
 */
pact_status pact_das_stack(const pact_geometry* g, const float* rf, int n_s, float fs, float t0,
                           const float* d, int m, float* stack, void* stream);

/*
 * Synthetic ring channel data: the input of Eq. 1 for end-to-end runs.
 * The paper's data are the time derivative of the photoacoustic pressure,
 * S = -2 dp/dt (Sec. S1.1); here every pixel p of the initial-pressure image
 * p0 emits one pulse that reaches transducer n after the straight-ray time
 * of flight of Eq. 2-3,
 *   tau(p, n) = int dl / v = (|r_p - r_n| - w(p, n)) / v0,
 * with w the wavefront error of pact_sos_to_delays on the segment r_p -> r_n
 * (same quadrature, mask and background), and
 *   rf[n][q] = sum_p p0_p (R_s / |r_p - r_n|)^spread psi(t0 + q/fs - tau(p, n)),
 *   psi(t) = (1 - t^2 / sigma^2) exp(-t^2 / (2 sigma^2)),
 * -2 dp/dt of an N-shaped pressure pulse p (the time derivative of a
 * Gaussian): even, psi(0) = 1, amplitude spectrum peaking at
 * 1 / (sqrt(2) pi sigma).  psi is evaluated within 6 sigma of each arrival
 * (|psi| < 6e-7 beyond).
 * Model mismatches for robustness runs: spread = 1/2 adds cylindrical
 * spreading; ring_dr moves the receiving ring to radius R_s = R + ring_dr
 * while the geometry (and DAS) keep R.  spread = ring_dr = 0 is the model
 * the method assumes.
 */
typedef struct pact_rf_params {
    float fs;        /* sample rate [Hz] > 0 */
    float t0;        /* time of sample 0 [s] */
    int   n_s;       /* samples per transducer, 1 <= n_s <= 49152 */
    float sigma;     /* pulse width [s] > 0, 6 sigma fs <= 1024 */
    float spread;    /* amplitude exponent (0: none, 0.5: cylindrical) */
    float ring_dr;   /* receiving-ring radius offset [m], R + ring_dr > 0 */
} pact_rf_params;

/*
 * Workspace bytes for pact_rf_synth processing up to `pixels_per_pass`
 * pixels per pass (N_t floats per pixel: the transposed wavefront errors of
 * one pass).  Any workspace of at least pact_rf_synth_workspace_size(g, 1)
 * bytes works; larger ones take fewer passes.  0 for an invalid geometry.
 */
size_t pact_rf_synth_workspace_size(const pact_geometry* g, int pixels_per_pass);

/*
 * rf = channel data of p0 (see above), overwritten.
 *   p0   DEVICE float [H][W]    initial pressure (pixels equal to 0 emit nothing)
 *   sos  DEVICE float [G][G]    node SOS [m/s]
 *   rp   HOST                   sampling, pulse and mismatch parameters
 *   rf   DEVICE float [N_t][n_s] output
 *   ws   DEVICE workspace, 256-byte aligned, ws_bytes >= pact_rf_synth_workspace_size(g, 1)
 * The passes over pixel blocks sum into rf in a fixed order; within a pass
 * the pulses of one transducer are summed with shared-memory atomics (the
 * rounding order can vary from run to run).
 * Errors: INVALID_ARG for null pointers, bad parameters or a small or
 * misaligned workspace; SHAPE for n_s or pulse widths beyond the limits.
 */
pact_status pact_rf_synth(const pact_geometry* g, const float* p0, const float* sos, const pact_rf_params* rp,
                          float* rf, void* ws, size_t ws_bytes, void* stream);

/*
 * Transducer band-limit for channel data (no counterpart in the paper: a model
 * mismatch for robustness studies, next to the spreading and ring-radius
 * offsets of pact_rf_synth).  Every channel is filtered along time by the
 * zero-phase impulse response
 *   h_k = (2 / Z) exp(-tau_k^2 / (2 s_t^2)) cos(2 pi fc tau_k),  tau_k = k / fs,
 * |k| <= K = ceil(4 s_t fs), Z = sum_k exp(-tau_k^2 / (2 s_t^2)) (unit gain at
 * fc), s_t = 1 / (2 pi s_f), s_f = frac_bw fc / (2 sqrt(2 ln 2)): the amplitude
 * response is a Gaussian in f of full width frac_bw fc at half amplitude.
 *   rf_in   DEVICE float [n_t][n_s]
 *   rf_out  DEVICE float [n_t][n_s], output; a different buffer from rf_in
 *   rf_out[n][q] = sum_k h_k rf_in[n][q - k], zero outside the record.
 * Errors: INVALID_ARG for NULL or equal buffers, sizes < 1, fs <= 0, fc not
 * in (0, fs/2), frac_bw not in (0, 2]; SHAPE for n_t > 65535 or K > 512.
 */
pact_status pact_rf_bandpass(const float* rf_in, float* rf_out, int n_t, int n_s, float fs, float fc, float frac_bw,
                             void* stream);

/*
 * Patch spectra (Sec. S1.5, the Y_i(k; d_j) of Eq. 5): crop each of the m
 * channels around every patch centre, multiply by the Gaussian window
 * exp(-|rho|^2 / (2 sigma^2)), FWHM = 2 sqrt(2 ln 2) sigma, rho measured from
 * local index P/2, and take the orthonormal 2-D DFT on the half-spectrum.
 *   stack  DEVICE float [m][H][W]
 *   Y      DEVICE c64 [N][m][P][P/2+1]   output
 */
pact_status pact_patch_fft(const pact_geometry* g, const pact_patches* pt, const float* stack, int m,
                           float* Y, void* stream);

/*
 * Wavefront errors, Eq. 2-3:  w_{i,n} = int_{r'_i}^{r_n} (1 - v0 / v(l)) dl,
 * evaluated as the integral of the slowness excess (v - v0)/v with
 * v - v0 interpolated directly from the node excesses, by the midpoint rule
 * with step ray_step over the part of the segment inside the mask (the last
 * partial step weighted by its length), plus (1 - v0/v_bg) times the
 * length outside the mask.
 *   sos  DEVICE float [G][G]   node SOS [m/s]
 *   w    DEVICE float [N][N_t] output [m]
 */
pact_status pact_sos_to_delays(const pact_geometry* g, const pact_patches* pt, const float* sos,
                               float* w, void* stream);

/*
 * pact_sos_to_delays that also sets clear[0 .. n_clear) to zero in the same
 * launch (no counterpart in the paper: an iteration-fusion helper).  A
 * recovery iteration (Sec. 3.3) passes the dL/dw buffer that the fused pass
 * (pact_mc_deconv_loss_tabled with accumulate = 1) adds its gradient to
 * next, which saves a clearing launch per iteration.
 *   clear    DEVICE float [n_clear], 16-byte aligned; may not overlap w or sos
 * Errors: those of pact_sos_to_delays; INVALID_ARG for a NULL or misaligned
 * clear with n_clear > 0.
 */
pact_status pact_sos_to_delays_clear(const pact_geometry* g, const pact_patches* pt, const float* sos, float* w,
                                     float* clear, size_t n_clear, void* stream);

/* Workspace bytes of pact_sos_to_delays_adj for this geometry. */
size_t pact_sos_to_delays_adj_workspace_size(const pact_geometry* g, const pact_patches* pt);

/*
 * Adjoint of Eq. 3 (backpropagation to the pixel-grid SOS, Sec. 3.3):
 *   dL_dsos[p][q] (+)= sum_{i,n} dL_dw[i][n] * sum_s h_s v0 / v(l_s)^2 * b_pq(l_s)
 * with b_pq the bilinear weight of node (p, q) at sample l_s.
 *   dL_dw    DEVICE float [N][N_t]
 *   dL_dsos  DEVICE float [G][G]   output (accumulate = 1 adds to it)
 *   ws       DEVICE workspace of at least the size above (256-byte aligned)
 * Errors: INVALID_ARG if ws is null or smaller than required.
 */
pact_status pact_sos_to_delays_adj(const pact_geometry* g, const pact_patches* pt, const float* sos,
                                   const float* dL_dw, float* dL_dsos, int accumulate, void* ws,
                                   size_t ws_bytes, void* stream);

/*
 * The two ends of a pixel-grid recovery iteration (Sec. 3.3: Adam on the
 * Eq. 7 loss, data term plus lambda TV) with fewer launches; no counterpart in
 * the paper (iteration fusion).  An iteration is
 *   pact_sos_to_delays_tv -> pact_mc_deconv_loss_tabled (accumulate = 1)
 *   -> pact_sos_to_delays_adj_adam
 * and equals pact_sos_to_delays_clear -> the fused pass -> pact_sos_to_delays_adj
 * -> pact_tv (value and gradient, accumulate = 1) -> pact_adam_step, up to the
 * rounding of the additions.
 *
 * pact_sos_to_delays_tv: pact_sos_to_delays_clear, and in the same launch the
 * TV terms of Eq. 7 at the SOS it reads: lambda times the subgradient
 * (sign(0) = 0) and lambda times TV(v) in per-CTA parts, into tv_ws.
 *   tv_ws   DEVICE, 256-byte aligned, pact_sos_to_delays_tv_workspace_size
 *           bytes; its contents are for the pact_sos_to_delays_adj_adam call
 *           of the same iteration (same geometry and patches).
 * Errors: those of pact_sos_to_delays_clear; INVALID_ARG for a NULL,
 * misaligned or small tv_ws or a non-finite lambda.
 *
 * pact_sos_to_delays_adj_adam: the adjoint of Eq. 3 as pact_sos_to_delays_adj,
 * then one kernel that per node adds the partial grids (fixed order) and the
 * TV subgradient from tv_ws, writes the gradient to dL_dsos (if not NULL),
 * and takes one Adam step on sos in place exactly as pact_adam_step (m, v,
 * step, step_counter, lr, betas, eps, mask with the same meaning); it also
 * adds lambda TV(v) to *loss (if loss and tv_ws are not NULL; the per-CTA parts
 * in a fixed order).  The TV terms were taken before this update, so no node
 * is read after another thread has moved it.
 *   sos      DEVICE float [G][G], updated in place
 *   tv_ws    as above, or NULL for lambda = 0 (no TV term)
 *   loss     DEVICE float [1] or NULL
 *   dL_dsos  DEVICE float [G][G] or NULL: the gradient of the step
 *   ws       as pact_sos_to_delays_adj
 * Errors: those of pact_sos_to_delays_adj and pact_adam_step.
 */
size_t pact_sos_to_delays_tv_workspace_size(const pact_geometry* g, const pact_patches* pt);
pact_status pact_sos_to_delays_tv(const pact_geometry* g, const pact_patches* pt, const float* sos, float* w,
                                  float* clear, size_t n_clear, float lambda, void* tv_ws, size_t tv_ws_bytes,
                                  void* stream);
pact_status pact_sos_to_delays_adj_adam(const pact_geometry* g, const pact_patches* pt, float* sos,
                                        const float* dL_dw, const void* tv_ws, float* loss, float* dL_dsos,
                                        float* m, float* v, int step, int* step_counter, float lr, float beta1,
                                        float beta2, float eps, const unsigned char* mask, void* ws,
                                        size_t ws_bytes, void* stream);

/*
 * Wavefront transfer functions, Eq. 4, in the sign that Eq. 1 implies for
 * the forward DFT kernel exp(-j k.rho) (the complex conjugate of the
 * printed form):
 *   H_ij(k) = 1/2 ( exp(+j|k|(d_j - W_i(ang k))) + exp(-j|k|(d_j - W_i(ang k + pi))) )
 * where W_i(phi) interpolates w_{i,.} linearly in ring angle at the point
 * where the ray from r'_i in direction phi meets the ring.
 *   w  DEVICE float [N][N_t];  d HOST float [m];  H DEVICE c64 [N][m][P][P/2+1]
 */
pact_status pact_psf_synth(const pact_geometry* g, const pact_patches* pt, const float* w,
                           const float* d, int m, float* H, void* stream);

/*
 * Adjoint of pact_psf_synth: dL_dw[i][n] (+)= sum over bins and channels of
 * Re(conj(dL_dH) dH/dw), where dL_dH holds (dL/dRe H, dL/dIm H) pairs
 * (the convention of PyTorch complex gradients).
 *   dL_dH DEVICE c64 [N][m][P][P/2+1];  dL_dw DEVICE float [N][N_t]
 */
pact_status pact_psf_synth_adj(const pact_geometry* g, const pact_patches* pt, const float* w,
                               const float* d, int m, const float* dL_dH, float* dL_dw,
                               int accumulate, void* stream);

/*
 * Multi-channel forward model, Eq. 5:  Y_ij(k) (+)= H_ij(k) X_i(k) with H as
 * in pact_psf_synth (synthesises measurements from a clean patch spectrum).
 *   X DEVICE c64 [N][P][P/2+1];  Y DEVICE c64 [N][m][P][P/2+1]
 */
pact_status pact_forward_model(const pact_geometry* g, const pact_patches* pt, const float* w,
                               const float* d, int m, const float* X, float* Y, int accumulate,
                               void* stream);

/* Workspace bytes of pact_mc_deconv_loss / pact_mc_deconv_loss_adj. */
size_t pact_mc_deconv_loss_workspace_size(const pact_geometry* g, const pact_patches* pt, int m);

/*
 * Fused multi-channel deconvolution and loss, Eq. 6-7, with the transfer
 * functions of Eq. 4 synthesised on the fly and never stored:
 *   X_i(k) = sum_j conj(H_ij) Y_ij / (sum_j |H_ij|^2 + eps)          (Eq. 6)
 *   L      = sum_i sum_k c_k |k|_mm sum_j |Y_ij - H_ij X_i|^2        (Eq. 7)
 * (|k| in rad/mm, c_k = 1 on columns k_x = 0 and Nyquist, 2 elsewhere;
 * X_i = 0 where the denominator is 0).  eps is the Wiener-style regulariser.
 * When dL_dw is not NULL the same pass also returns the exact gradient
 * dL/dw (hand-written adjoint: X_i is recomputed, never stored).
 *   w        DEVICE float [N][N_t]          wavefront errors
 *   Y        DEVICE c64 [N][m][P][P/2+1]    patch spectra, 16-byte aligned
 *   d        HOST float [m]                 delays [m]
 *   loss     DEVICE float [1]               output (data term only)
 *   loss_pp  DEVICE float [N] or NULL       per-patch data term
 *   Xhat     DEVICE c64 [N][P][P/2+1] or NULL
 *   dL_dw    DEVICE float [N][N_t] or NULL  output gradient
 *   ws       DEVICE workspace (256-byte aligned) of the size above
 * For eps >= 1e-6 (with N_t a multiple of 4 and w 16-byte aligned, else as
 * for small eps but in FP32) the residual energy of a bin is evaluated as
 * sum_j |Y_ij|^2 - |A|^2 (B + 2 eps) / (B + eps)^2 (A, B the numerator and
 * denominator sums of Eq. 6), so each Y element is read once; its FP32
 * rounding is about 1e-7 of sum_j |Y_ij|^2 per bin, of either sign.  When
 * eps < 1e-6 the per-bin channel-sum denominator and the division run in FP64
 * and the residual Y_ij - H_ij X_i is formed explicitly (a second pass over a
 * shared-memory copy of the bin tile), so an exact fit gives a loss of
 * rounding size relative to the residual, not to the data.
 * Errors: INVALID_ARG (null w/Y/loss/ws, eps < 0, small ws,
 * misaligned Y), SHAPE (m > PACT_MAX_CHANNELS, P odd or out of range, n_t too
 * large for shared memory).  Every device-side wait of the pass is bounded
 * (pact_set_wait_limit_ns, default 200 ms); a wait that gives up (never
 * expected) makes the loss and dL_dw NaN and sets the status word that
 * pact_mc_deconv_status reads, instead of hanging.  No CTA of the pass ever
 * waits for another CTA (so the result does not depend on how many of its
 * CTAs are resident at once); dL_dw is cleared by a memset before the
 * kernel.
 */
pact_status pact_mc_deconv_loss(const pact_geometry* g, const pact_patches* pt, const float* w,
                                const float* Y, const float* d, int m, float eps, float* loss,
                                float* loss_pp, float* Xhat, float* dL_dw, void* ws,
                                size_t ws_bytes, void* stream);

/*
 * Standalone adjoint of pact_mc_deconv_loss: dL_dw (+)= dL_dloss * dL/dw,
 * dL_dloss a DEVICE float scalar (NULL = 1).  Same workspace rules.
 */
pact_status pact_mc_deconv_loss_adj(const pact_geometry* g, const pact_patches* pt, const float* w,
                                    const float* Y, const float* d, int m, float eps,
                                    const float* dL_dloss, float* dL_dw, int accumulate, void* ws,
                                    size_t ws_bytes, void* stream);

/*
 * Prebuilt tables for repeated pact_mc_deconv_loss calls.  Everything in the
 * fused pass that depends only on the geometry, the patch centres and the
 * delays -- the ring coordinates of the directions ang k and ang k + pi for
 * every (patch, bin) (the lookups of Eq. 4), exp(j|k|d_j) per (channel, bin),
 * and the per-bin sums C2 = sum_j exp(2j|k|d_j) in FP32 and FP64 -- is built
 * once by pact_mc_deconv_tables; a recovery loop (Sec. 3.3) keeps them for
 * every iteration, where pact_mc_deconv_loss rebuilds them per call.
 *   tables   DEVICE, 256-byte aligned, pact_mc_deconv_tables_size bytes,
 *            owned by the caller, written by pact_mc_deconv_tables.
 * pact_mc_deconv_loss_tabled takes the arguments of pact_mc_deconv_loss plus
 * the tables, and a workspace of pact_mc_deconv_loss_tabled_workspace_size
 * bytes (the per-call scratch only); loss or dL_dw may be NULL (not both).
 * With accumulate = 1 the gradient is added to dL_dw (no clearing launch):
 * a recovery iteration clears dL_dw in its pact_sos_to_delays_clear call
 * and accumulates here; with 0 dL_dw is cleared first (a memset).
 * The tables carry a fingerprint of (geometry, N, P, centres pointer, m, d);
 * a call whose arguments do not match it writes NaN to loss and dL_dw.  They
 * also hold the CTA-done ticket of the streaming kernel, which every call
 * leaves at zero: calls that share one table set must be ordered (one stream),
 * and after a call that reported a timeout the tables must be rebuilt.
 * Errors as pact_mc_deconv_loss, plus INVALID_ARG for NULL, misaligned or
 * small tables.
 */
size_t pact_mc_deconv_tables_size(const pact_geometry* g, const pact_patches* pt, int m);
size_t pact_mc_deconv_loss_tabled_workspace_size(const pact_geometry* g, const pact_patches* pt, int m);
pact_status pact_mc_deconv_tables(const pact_geometry* g, const pact_patches* pt, const float* d, int m,
                                  void* tables, size_t tables_bytes, void* stream);
pact_status pact_mc_deconv_loss_tabled(const pact_geometry* g, const pact_patches* pt, const float* w,
                                       const float* Y, const float* d, int m, float eps, const void* tables,
                                       size_t tables_bytes, float* loss, float* loss_pp, float* Xhat,
                                       float* dL_dw, int accumulate, void* ws, size_t ws_bytes, void* stream);

/*
 * Failure detection of the fused pass (no counterpart in the paper).
 * pact_mc_deconv_status reads and clears the status word of one table block:
 * pass the prebuilt tables (tables != NULL, ws = NULL) or the workspace of a
 * pact_mc_deconv_loss / _adj call (ws != NULL, tables = NULL; its tables are
 * rebuilt, and the word cleared, by every such call).  It synchronises the
 * stream and returns PACT_ERR_TIMEOUT if a wait of a call since the last
 * read gave up (that call's loss and dL_dw are then NaN), else PACT_OK.
 * pact_mc_deconv_inject_stall is a test hook: it sets a flag in the prebuilt
 * tables (ws must be NULL) that makes the next streaming call's consumer
 * warps withhold the release of their first pipeline stage, a release that
 * then never comes, so the producer's wait for it runs into the wait limit,
 * the consumers' wait for the next stage does too, and the call reports
 * PACT_ERR_TIMEOUT through the status word with NaN outputs.  Every bulk
 * copy the kernel issued has completed by then; nothing faults or hangs.
 * The launch clears the flag, so the call after it runs normally.
 *   g, pt, m  the problem the tables were built for (layout only)
 */
pact_status pact_mc_deconv_status(const pact_geometry* g, const pact_patches* pt, int m, void* tables,
                                  void* ws, void* stream);
pact_status pact_mc_deconv_inject_stall(const pact_geometry* g, const pact_patches* pt, int m, void* tables,
                                        void* ws, void* stream);

/*
 * Bound on every device-side wait of the kernels launched after this call
 * (fused pass, neural-field and CNN kernels), in ns: 0 restores the default
 * (200 ms), otherwise 1e5 <= ns <= 1e10 (INVALID_ARG outside).  Process-wide;
 * a launch captured into a CUDA graph keeps the limit it saw at capture.
 */
pact_status pact_set_wait_limit_ns(unsigned long long ns);
unsigned long long pact_get_wait_limit_ns(void);

/*
 * pact_mc_deconv_loss without a workspace argument.  The paper has no
 * counterpart: this is a library-usage variant of pact_mc_deconv_loss with
 * identical arithmetic and outputs.
 *
 * Some callers cannot allocate device memory: a plug-in whose host
 * application owns every device buffer and forbids cudaMalloc, or a
 * real-time acquisition loop that must not allocate (allocation can block
 * or fail mid-scan).  This entry point allocates nothing; its scratch space
 * is a fixed device array of PACT_NOALLOC_SCRATCH_BYTES inside the library,
 * held by every GPU that loads the library until the process exits.  The
 * caller still passes all inputs and outputs.
 *   - Problems whose scratch need (pact_mc_deconv_loss_workspace_size)
 *     exceeds PACT_NOALLOC_SCRATCH_BYTES are rejected with PACT_ERR_SHAPE
 *     and a message giving both sizes; nothing is launched.
 *   - The first call on each device looks up the device address of the
 *     array (with that device current) and caches it; make that first call
 *     before any stream capture.  A call that reports PACT_ERR_CUDA drops
 *     the cached address, so after cudaDeviceReset (which unloads the
 *     array with the module) the first call may fail once and the next
 *     looks the address up again.
 *   - Every call on a device shares the one array and it keeps the last
 *     call's contents; the kernels overwrite every scratch entry they read,
 *     so no clearing is needed.  Calls that overlap on the GPU (different
 *     streams, or several host threads) race on the array: issue them in
 *     order on one stream.
 * Arguments, layouts and errors are those of pact_mc_deconv_loss.
 */
#define PACT_NOALLOC_SCRATCH_BYTES (16u << 20)   /* 16 MiB */
pact_status pact_mc_deconv_loss_noalloc(const pact_geometry* g, const pact_patches* pt, const float* w,
                                        const float* Y, const float* d, int m, float eps, float* loss,
                                        float* loss_pp, float* Xhat, float* dL_dw, void* stream);

/*
 * Total variation regulariser of Eq. 7 on the pixel-grid SOS:
 *   TV(v) = sum |v[p+1][q] - v[p][q]| + |v[p][q+1] - v[p][q]|
 *   value    DEVICE float [1] or NULL: value (+)= lambda * TV(v)
 *   dL_dsos  DEVICE float [G][G] or NULL: (+)= lambda * subgradient
 *            (sign(0) = 0)
 * `accumulate` applies to both outputs.  The value is summed per CTA and
 * added with one atomic per CTA (summation order not fixed).
 */
pact_status pact_tv(const pact_geometry* g, const float* sos, float lambda, float* value,
                    float* dL_dsos, int accumulate, void* stream);

/*
 * One Adam step (Kingma & Ba; Sec. 3.3 trains the SOS parameters with
 * Adam) on n parameters, bias-corrected with step count t:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   param -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * Entries whose mask byte is 0 are left unchanged (mask NULL = all train).
 *   param, m, v   DEVICE float [n] (updated in place);  grad DEVICE float [n]
 *   step          t >= 1, used when step_counter is NULL
 *   step_counter  DEVICE int [2] or NULL: [0] = steps taken so far, [1] =
 *                 the kernel's completion count, 0 between calls (zero both
 *                 before the first call).  The update uses t = [0] + 1 and
 *                 the kernel then increments [0] itself (so a call captured
 *                 in a CUDA graph advances on every replay).
 */
pact_status pact_adam_step(int n, float* param, const float* grad, float* m, float* v, int step,
                           int* step_counter, float lr, float beta1, float beta2, float eps,
                           const unsigned char* mask, void* stream);

/*
 * Neural-field SOS (Sec. 3.3: the SOS as a coordinate-based network; here a
 * Fourier-feature MLP on BF16 tensor cores with FP32 accumulation).  For
 * every SOS node (row-major over the G x G grid) with position (x, y) over
 * the field of view G sos_dx:
 *   f = [sin 2 pi f_l x, cos 2 pi f_l x, sin 2 pi f_l y, cos 2 pi f_l y]_{l<16},
 *       f_l = 64^(l/15) cycles per field of view                      (64)
 *   h_l = relu(W_l h_{l-1} + b_l), l = 1..4, width 128
 *   v = v_mid + v_half tanh(w5 . h_4 + b5) inside the mask, v_bg outside.
 * Parameters are one FP32 vector in the order W1[128][64], b1[128],
 * W2[128][128], b2, W3, b3, W4, b4, w5[128], b5[1] (pact_nf_param_count()
 * entries, 16-byte aligned); weights and activations are rounded to BF16.
 *   mask  DEVICE uint8 [G][G] or NULL (all nodes trainable)
 *   sos   DEVICE float [G][G] output
 *   ws    DEVICE workspace (pact_nf_workspace_size), which also carries the
 *         activations from pact_nf_forward to the next pact_nf_backward
 * pact_nf_backward: dL_dparams (+)= (dL/dsos) d sos / d params for the
 * parameters of the last forward call on this workspace.
 * A tensor-core completion wait that gives up (never expected) poisons the
 * outputs with NaN and sets a status word that pact_nf_status reports
 * (PACT_ERR_TIMEOUT); pact_nf_status synchronises the stream.
 */
int pact_nf_param_count(void);
size_t pact_nf_workspace_size(const pact_geometry* g);
pact_status pact_nf_forward(const pact_geometry* g, const float* params, const unsigned char* mask, float v_mid,
                            float v_half, float* sos, void* ws, size_t ws_bytes, void* stream);
pact_status pact_nf_backward(const pact_geometry* g, const float* params, const unsigned char* mask, float v_mid,
                             float v_half, const float* dL_dsos, float* dL_dparams, int accumulate, void* ws,
                             size_t ws_bytes, void* stream);
pact_status pact_nf_status(const pact_geometry* g, const void* ws, size_t ws_bytes, int* host_status,
                           void* stream);

/*
 * The paper's neural field (Sec. 3.3): a SIREN without hidden layers, 256
 * sine features of the node coordinates and a linear output, plus an output
 * scale and offset -- 1027 parameters:
 *   v(x) = offset + scale (sum_f w2_f sin(omega0 (W1_f . x + b1_f)) + b2)
 * on the mask (v_bg outside), x = ((col - (G-1)/2), (row - (G-1)/2)) / ((G-1)/2).
 * Parameters (FP32, flat): W1 [256][2], b1 [256], w2 [256], b2, scale, offset.
 * FP32 on the CUDA cores (two inputs: no contraction worth a tensor core).
 *   params    DEVICE float [1027];  mask DEVICE uint8 [G][G] or NULL
 *   sos       DEVICE float [G][G] output of pact_siren_forward
 *   dL_dsos   DEVICE float [G][G];  dL_dparams DEVICE float [1027] (accumulate = 1 adds)
 *   ws        DEVICE workspace of pact_siren_workspace_size bytes; it carries the
 *             network output from forward to backward, so pact_siren_backward must
 *             follow a pact_siren_forward with the same arguments and workspace.
 * The backward pass is deterministic (per-chunk partial sums, fixed-order reduction).
 */
int pact_siren_param_count(void);
size_t pact_siren_workspace_size(const pact_geometry* g);
pact_status pact_siren_forward(const pact_geometry* g, const float* params, const unsigned char* mask, float omega0,
                               float* sos, void* ws, size_t ws_bytes, void* stream);
pact_status pact_siren_backward(const pact_geometry* g, const float* params, const unsigned char* mask, float omega0,
                                const float* dL_dsos, float* dL_dparams, int accumulate, void* ws, size_t ws_bytes,
                                void* stream);

/* Workspace bytes of pact_stitch. */
size_t pact_stitch_workspace_size(const pact_geometry* g, const pact_patches* pt);

/*
 * Stitching (Sec. S1.5): every deconvolved patch irfft2(Xhat_i) (orthonormal
 * inverse of the half-spectrum, window already applied at cropping) is
 * translated to its centre and summed; the sum is divided by the summed
 * Gaussian windows (0 where no window reaches).  The sums run in FP64 (the
 * workspace holds FP64 images), where the few FP32 terms of a pixel add
 * exactly: the image is the same in every run.
 *   Xhat   DEVICE c64 [N][P][P/2+1];  image DEVICE float [H][W] output
 */
pact_status pact_stitch(const pact_geometry* g, const pact_patches* pt, const float* Xhat,
                        float* image, void* ws, size_t ws_bytes, void* stream);

/*
 * pact_stitch for every channel of a patch-spectrum set at once: the delay
 * stack of the forward model (Eq. 5) in the image domain,
 *   stack[j] = stitch of the patches Y[:, j]   (Sec. S1.5, window once at crop).
 *   Y      DEVICE c64 [N][m][P][P/2+1];  stack DEVICE float [m][H][W] output
 *   ws     DEVICE workspace of pact_stitch_channels_workspace_size bytes
 */
size_t pact_stitch_channels_workspace_size(const pact_geometry* g, const pact_patches* pt, int m);
pact_status pact_stitch_channels(const pact_geometry* g, const pact_patches* pt, int m, const float* Y,
                                 float* stack, void* ws, size_t ws_bytes, void* stream);

/*
 * Warm-start CNN.  The paper has no counterpart: it recovers the SOS by
 * test-time optimisation alone (Sec. 3.3).  This learned initialiser maps a
 * delay stack (Eq. 1 / Eq. 5, the "focal stack" of Sec. 3.2) to an SOS map
 * from which that optimisation starts; it is trained on stacks that the
 * forward model of this library generates from random SOS fields, and the
 * plain optimisation refines its output.  BF16 tensor-core arithmetic with
 * FP32 accumulation; activations are stored in BF16.
 *
 * Geometry: a square image of 4 G pixels per side, G (the SOS grid) a
 * multiple of 8.  Network, with R = G and Cp = 16, 32 or 64 (the stack's m
 * channels zero-padded):
 *   x  = 4x4 block means of the stack / their root-mean-square   [R][R][Cp] BF16
 *   five 3x3 convolutions with ReLU (zero padding): Cp->32 at R, 2x2 mean,
 *   32->64 at R/2, 2x2 mean, then three 64->64 at R/4;
 *   z  = w6 . h5 + b6;  v = v_mid + v_half tanh(z) on the R/4 grid;
 *   sos = bilinear x4 upsampling of v (sample (q + 0.5)/4 - 0.5, clamped),
 *         v_bg outside the mask                                   [G][G]
 * Parameters (FP32, flat, in this order): W_l [c_out][c_in][3][3], b_l [c_out]
 * for l = 1..5 (c_in of W1 is m), then w6 [64], b6 [1];
 * pact_cnn_param_count(m) gives the total.
 *
 *   pact_cnn_pool_stack   stack DEVICE float [m][4G][4G] -> x DEVICE BF16
 *                         [G][G][Cp] (16-byte aligned), workspace of
 *                         pact_cnn_pool_workspace_size bytes.
 *   pact_cnn_forward      x DEVICE BF16 [batch][G][G][Cp] -> sos DEVICE float
 *                         [batch][G][G]; mask DEVICE uint8 [G][G] or NULL.
 *                         Keeps the activations in the workspace
 *                         (pact_cnn_workspace_size(g, m, batch) bytes, 256-byte
 *                         aligned) for pact_cnn_backward.
 *   pact_cnn_backward     dL_dsos DEVICE float [batch][G][G] -> dL_dparams
 *                         (accumulate = 1 adds); must follow pact_cnn_forward
 *                         with the same g, m, batch, params, x, mask and
 *                         workspace.
 *   pact_cnn_mse          training loss mean over samples and mask nodes of
 *                         ((sos - sos_true) / scale)^2 into loss DEVICE [1] and
 *                         its gradient into dL_dsos (NULL to skip); mask_count
 *                         = nonzero mask entries (G^2 when mask is NULL);
 *                         scratch DEVICE float [batch].
 *   pact_cnn_status       reads the workspace status word (synchronises the
 *                         stream): PACT_ERR_TIMEOUT if a tensor-core
 *                         completion wait gave up (the outputs are then NaN).
 * Errors: SHAPE for an unsupported geometry or m, INVALID_ARG for null or
 * misaligned pointers and small workspaces.
 */
int pact_cnn_param_count(int m);
int pact_cnn_input_channels(int m);
size_t pact_cnn_pool_workspace_size(const pact_geometry* g, int m);
pact_status pact_cnn_pool_stack(const pact_geometry* g, const float* stack, int m, void* x, void* ws,
                                size_t ws_bytes, void* stream);
size_t pact_cnn_workspace_size(const pact_geometry* g, int m, int batch);
pact_status pact_cnn_forward(const pact_geometry* g, int m, int batch, const float* params, const void* x,
                             const unsigned char* mask, float v_mid, float v_half, float* sos, void* ws,
                             size_t ws_bytes, void* stream);
pact_status pact_cnn_backward(const pact_geometry* g, int m, int batch, const float* params, const void* x,
                              const unsigned char* mask, float v_half, const float* dL_dsos, float* dL_dparams,
                              int accumulate, void* ws, size_t ws_bytes, void* stream);
pact_status pact_cnn_mse(const pact_geometry* g, int batch, const float* sos, const float* sos_true,
                         const unsigned char* mask, int mask_count, float scale, float* loss, float* dL_dsos,
                         float* scratch, void* stream);
pact_status pact_cnn_status(const pact_geometry* g, int m, int batch, const void* ws, size_t ws_bytes,
                            int* host_status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PACT_H */
