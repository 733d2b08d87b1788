"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
library routines it does not use (numpy.fft, torch.optim.Adam), closed forms,
exact symmetries, brute force on tiny inputs and central finite differences.
Each test names the definition (paper equation / section) it pins."""
import math

import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs

DT = torch.float64


def _g(cfg):
    return O.geom(cfg)


# ---------------------------------------------------------------- DFT (Sec. S1.5)

@pytest.mark.parametrize("P", [8, 16, 32, 80])
def test_rfft2_matches_numpy(P):
    rng = np.random.default_rng(P)
    x = rng.standard_normal((3, 2, P, P))
    ours = O.rfft2_ortho(torch.tensor(x)).numpy()
    ref = np.fft.rfft2(x, norm="ortho")
    assert np.abs(ours - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("P", [8, 32, 80])
def test_irfft2_matches_numpy(P):
    rng = np.random.default_rng(P + 1)
    X = rng.standard_normal((2, P, P // 2 + 1)) + 1j * rng.standard_normal((2, P, P // 2 + 1))
    ours = O.irfft2_ortho(torch.tensor(X)).numpy()
    ref = np.fft.irfft2(X, s=(P, P), norm="ortho")
    assert np.abs(ours - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_parseval_half_spectrum():
    """Orthonormal DFT: spatial energy equals the c_k-weighted half-spectrum energy."""
    P = 32
    cfg = inputs.config_tiny(p=P)
    x = np.random.default_rng(3).standard_normal((P, P))
    Y = O.rfft2_ortho(torch.tensor(x))
    ck = O.kgrid(_g(cfg))[4]
    assert abs(float((ck * Y.abs() ** 2).sum()) - float((x ** 2).sum())) < 1e-10 * float((x ** 2).sum())


def test_window_fwhm():
    """Gaussian window: 1 at the patch centre, 1/2 at half the FWHM."""
    cfg = inputs.config_tiny(p=32).replace(dx=0.1e-3)
    g = _g(cfg)
    g.window_fwhm = 1.0e-3                      # half width = 5 pixels
    win = O.window(g).numpy()
    c = cfg.p // 2
    assert win[c, c] == 1.0
    for r, q in [(c + 5, c), (c - 5, c), (c, c + 5), (c, c - 5)]:
        assert abs(win[r, q] - 0.5) < 1e-14


# ---------------------------------------------------------------- rays (Eq. 2-3)

def test_uniform_sos_zero_wavefront():
    cfg = inputs.config_small()
    g = _g(cfg)
    sos = np.full((cfg.sos_g, cfg.sos_g), cfg.v0)
    w = O.wavefront_errors(g, sos, cfg.centres())
    assert float(w.abs().max()) == 0.0


def test_constant_sos_chord_closed_form():
    """All nodes at c: w = (1 - v0/c) * (length of the segment inside the mask);
    the chord is measured independently by dense sampling of the segment."""
    cfg = inputs.config_small()
    g = _g(cfg)
    c = 1555.0
    w = O.wavefront_errors(g, np.full((cfg.sos_g, cfg.sos_g), c), cfg.centres()).numpy()
    cen = O.centre_xy(g, cfg.centres()).numpy()
    rn = O.transducers(g).numpy()
    t = (np.arange(200000) + 0.5) / 200000
    for i in [0, 4, 8]:
        for n in [0, 37, 101, 200]:
            p = cen[i][None, :] + t[:, None] * (rn[n] - cen[i])[None, :]
            L = np.linalg.norm(rn[n] - cen[i])
            chord = L * np.mean((p ** 2).sum(1) <= g.mask_radius ** 2)
            assert abs(w[i, n] - (1 - cfg.v0 / c) * chord) < 2e-5 * L * abs(1 - cfg.v0 / c) + 1e-12


def test_linear_sos_matches_log_integral():
    """v = a + b x inside the node hull: along a ray v is affine in arc length,
    int (1 - v0/v) ds = len - (v0/b') ln(v_out/v_in); the midpoint rule is within
    its error bound (len h^2 / 24) max |f''|."""
    cfg = inputs.config_small()
    g = _g(cfg)
    g.mask_radius = 0.8 * (cfg.sos_g - 1) / 2 * cfg.sos_dx      # disk inside the node hull
    G = cfg.sos_g
    xs = (np.arange(G) - (G - 1) / 2) * cfg.sos_dx
    a, b = 1500.0, 4000.0                                     # m/s and m/s per m
    sos = np.tile(a + b * xs[None, :], (G, 1))
    cen = O.centre_xy(g, cfg.centres()).numpy()
    rn = O.transducers(g).numpy()
    w = O.wavefront_errors(g, sos, cfg.centres()).numpy()
    Rm = g.mask_radius
    for i in range(len(cen)):
        for n in range(0, cfg.n_t, 17):
            A, Bp = cen[i], rn[n]
            L = np.linalg.norm(Bp - A)
            e = (Bp - A) / L
            ce = A @ e
            disc = ce * ce - (A @ A - Rm * Rm)
            s0, s1 = max(-ce - math.sqrt(disc), 0.0), min(-ce + math.sqrt(disc), L)
            ap = a + b * A[0]
            bp = b * e[0]
            if abs(bp) < 1e-9:
                exact = (s1 - s0) * (1 - cfg.v0 / ap)
            else:
                exact = (s1 - s0) - cfg.v0 / bp * math.log((ap + bp * s1) / (ap + bp * s0))
            vmin = min(ap + bp * s0, ap + bp * s1)
            f2 = 2 * cfg.v0 * bp * bp / vmin ** 3
            bound = (s1 - s0) * g.ray_step ** 2 / 24 * f2 * 1.01 + 1e-15
            assert abs(w[i, n] - exact) <= bound


def test_rotation_by_90_degrees_shifts_transducers():
    """Rotating the SOS map and the patch centre by +90 deg maps transducer n to
    n + N_t/4 (N_t divisible by 4): w' [n + N_t/4] = w [n].  Pins the axis
    and angle frames of the ray integral."""
    cfg = inputs.config_small()
    g = _g(cfg)
    case = inputs.make_case(cfg, 7)
    sos = case["sos_true"].astype(np.float64)
    G = cfg.sos_g
    # v'(x, y) = v(y, -x): node (p, q) takes node (G-1-q, p)
    rot = np.empty_like(sos)
    for p in range(G):
        for q in range(G):
            rot[p, q] = sos[G - 1 - q, p]
    cen = cfg.centres()
    cen_rot = np.stack([cen[:, 1], cfg.img_w - 1 - cen[:, 0]], 1)     # (a, b) -> (b, W-1-a)
    w = O.wavefront_errors(g, sos, cen).numpy()
    wr = O.wavefront_errors(g, rot, cen_rot).numpy()
    assert np.abs(np.roll(w, cfg.n_t // 4, axis=1) - wr).max() < 1e-13


# ---------------------------------------------------------------- transfer functions (Eq. 4)

def _tiny_tf(p=16, m=4, seed=0):
    cfg = inputs.config_tiny(p=p, m=m)
    g = _g(cfg)
    rng = np.random.default_rng(seed)
    w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng).astype(np.float64)
    return cfg, g, w


def test_tf_zero_wavefront_is_cosine():
    cfg, g, _ = _tiny_tf()
    w = np.zeros((cfg.n_patches, cfg.n_t))
    H = O.transfer_functions(g, w, cfg.centres(), cfg.delays())
    kmag = O.kgrid(g)[2]
    d = torch.tensor(cfg.delays(), dtype=DT)
    ref = torch.cos(kmag[None, None] * d[None, :, None, None]).expand_as(H.real)
    assert float((H - ref.to(H.dtype)).abs().max()) < 1e-14


def test_tf_identity_at_zero_delay():
    cfg, g, _ = _tiny_tf()
    w = np.zeros((cfg.n_patches, cfg.n_t))
    H = O.transfer_functions(g, w, cfg.centres(), np.zeros(3))
    assert float((H - 1).abs().max()) == 0.0


def test_tf_bounds_dc_and_hermitian():
    """|H| <= 1, H(0) = 1, and H(-k) = conj(H(k)) on column k_x = 0 (real PSF)."""
    cfg, g, w = _tiny_tf()
    H = O.transfer_functions(g, w, cfg.centres(), cfg.delays())
    assert float(H.abs().max()) <= 1 + 1e-14
    assert float((H[..., 0, 0] - 1).abs().max()) < 1e-15
    P = cfg.p
    for u in range(1, P // 2):
        assert float((H[..., u, 0] - torch.conj(H[..., P - u, 0])).abs().max()) < 1e-13


def test_first_order_wavefront_is_translation():
    """w(theta) = a cos(theta) + b sin(theta) at d = 0 turns H into the phase ramp
    exp(-j k.(a, b)): the PSF is the point (a, b) (the first-order term shifts
    the PSF).  Exact up to the ring-angle interpolation error."""
    cfg = inputs.config_tiny(p=32, m=1).replace(n_t=1024)
    g = _g(cfg)
    a, b = 3 * cfg.dx, -2 * cfg.dx
    cen = O.centre_xy(g, cfg.centres())
    rn = O.transducers(g)
    th = torch.atan2(rn[None, :, 1] - cen[:, None, 1], rn[None, :, 0] - cen[:, None, 0])
    w = a * torch.cos(th) + b * torch.sin(th)
    H = O.transfer_functions(g, w, cfg.centres(), np.zeros(1))[:, 0]
    kx, ky = O.kgrid(g)[:2]
    ramp = torch.exp(-1j * (kx * a + ky * b).to(torch.complex128))
    assert float((H - ramp[None]).abs().max()) < 2e-3
    h = O.irfft2_ortho(H)
    P = cfg.p
    for i in range(h.shape[0]):
        r, c = np.unravel_index(int(torch.argmax(h[i])), (P, P))
        assert (r, c) == ((-2) % P, 3)


def _point_source_rf(g, src, w_fn, fs, n_s, t0, sig_t):
    """Channel data of a point source whose arrivals carry wavefront error w_n:
    t_n = (|r_s - r_n| - w_n)/v0 (Eq. 3 solved for the time of flight),
    Gaussian pulse of width sig_t."""
    rn = O.transducers(g).numpy()
    e = rn - src[None, :]
    dist = np.linalg.norm(e, axis=1)
    th = np.arctan2(e[:, 1], e[:, 0])
    tn = (dist - w_fn(th)) / g.v0
    t = t0 + np.arange(n_s) / fs
    return np.exp(-((t[None, :] - tn[:, None]) ** 2) / (2 * sig_t ** 2))


def test_das_point_source_shift_matches_tf_sign():
    """Eq. 1 and Eq. 4 agree: DAS of a point source whose arrivals carry
    w = a cos(theta) + b sin(theta) peaks at r_s + (a, b), the same translation
    the transfer function gives (and the opposite of the conjugated form)."""
    cfg = inputs.config_tiny(p=32, m=1).replace(dx=0.1e-3, n_t=256)
    g = _g(cfg)
    src_px = (32, 32)
    sx, sy = (np.array([src_px[1], src_px[0]]) - (cfg.img_w - 1) / 2) * cfg.dx
    a, b = 3 * cfg.dx, -2 * cfg.dx
    fs, n_s, t0 = 100e6, 1400, 0.0
    rf = _point_source_rf(g, np.array([sx, sy]), lambda th: a * np.cos(th) + b * np.sin(th),
                          fs, n_s, t0, sig_t=0.6e-7)
    img = O.das_stack(g, rf, fs, t0, np.zeros(1))[0].numpy()
    r, c = np.unravel_index(int(np.argmax(img)), img.shape)
    assert (r - src_px[0], c - src_px[1]) == (-2, 3)
    # the same shift through the transfer function of the patch centred on r_s
    cen = np.array([src_px])
    rn = O.transducers(g).numpy()
    th = np.arctan2(rn[:, 1] - sy, rn[:, 0] - sx)
    w = (a * np.cos(th) + b * np.sin(th))[None]
    H = O.transfer_functions(g, w, cen, np.zeros(1))[:, 0]
    h = O.irfft2_ortho(H)[0].numpy()
    r2, c2 = np.unravel_index(int(np.argmax(h)), h.shape)
    P = cfg.p
    assert (r2, c2) == ((-2) % P, 3)


def test_das_linear_and_single_sample_arc():
    """Eq. 1 is linear in S, and one nonzero sample q of transducer n lights
    exactly the pixels with |((|r'-r_n| - d)/v0 - t0) fs - q| < 1."""
    cfg = inputs.config_tiny(p=16, m=2).replace(img_h=24, img_w=24, n_t=8)
    g = _g(cfg)
    fs, n_s, t0 = 40e6, 300, 0.0
    rng = np.random.default_rng(5)
    s1 = rng.standard_normal((cfg.n_t, n_s))
    s2 = rng.standard_normal((cfg.n_t, n_s))
    d = np.array([-2e-4, 3e-4])
    y1 = O.das_stack(g, s1, fs, t0, d)
    y2 = O.das_stack(g, s2, fs, t0, d)
    y12 = O.das_stack(g, 2 * s1 - 0.5 * s2, fs, t0, d)
    assert float((y12 - (2 * y1 - 0.5 * y2)).abs().max()) < 1e-12
    q, n = 150, 3
    imp = np.zeros((cfg.n_t, n_s))
    imp[n, q] = 1.0
    y = O.das_stack(g, imp, fs, t0, d).numpy()
    rn = O.transducers(g).numpy()[n]
    for j in range(2):
        for a in range(cfg.img_h):
            for bcol in range(cfg.img_w):
                x = (bcol - (cfg.img_w - 1) / 2) * cfg.dx
                yy = (a - (cfg.img_h - 1) / 2) * cfg.dx
                qq = ((math.hypot(x - rn[0], yy - rn[1]) - d[j]) / cfg.v0 - t0) * fs
                expect = max(0.0, 1.0 - abs(qq - q))
                assert abs(y[j, a, bcol] - expect) < 1e-9


# ---------------------------------------------------------------- deconvolution and loss (Eq. 5-7)

def _spectra_case(p=16, m=4, seed=1):
    cfg, g, w = _tiny_tf(p, m, seed)
    rng = np.random.default_rng(seed + 10)
    X = torch.tensor(rng.standard_normal((cfg.n_patches, p, p // 2 + 1))
                     + 1j * rng.standard_normal((cfg.n_patches, p, p // 2 + 1)))
    H = O.transfer_functions(g, w, cfg.centres(), cfg.delays())
    return cfg, g, w, H, X


def test_noise_free_exact_recovery_eps0():
    """Y = H X exactly and eps = 0: X_hat = X and the data loss vanishes."""
    cfg, g, w, H, X = _spectra_case()
    Y = O.forward_spectra(H, X)
    Xh = O.deconvolve(H, Y, 0.0)
    assert float((Xh - X).abs().max()) < 1e-12 * float(X.abs().max())
    assert float(O.data_loss(g, H, Y, Xh)) < 1e-20 * float((Y.abs() ** 2).sum())


def test_single_channel_zero_loss_eps0():
    """M = 1, eps = 0: plain inverse filter, residual zero wherever H != 0."""
    cfg, g, w, H, X = _spectra_case(m=1)
    rng = np.random.default_rng(9)
    Y = torch.tensor(rng.standard_normal(H.shape) + 1j * rng.standard_normal(H.shape))
    Xh = O.deconvolve(H, Y, 0.0)
    R = Y - H * Xh[:, None]
    assert float(R.abs().max()) < 1e-10 * float(Y.abs().max())


def test_regularised_residual_closed_form():
    """eps > 0, Y = H X: R_j = H_j X eps / (B + eps)."""
    cfg, g, w, H, X = _spectra_case()
    eps = 0.3
    Y = O.forward_spectra(H, X)
    Xh = O.deconvolve(H, Y, eps)
    B = (H.abs() ** 2).sum(1)
    R = Y - H * Xh[:, None]
    ref = H * (X * eps / (B + eps))[:, None]
    assert float((R - ref).abs().max()) < 1e-12 * float(Y.abs().max())


def test_residual_energy_closed_form():
    """sum_j |R_j|^2 = E - |A|^2 (B + 2 eps) / (B + eps)^2 (FP64)."""
    cfg, g, w, H, X = _spectra_case()
    rng = np.random.default_rng(2)
    Y = torch.tensor(rng.standard_normal(H.shape) + 1j * rng.standard_normal(H.shape))
    for eps in [0.0, 1e-3, 0.5]:
        Xh = O.deconvolve(H, Y, eps)
        R = Y - H * Xh[:, None]
        lhs = (R.abs() ** 2).sum(1)
        A = (torch.conj(H) * Y).sum(1)
        B = (H.abs() ** 2).sum(1)
        E = (Y.abs() ** 2).sum(1)
        rhs = E - A.abs() ** 2 * (B + 2 * eps) / (B + eps) ** 2
        assert float((lhs - rhs).abs().max()) < 1e-10 * float(E.max())


@pytest.mark.parametrize("P", [8, 16])
def test_product_is_circular_convolution(P):
    """Eq. 5 <-> the isoplanatic convolution y = h * x: with w = 0 the PSF is
    real and even, and P irfft2(H X) equals the brute-force circular
    convolution of h = irfft2(H) with x (orthonormal DFT on P x P)."""
    cfg = inputs.config_tiny(p=P, m=3)
    g = _g(cfg)
    H = O.transfer_functions(g, np.zeros((cfg.n_patches, cfg.n_t)), cfg.centres(), cfg.delays())[0]
    x = np.random.default_rng(P).standard_normal((P, P))
    X = O.rfft2_ortho(torch.tensor(x))
    for j in range(3):
        h = O.irfft2_ortho(H[j]).numpy()
        y = O.irfft2_ortho(H[j] * X).numpy()
        brute = np.zeros((P, P))
        for a in range(P):
            for b in range(P):
                s = 0.0
                for a2 in range(P):
                    for b2 in range(P):
                        s += h[a2, b2] * x[(a - a2) % P, (b - b2) % P]
                brute[a, b] = s
        assert np.abs(P * y - brute).max() < 1e-10 * max(1.0, np.abs(brute).max())


def test_product_is_circular_convolution_scale():
    """Scale of the orthonormal DFT: a unit delta has the flat spectrum 1/P,
    and multiplying by it returns x / P."""
    P = 8
    h = np.zeros((P, P))
    h[0, 0] = 1.0                                 # delta at the origin
    x = np.random.default_rng(1).standard_normal((P, P))
    Hh = O.rfft2_ortho(torch.tensor(h))           # = 1/P everywhere
    assert float((Hh - 1.0 / P).abs().max()) < 1e-15
    y = O.irfft2_ortho(Hh * O.rfft2_ortho(torch.tensor(x))).numpy()
    assert np.abs(P * y - x).max() < 1e-12


# ---------------------------------------------------------------- gradients (Eq. 7, Sec. 3.3)

def test_envelope_identity_and_regularised_adjoint():
    """dL/dconj(H_j) = -w_k conj(X) R_j at eps = 0 and, for eps > 0,
    -(w_k conj(X)/D) ((B + 2 eps) R_j - eps X H_j), checked against central
    finite differences in Re H and Im H (dL/dRe + j dL/dIm = 2 dL/dconj(H))."""
    cfg = inputs.config_tiny(p=8, m=3, grid=1)
    g = _g(cfg)
    rng = np.random.default_rng(4)
    shp = (1, 3, 8, 5)
    H0 = torch.tensor(rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    Y = torch.tensor(rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    kmag, ck = O.kgrid(g)[2], O.kgrid(g)[4]
    om = ck * kmag * 1e-3
    for eps in [0.0, 0.2]:
        def L(H):
            return float(O.data_loss(g, H, Y, O.deconvolve(H, Y, eps)))
        Xh = O.deconvolve(H0, Y, eps)
        R = Y - H0 * Xh[:, None]
        B = (H0.abs() ** 2).sum(1)
        D = B + eps
        G = -(om * torch.conj(Xh) / D)[:, None] * ((B + 2 * eps)[:, None] * R - eps * (Xh[:, None] * H0))
        for (j, u, v) in [(0, 1, 1), (2, 3, 4), (1, 6, 2)]:
            hstep = 1e-6
            e = torch.zeros_like(H0)
            e[0, j, u, v] = hstep
            dre = (L(H0 + e) - L(H0 - e)) / (2 * hstep)
            dim = (L(H0 + 1j * e) - L(H0 - 1j * e)) / (2 * hstep)
            got = complex(2 * G[0, j, u, v])
            assert abs(complex(dre, dim) - got) < 1e-6 * max(1.0, abs(got))


def test_grad_w_matches_finite_differences():
    cfg = inputs.config_tiny(p=16, m=4)
    g = _g(cfg)
    rng = np.random.default_rng(11)
    w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng).astype(np.float64)
    Y = torch.tensor(rng.standard_normal((cfg.n_patches, cfg.m, 16, 9))
                     + 1j * rng.standard_normal((cfg.n_patches, cfg.m, 16, 9)))
    L0, _, _, grad = O.mc_deconv_loss(g, w, Y, cfg.centres(), cfg.delays(), 1e-3)
    for (i, n) in [(0, 3), (1, 20), (3, 50), (2, 63)]:
        h = 1e-8
        wp = w.copy(); wp[i, n] += h
        wm = w.copy(); wm[i, n] -= h
        fd = (float(O.mc_deconv_loss(g, wp, Y, cfg.centres(), cfg.delays(), 1e-3, False)[0])
              - float(O.mc_deconv_loss(g, wm, Y, cfg.centres(), cfg.delays(), 1e-3, False)[0])) / (2 * h)
        assert abs(fd - float(grad[i, n])) < 1e-5 * float(grad.abs().max())


def test_grad_sos_matches_finite_differences():
    cfg = inputs.config_tiny(p=16, m=4)
    g = _g(cfg)
    case = inputs.make_case(cfg, 3)
    rng = np.random.default_rng(12)
    Y = torch.tensor(rng.standard_normal((cfg.n_patches, cfg.m, 16, 9))
                     + 1j * rng.standard_normal((cfg.n_patches, cfg.m, 16, 9)))
    sos = case["sos_true"].astype(np.float64)
    L0, _, _, gs = O.objective(g, sos, Y, cfg.centres(), cfg.delays(), 1e-3, 1e-4)
    G = cfg.sos_g
    for (p, q) in [(7, 7), (4, 9), (10, 3), (8, 12)]:
        h = 1e-3
        sp = sos.copy(); sp[p, q] += h
        sm = sos.copy(); sm[p, q] -= h
        fd = (float(O.objective(g, sp, Y, cfg.centres(), cfg.delays(), 1e-3, 1e-4, False)[0])
              - float(O.objective(g, sm, Y, cfg.centres(), cfg.delays(), 1e-3, 1e-4, False)[0])) / (2 * h)
        assert abs(fd - float(gs[p, q])) < 1e-4 * float(gs.abs().max()) + 1e-9


def test_ray_adjoint_matches_finite_differences():
    cfg = inputs.config_tiny(p=16, m=4)
    g = _g(cfg)
    case = inputs.make_case(cfg, 4)
    sos = case["sos_true"].astype(np.float64)
    r = np.random.default_rng(13).standard_normal((cfg.n_patches, cfg.n_t))
    gs = O.sos_to_delays_adj(g, sos, cfg.centres(), r).numpy()
    for (p, q) in [(7, 8), (3, 3), (12, 5)]:
        h = 1e-2
        sp = sos.copy(); sp[p, q] += h
        sm = sos.copy(); sm[p, q] -= h
        fd = float(((O.wavefront_errors(g, sp, cfg.centres()) - O.wavefront_errors(g, sm, cfg.centres())).numpy() * r).sum()) / (2 * h)
        assert abs(fd - gs[p, q]) < 1e-6 * np.abs(gs).max()


def test_tv_linear_ramp_closed_form():
    """TV of v[p, q] = a p + b q on a G x G grid is G (G-1) (|a| + |b|); its
    subgradient is zero on a constant map (sign(0) = 0)."""
    G = 9
    a, b = 1.5, -0.25
    p, q = np.meshgrid(np.arange(G), np.arange(G), indexing="ij")
    v = torch.tensor(a * p + b * q, dtype=DT)
    assert abs(float(O.tv(v)) - G * (G - 1) * (abs(a) + abs(b))) < 1e-12
    c = torch.full((G, G), 1500.0, dtype=DT, requires_grad=True)
    (gc,) = torch.autograd.grad(O.tv(c), c)
    assert float(gc.abs().max()) == 0.0


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(6)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(6)]
    tp = torch.tensor(p0, dtype=DT, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = torch.tensor(p0), torch.zeros(50, dtype=DT), torch.zeros(50, dtype=DT)
    for t, gr in enumerate(grads, 1):
        opt.zero_grad()
        tp.grad = torch.tensor(gr, dtype=DT)
        opt.step()
        p, m, v = O.adam_step(p, gr, m, v, t, 0.1)
    assert float((p - tp.detach()).abs().max()) < 1e-14


def test_adam_mask_freezes_nodes():
    p0 = np.arange(6.0)
    mask = np.array([1, 0, 1, 0, 1, 1])
    p, m, v = O.adam_step(p0, np.ones(6), np.zeros(6), np.zeros(6), 1, 0.5, mask=mask)
    assert float(p[1]) == 1.0 and float(p[3]) == 3.0 and float(m[1]) == 0.0
    assert abs(float(p[0]) - (0.0 - 0.5)) < 1e-7


# ---------------------------------------------------------------- stitching (Sec. S1.5)

def test_stitch_of_windowed_patches_is_identity():
    """Patches that are the windowed crops of an image stitch back to that image
    wherever a window reaches; windowed all-ones patches give 1."""
    cfg = inputs.config_small()
    g = _g(cfg)
    x = np.random.default_rng(8).standard_normal((cfg.img_h, cfg.img_w))
    X = O.patch_spectra(g, x[None], cfg.centres())[:, 0]
    out = O.stitch(g, X, cfg.centres()).numpy()
    ones = O.stitch(g, O.patch_spectra(g, np.ones((1, cfg.img_h, cfg.img_w)), cfg.centres())[:, 0],
                    cfg.centres()).numpy()
    P = cfg.p
    cov = np.zeros_like(x, dtype=bool)
    for ca, cb in cfg.centres():
        cov[max(ca - P // 2, 0):ca + P // 2, max(cb - P // 2, 0):cb + P // 2] = True
    assert np.abs(out - x)[cov].max() < 1e-10
    assert np.abs(ones - 1)[cov].max() < 1e-12
    assert np.abs(out[~cov]).max() == 0.0


def test_quality_metrics_closed_forms():
    """PSNR/SSIM helpers used for the recovered images: known values."""
    from paper_2409_10876_gb300 import quality
    rng = np.random.default_rng(30)
    ref = rng.uniform(0, 1, (40, 40))
    assert quality.psnr(ref + 0.1, ref) == pytest.approx(20.0, abs=1e-9)        # MSE 0.01
    assert quality.ssim(ref, ref) == pytest.approx(1.0, abs=1e-12)
    assert quality.ssim(0.5 * ref, ref) < 0.95
    noisy = ref + 0.3 * rng.standard_normal(ref.shape)
    assert quality.ssim(noisy, ref) < quality.ssim(ref + 0.05 * rng.standard_normal(ref.shape), ref)
