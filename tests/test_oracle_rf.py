"""Pins of the FP64 channel-data oracle (the input of Eq. 1) against closed
forms that do not come from the oracle: the pulse's extremes and spectrum
(numpy FFT), straight-line times of flight in uniform media, chord lengths of
a constant-SOS disk, the spreading and ring-offset factors, linearity, and the
DAS value at a source whose wavefront error is the same for all transducers."""
import math

import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from oracle import rf_oracle as R
from paper_2409_10876_gb300 import inputs


def _tiny(**kw):
    return inputs.config_tiny(p=16, m=2).replace(img_h=33, img_w=33, dx=0.2e-3, n_t=24, **kw)


def _ring(cfg, radius=None):
    a = 2 * np.pi * np.arange(cfg.n_t) / cfg.n_t + cfg.ring_phase
    r = cfg.ring_radius if radius is None else radius
    return np.stack([r * np.cos(a), r * np.sin(a)], 1)


def _pix(cfg, row, col):
    return np.array([(col - (cfg.img_w - 1) / 2) * cfg.dx, (row - (cfg.img_h - 1) / 2) * cfg.dx])


def _psi(t, sigma):
    u = t / sigma
    return (1.0 - u * u) * np.exp(-0.5 * u * u)


def test_pulse_shape_and_spectrum():
    """psi = -2 dp/dt (Sec. S1.1) of the N-shaped pressure pulse
    p(t) = -sigma t exp(-t^2/(2 sigma^2)) / 2 (compression, then rarefaction),
    by central differences of p;
    psi is even with psi(0) = 1 and minima -2 exp(-3/2) at +-sqrt(3) sigma; its
    amplitude spectrum (numpy's FFT) peaks at 1 / (sqrt(2) pi sigma)."""
    sig = inputs.config_rf().rf_sigma
    t = np.linspace(-6 * sig, 6 * sig, 120001)
    dt = t[1] - t[0]
    p = lambda tt: -sig * tt * np.exp(-tt * tt / (2 * sig * sig)) / 2
    psi_fd = -2 * (p(t + dt) - p(t - dt)) / (2 * dt) / sig          # psi is scaled by 1/sigma
    y = R.pulse(t, sig).numpy()
    assert np.abs(y - psi_fd).max() < 1e-6
    assert np.array_equal(R.pulse(-t, sig).numpy(), y)
    assert float(R.pulse(0.0, sig)) == 1.0
    assert abs(t[np.argmin(y)] ** 2 - 3 * sig * sig) < 4 * sig * dt
    assert y.min() == pytest.approx(-2 * np.exp(-1.5), rel=1e-8)
    ds = sig / 200
    tt = (np.arange(1 << 18) - (1 << 17)) * ds
    spec = np.abs(np.fft.rfft(R.pulse(tt, sig).numpy()))
    f = np.fft.rfftfreq(tt.size, ds)
    assert abs(f[np.argmax(spec)] - 1 / (np.sqrt(2) * np.pi * sig)) <= f[1]
    for level in (0.5, 0.1):
        lo, hi = R.pulse_band(sig, level)
        above = f[spec >= level * spec.max()]
        assert abs(above.min() - lo) <= 2 * f[1] and abs(above.max() - hi) <= 2 * f[1]
    lo, hi = R.pulse_band(sig, 0.5)
    assert 1.8e6 < lo < 2.0e6 and 6.4e6 < hi < 6.7e6
    lo, hi = R.pulse_band(sig, 0.1)
    assert 0.7e6 < lo < 0.9e6 and 8.7e6 < hi < 9.0e6


def test_uniform_sos_is_straight_line_time_of_flight():
    cfg = _tiny()
    g = O.geom(cfg)
    sos = np.full((cfg.sos_g, cfg.sos_g), cfg.v0)
    p0 = np.zeros((cfg.img_h, cfg.img_w))
    p0[7, 21] = 0.8
    fs, t0, n_s, sig = 100e6, 2e-6, 900, 3e-8
    S = R.rf_synth(g, p0, sos, fs, t0, n_s, sig).numpy()
    L = np.linalg.norm(_ring(cfg) - _pix(cfg, 7, 21)[None], axis=1)
    t = t0 + np.arange(n_s) / fs
    ref = 0.8 * _psi(t[None] - L[:, None] / cfg.v0, sig)
    assert np.abs(S - ref).max() < 1e-12


def test_constant_sos_disk_delays_by_the_chord():
    """v = c inside the mask disk, v_bg = v0 outside: tau = (L - (1 - v0/c) chord)/v0
    with the chord of the segment pixel -> transducer through the disk."""
    c = 1580.0
    cfg = _tiny()
    g = O.geom(cfg)
    sos = np.full((cfg.sos_g, cfg.sos_g), c)
    p0 = np.zeros((cfg.img_h, cfg.img_w))
    p0[3, 2] = 1.0                       # a corner pixel outside the disk: some rays miss it
    p0[20, 14] = -0.5
    fs, t0, n_s, sig = 80e6, 4e-6, 900, 4e-8
    S = R.rf_synth(g, p0, sos, fs, t0, n_s, sig).numpy()
    rn = _ring(cfg)
    t = t0 + np.arange(n_s) / fs
    ref = np.zeros_like(S)
    for (row, col), amp in (((3, 2), 1.0), ((20, 14), -0.5)):
        a = _pix(cfg, row, col)
        for n in range(cfg.n_t):
            e = rn[n] - a
            L = np.linalg.norm(e)
            u = e / L
            b = a @ u
            disc = b * b - (a @ a - cfg.mask_radius ** 2)
            chord = 0.0
            if disc > 0:
                s0, s1 = np.clip([-b - math.sqrt(disc), -b + math.sqrt(disc)], 0.0, L)
                chord = s1 - s0
            tau = (L - (1 - cfg.v0 / c) * chord) / cfg.v0
            ref[n] += amp * _psi(t - tau, sig)
    assert np.abs(S - ref).max() < 1e-9


def test_linear_in_the_source_image():
    cfg = _tiny()
    g = O.geom(cfg)
    case = inputs.make_case(cfg.replace(sos_kind="blobs"), 4)
    rng = np.random.default_rng(3)
    p1 = (rng.uniform(size=(cfg.img_h, cfg.img_w)) < 0.03) * rng.uniform(0.2, 1.0, (cfg.img_h, cfg.img_w))
    p2 = (rng.uniform(size=(cfg.img_h, cfg.img_w)) < 0.03) * rng.uniform(0.2, 1.0, (cfg.img_h, cfg.img_w))
    args = (case["sos_true"], 60e6, 3e-6, 700, 4e-8)
    s1 = R.rf_synth(g, p1, *args)
    s2 = R.rf_synth(g, p2, *args)
    s12 = R.rf_synth(g, 2 * p1 - 0.5 * p2, *args)
    assert float((s12 - (2 * s1 - 0.5 * s2)).abs().max()) < 1e-10 * float(s1.abs().max())


def test_spreading_and_ring_offset():
    cfg = _tiny()
    g = O.geom(cfg)
    sos = np.full((cfg.sos_g, cfg.sos_g), cfg.v0)
    p0 = np.zeros((cfg.img_h, cfg.img_w))
    p0[11, 26] = 1.0
    fs, t0, n_s, sig, dr = 100e6, 2e-6, 1000, 3e-8, 0.3e-3
    S = R.rf_synth(g, p0, sos, fs, t0, n_s, sig, spread=0.5, ring_dr=dr).numpy()
    Rs = cfg.ring_radius + dr
    L = np.linalg.norm(_ring(cfg, Rs) - _pix(cfg, 11, 26)[None], axis=1)
    t = t0 + np.arange(n_s) / fs
    ref = np.sqrt(Rs / L)[:, None] * _psi(t[None] - L[:, None] / cfg.v0, sig)
    assert np.abs(S - ref).max() < 1e-12
    # a channel subset gives those rows of the full record
    sub = R.rf_synth(g, p0, sos, fs, t0, n_s, sig, spread=0.5, ring_dr=dr, channels=[0, 5, 23]).numpy()
    assert np.array_equal(sub, S[[0, 5, 23]])


def test_das_of_a_centred_source_follows_the_pulse():
    """A source at the disk centre in a constant-SOS disk has the same wavefront
    error w = (1 - v0/c) R_mask on every ray, so Eq. 1 at the source gives
    y(d) = N_t psi((w - d)/v0) (up to the linear interpolation of S)."""
    c = 1560.0
    cfg = _tiny()
    g = O.geom(cfg)
    sos = np.full((cfg.sos_g, cfg.sos_g), c)
    p0 = np.zeros((cfg.img_h, cfg.img_w))
    p0[16, 16] = 1.0                     # 33 x 33 image: pixel (16, 16) is the origin
    fs, t0, n_s, sig = 2e9, 4e-6, 14000, 4e-8
    S = R.rf_synth(g, p0, sos, fs, t0, n_s, sig)
    w = (1 - cfg.v0 / c) * cfg.mask_radius
    d = np.array([w - 2 * sig * cfg.v0, w - sig * cfg.v0, w, w + 0.5 * sig * cfg.v0])
    y = R.das_at(g, S, fs, t0, d, torch.tensor([16]), torch.tensor([16])).numpy()[:, 0]
    ref = cfg.n_t * _psi((w - d) / cfg.v0, sig)
    assert np.abs(y - ref).max() < 1e-3 * cfg.n_t


def test_das_at_equals_the_full_stack():
    cfg = _tiny()
    g = O.geom(cfg)
    rng = np.random.default_rng(8)
    rf = rng.standard_normal((cfg.n_t, 300))
    d = np.array([-2e-4, 1e-4])
    full = O.das_stack(g, rf, 40e6, 1e-6, d).numpy()
    rows, cols = np.array([0, 5, 16, 32]), np.array([32, 7, 16, 0])
    part = R.das_at(g, rf, 40e6, 1e-6, d, torch.tensor(rows), torch.tensor(cols)).numpy()
    assert np.abs(part - full[:, rows, cols]).max() < 1e-12


def test_bandpass_taps_closed_forms():
    """The band-limit filter against its definition: an impulse gives the
    taps back, a constant gives their sum, a long cosine at fc keeps its
    amplitude (|H(fc)| = 1 + the image term), and the half-amplitude points
    sit at fc -/+ frac_bw fc / 2 (the Gaussian response)."""
    import math
    fs, fc, bw = 40e6, 5e6, 0.6
    h = R.bandpass_taps(fs, fc, bw).numpy()
    K = (h.size - 1) // 2
    assert np.allclose(h, h[::-1])                                     # zero phase
    n_s = 600
    x = np.zeros((3, n_s))
    x[0, 300] = 1.0
    x[1, :] = 1.0
    q = np.arange(n_s)
    x[2] = np.cos(2 * math.pi * fc * q / fs)
    y = R.rf_bandpass(torch.as_tensor(x), fs, fc, bw).numpy()
    assert np.allclose(y[0, 300 - K:300 + K + 1], h, atol=1e-15) and abs(y[0]).sum() == pytest.approx(abs(h).sum())
    assert np.allclose(y[1, K:n_s - K], h.sum(), atol=1e-12)
    gain = float(R.bandpass_response(fs, fc, bw, [fc])[0])
    assert abs(gain - 1.0) < 1e-3
    assert np.allclose(y[2, K:n_s - K], gain * x[2, K:n_s - K], atol=1e-9)
    lo, hi = R.bandpass_response(fs, fc, bw, [fc * (1 - bw / 2), fc * (1 + bw / 2)]).numpy()
    assert abs(lo - 0.5) < 0.02 and abs(hi - 0.5) < 0.02
    assert float(R.bandpass_response(fs, fc, bw, [0.0])[0]) < 1e-3    # DC rejected
