"""FP64 CPU oracle of the ring channel data that feeds Eq. 1 (synthetic RF).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path never calls it and shares no code with it.

The paper's experiments start from ring channel data S(n, t); DAS (Eq. 1)
turns S into the delay stack.  Its simulated data are the time derivative of
the photoacoustic pressure, S = -2 dp/dt, standing in for the transducer
response (Sec. S1.1).  With the
straight-ray model of Eq. 2-3 the time of flight from an image point r' to
transducer n is

    tau(r', n) = int dl / v = (|r' - r_n| - w(r', n)) / v0,

w the wavefront error of Eq. 3 evaluated on the segment r' -> r_n (same
quadrature, mask and background as ``pact_oracle.wavefront_errors``).
Every pixel p of the initial-pressure image p0 emits one band-limited pulse:

    S(t_q, n) = sum_p p0_p a(p, n) psi(t_q - tau(p, n)),   t_q = t0 + q / fs,

Readings (the paper's data come from a full-wave simulator; here the
pressure at the transducer is the N-shaped pulse of a small absorber, the
time derivative of a Gaussian, and the path is the straight ray of Eq. 2-3):

* psi = -2 dp/dt of p(t) = -sigma t exp(-t^2 / (2 sigma^2)) / 2, i.e. minus the
  second derivative of a Gaussian, scaled to psi(0) = 1:
      psi(t) = (1 - t^2 / sigma^2) exp(-t^2 / (2 sigma^2)).
  It is even, so the DAS image of a point source has the real, even
  spectrum that the transfer functions of Eq. 4 assume (an odd pulse would
  give the two ring directions of Eq. 4 opposite signs).  Its amplitude
  spectrum is proportional to f^2 exp(-2 pi^2 sigma^2 f^2), peaking at
  1 / (sqrt(2) pi sigma); sigma = 1 / (sqrt(2) pi 4 MHz) puts the
  half-amplitude band at 1.9-6.5 MHz and the -20 dB band at 0.8-8.8 MHz.
* a(p, n) = (R_s / |r_p - r_n|)^gamma: gamma = 0 (the default) is the model
  the method assumes; gamma = 1/2 adds cylindrical spreading, a model
  mismatch for robustness studies.
* The transducers may sit on a ring of radius R_s = R + dR (dR = 0 by
  default) while DAS and the method keep R: a ring-radius mismatch.
"""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np
import torch

from . import pact_oracle as O

DT = torch.float64


def pulse(t, sigma: float) -> torch.Tensor:
    """psi(t) = (1 - t^2 / sigma^2) exp(-t^2 / (2 sigma^2))."""
    t = O._t(t)
    u = t / sigma
    return (1.0 - u * u) * torch.exp(-0.5 * u * u)


def synthesis_geometry(g, ring_dr: float = 0.0) -> SimpleNamespace:
    """The geometry with the transducer ring moved to radius R + ring_dr."""
    d = dict(vars(g))
    d["ring_radius"] = g.ring_radius + ring_dr
    return SimpleNamespace(**d)


def time_of_flight(g, sos, rows, cols, channels=None, ring_dr: float = 0.0):
    """tau(p, n) [K, C] in seconds and the path lengths |r_p - r_n| [K, C] for
    pixels (rows[k], cols[k]) and transducers `channels` (all if None), with
    w from the Eq. 3 straight-ray integral to the (possibly moved) ring."""
    gs = synthesis_geometry(g, ring_dr)
    rn = O.transducers(gs)
    if channels is not None:
        rn = rn[torch.as_tensor(np.asarray(channels), dtype=torch.long)]
    x, y = O.pixel_xy(g, rows, cols)
    K, C = x.shape[0], rn.shape[0]
    start = torch.stack([x, y], 1)[:, None, :].expand(K, C, 2).reshape(-1, 2)
    end = rn[None, :, :].expand(K, C, 2).reshape(-1, 2)
    sos = O._t(sos)
    px, py, wgt, outside = O.ray_quadrature(gs, start, end)
    v = O.sos_bilinear(gs, sos, px, py)
    w = (wgt * (1.0 - gs.v0 / v)).sum(1) + outside * (1.0 - gs.v0 / gs.v_bg)
    L = torch.linalg.norm(end - start, dim=1)
    return ((L - w) / gs.v0).reshape(K, C), L.reshape(K, C)


def rf_synth(g, p0, sos, fs: float, t0: float, n_s: int, sigma: float, spread: float = 0.0,
             ring_dr: float = 0.0, channels=None, chunk: int = 8) -> torch.Tensor:
    """S[C][n_s]: channel data of the sources p0 [H][W] for the transducers
    `channels` (all if None); only pixels with p0 != 0 emit."""
    p0 = O._t(p0)
    rows, cols = torch.nonzero(p0 != 0, as_tuple=True)
    n_ch = g.n_t if channels is None else len(channels)
    S = torch.zeros(n_ch, n_s, dtype=DT)
    t = t0 + torch.arange(n_s, dtype=DT) / fs
    Rs = g.ring_radius + ring_dr
    for k0 in range(0, rows.shape[0], chunk):
        r, c = rows[k0:k0 + chunk], cols[k0:k0 + chunk]
        tau, L = time_of_flight(g, sos, r, c, channels, ring_dr)
        amp = p0[r, c][:, None] * (Rs / L) ** spread
        S += (amp[:, :, None] * pulse(t[None, None, :] - tau[:, :, None], sigma)).sum(0)
    return S


def das_at(g, rf, fs: float, t0: float, d, rows, cols) -> torch.Tensor:
    """Eq. 1 at the listed pixels only: y(r'_k; d_j) = sum_n S((|r'_k - r_n| -
    d_j)/v0, n), S linearly interpolated at rate fs from time t0 and zero
    outside the record.  Returns [M, K]."""
    rf = O._t(rf)
    d = O._t(d)
    n_t, n_s = rf.shape
    rn = O.transducers(g)
    x, y = O.pixel_xy(g, rows, cols)
    out = torch.zeros(d.shape[0], x.shape[0], dtype=DT)
    for n in range(n_t):
        dist = torch.sqrt((x - rn[n, 0]) ** 2 + (y - rn[n, 1]) ** 2)
        for j in range(d.shape[0]):
            q = ((dist - d[j]) / g.v0 - t0) * fs
            q0 = torch.floor(q)
            f = q - q0
            i0 = q0.long()
            for k, wk in ((i0, 1.0 - f), (i0 + 1, f)):
                ok = (k >= 0) & (k < n_s)
                out[j] += torch.where(ok, wk * rf[n, k.clamp(0, n_s - 1)], torch.zeros((), dtype=DT))
    return out


# ---------------------------------------------------------------------------
# Transducer band-limit (a model mismatch for robustness studies: the method
# assumes the channel data above; a real transducer also band-passes it).
#
# Reading: the transducer's impulse response is a Gaussian-windowed cosine at
# the centre frequency fc,
#     h(tau) = (2 / Z) exp(-tau^2 / (2 s_t^2)) cos(2 pi fc tau),
# sampled at tau_k = k / fs for |k| <= K = ceil(4 s_t fs), Z = sum_k of the
# window (unit gain at fc up to the image at -fc), zero phase (no shift of
# the times of flight).  Its amplitude response near fc is a Gaussian in f
# whose full width at half amplitude is frac_bw * fc:
#     s_f = frac_bw fc / (2 sqrt(2 ln 2)),   s_t = 1 / (2 pi s_f).
# Every channel is filtered along time, zero outside the record.
# ---------------------------------------------------------------------------

def bandpass_taps(fs: float, fc: float, frac_bw: float) -> torch.Tensor:
    """Taps h_k, k = -K .. K, of the transducer impulse response (see above)."""
    s_f = frac_bw * fc / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    s_t = 1.0 / (2.0 * math.pi * s_f)
    K = int(math.ceil(4.0 * s_t * fs))
    tau = torch.arange(-K, K + 1, dtype=DT) / fs
    env = torch.exp(-0.5 * (tau / s_t) ** 2)
    return 2.0 * env * torch.cos(2.0 * math.pi * fc * tau) / env.sum()


def bandpass_response(fs: float, fc: float, frac_bw: float, f) -> torch.Tensor:
    """|H(f)| of the sampled taps: the magnitude of sum_k h_k exp(-2 pi j f k / fs)."""
    h = bandpass_taps(fs, fc, frac_bw)
    K = (h.numel() - 1) // 2
    k = torch.arange(-K, K + 1, dtype=DT)
    f = O._t(f).reshape(-1, 1)
    ph = 2.0 * math.pi * f * k / fs
    return torch.sqrt((h * torch.cos(ph)).sum(1) ** 2 + (h * torch.sin(ph)).sum(1) ** 2)


def rf_bandpass(rf, fs: float, fc: float, frac_bw: float) -> torch.Tensor:
    """out[n, q] = sum_k h_k rf[n, q - k], zero outside 0 <= q - k < n_s."""
    rf = O._t(rf)
    h = bandpass_taps(fs, fc, frac_bw)
    K = (h.numel() - 1) // 2
    n_t, n_s = rf.shape
    pad = torch.zeros((n_t, n_s + 2 * K), dtype=DT)
    pad[:, K:K + n_s] = rf
    out = torch.zeros((n_t, n_s), dtype=DT)
    for j in range(2 * K + 1):                # tap k = j - K reads rf[q - k] = pad[q - k + K]
        k = j - K
        out += h[j] * pad[:, K - k:K - k + n_s]
    return out


def pulse_band(sigma: float, level: float = 0.5):
    """Frequencies [Hz] where the amplitude spectrum of psi falls to `level`
    of its peak, from the closed form x^2 exp(1 - x^2) = level with
    x = f / f_peak, f_peak = 1 / (sqrt(2) pi sigma)."""
    from scipy.optimize import brentq
    fp = 1.0 / (math.sqrt(2.0) * math.pi * sigma)
    fn = lambda x: x * x * math.exp(1.0 - x * x) - level
    return fp * brentq(fn, 1e-9, 1.0), fp * brentq(fn, 1.0, 50.0)
