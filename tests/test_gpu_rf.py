"""Synthetic ring channel data on the GPU (pact_rf_synth) vs the FP64 oracle,
and the channel-data end of the 1024 x 1024 / 1024-element workload: channel
data -> DAS (Eq. 1) in closed form.

Tolerance: relative L2 1e-4 on the channel data (the arrival times carry the
FP32 wavefront error of Eq. 3, ~1e-7 of w, i.e. well below 1e-4 of a pulse
width; path lengths and sample positions are formed in FP64)."""
import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from oracle import rf_oracle as R
from paper_2409_10876_gb300 import inputs, pact

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _tiny():
    return inputs.config_tiny(p=16, m=2, n_t=64)


@pytest.mark.parametrize("spread,ring_dr", [(0.0, 0.0), (0.5, 0.2e-3)])
def test_rf_synth_matches_oracle(spread, ring_dr):
    cfg = _tiny()
    case = inputs.make_case(cfg, 11)
    pb = pact.Problem(cfg, DEV)
    fs, t0, n_s, sig = cfg.rf_fs, 1e-6, 520, cfg.rf_sigma
    rf = pact.rf_synth(pb, torch.as_tensor(case["ip"], device=DEV), torch.as_tensor(case["sos_true"], device=DEV),
                       fs, t0, n_s, sig, spread, ring_dr).cpu().numpy()
    ref = R.rf_synth(O.geom(cfg), case["ip"], case["sos_true"], fs, t0, n_s, sig, spread, ring_dr).numpy()
    assert np.abs(ref).max() > 1.0
    assert rel(rf, ref) <= 1e-4


def test_rf_synth_passes_and_empty_image():
    cfg = _tiny()
    case = inputs.make_case(cfg, 12)
    pb = pact.Problem(cfg, DEV)
    p0 = torch.as_tensor(case["ip"], device=DEV)
    sos = torch.as_tensor(case["sos_true"], device=DEV)
    args = (cfg.rf_fs, 1e-6, 520, cfg.rf_sigma)
    one = pact.rf_synth(pb, p0, sos, *args).cpu().numpy()
    many = pact.rf_synth(pb, p0, sos, *args, pixels_per_pass=97).cpu().numpy()     # 43 passes, ragged last
    assert rel(many, one) <= 1e-6
    # overwrites, and an image without sources gives silence
    rf = torch.full((cfg.n_t, 520), 7.0, device=DEV)
    pact.rf_synth(pb, torch.zeros_like(p0), sos, *args, rf=rf)
    assert float(rf.abs().max()) == 0.0


def test_rf_synth_record_edges():
    """Arrivals near and beyond both ends of the record: only the samples
    inside [0, n_s) are written, exactly as the oracle's full-length pulse."""
    cfg = _tiny()
    pb = pact.Problem(cfg, DEV)
    sos = np.full((cfg.sos_g, cfg.sos_g), cfg.v0, np.float32)
    p0 = np.zeros((cfg.img_h, cfg.img_w), np.float32)
    p0[3, 5], p0[40, 60], p0[63, 0] = 1.0, -0.7, 0.4
    fs, sig = cfg.rf_fs, cfg.rf_sigma
    for t0, n_s in [(6.5e-6, 40), (1e-6, 170), (12.5e-6, 3)]:
        rf = pact.rf_synth(pb, torch.as_tensor(p0, device=DEV), torch.as_tensor(sos, device=DEV),
                           fs, t0, n_s, sig).cpu().numpy()
        ref = R.rf_synth(O.geom(cfg), p0, sos, fs, t0, n_s, sig).numpy()
        assert np.abs(rf - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-3)


def test_rf_synth_full_size_sampled():
    """1024 transducers x 4096 samples at 40 MHz through a 256 x 256 SOS map:
    the launch the end-to-end workload runs, checked on sampled transducers
    for a sparse source image (the channel data are linear in p0)."""
    cfg = inputs.config_rf()
    case = inputs.make_case(cfg.replace(m=1), 5)
    pb = pact.Problem(cfg, DEV)
    rng = np.random.default_rng(9)
    p0 = np.zeros((cfg.img_h, cfg.img_w), np.float32)
    idx = rng.choice(cfg.img_h * cfg.img_w, 300, replace=False)
    p0.ravel()[idx] = rng.uniform(0.2, 1.0, idx.size)
    rf = pact.rf_synth(pb, torch.as_tensor(p0, device=DEV), torch.as_tensor(case["sos_true"], device=DEV),
                       cfg.rf_fs, cfg.rf_t0, cfg.rf_ns, cfg.rf_sigma).cpu().numpy()
    ch = [0, 1, 255, 256, 511, 640, 1000, 1023]
    ref = R.rf_synth(O.geom(cfg), p0, case["sos_true"], cfg.rf_fs, cfg.rf_t0, cfg.rf_ns, cfg.rf_sigma,
                     channels=ch).numpy()
    assert rel(rf[ch], ref) <= 1e-4


def test_rf_to_das_centred_source_closed_form():
    """Channel data of one source near the centre of a constant-SOS disk, then
    Eq. 1 at that pixel: y(d) = sum_n psi((w_n - d)/v0) with w_n = (1 - v0/c)
    times the chord from the source to the disk edge toward transducer n
    (closed form), on the 1024 x 1024 / 1024-element geometry."""
    c = 1560.0
    cfg = inputs.config_rf()
    pb = pact.Problem(cfg, DEV)
    src = (512, 512)
    p0 = torch.zeros((cfg.img_h, cfg.img_w), device=DEV)
    p0[src] = 1.0
    sos = torch.full((cfg.sos_g, cfg.sos_g), c, device=DEV)
    fs, t0, n_s, sig = 1e9, 25e-6, 4096, cfg.rf_sigma
    rf = pact.rf_synth(pb, p0, sos, fs, t0, n_s, sig)
    w0 = (1 - cfg.v0 / c) * cfg.mask_radius
    d = np.array([w0 - 2 * sig * cfg.v0, w0 - sig * cfg.v0, w0, w0 + 0.5 * sig * cfg.v0, w0 + sig * cfg.v0],
                 np.float32)
    st = pact.das_stack(pb, rf, fs, t0, d)[:, src[0], src[1]].cpu().numpy()
    a = 2 * np.pi * np.arange(cfg.n_t) / cfg.n_t + cfg.ring_phase
    rn = cfg.ring_radius * np.stack([np.cos(a), np.sin(a)], 1)
    x = np.array([(src[1] - (cfg.img_w - 1) / 2) * cfg.dx, (src[0] - (cfg.img_h - 1) / 2) * cfg.dx])
    e = rn - x
    u = e / np.linalg.norm(e, axis=1, keepdims=True)
    b = u @ x
    chord = -b + np.sqrt(b * b - (x @ x - cfg.mask_radius ** 2))
    wn = (1 - cfg.v0 / c) * chord
    uu = (wn[None, :] - d[:, None].astype(np.float64)) / cfg.v0 / sig
    ref = ((1.0 - uu * uu) * np.exp(-0.5 * uu * uu)).sum(1)
    assert np.abs(st - ref).max() <= 2e-3 * cfg.n_t


@pytest.mark.parametrize("n_t,n_s,fc,bw", [(12, 1000, 5e6, 0.6), (3, 20, 8e6, 0.3), (1024, 4096, 4e6, 1.0)])
def test_rf_bandpass_matches_oracle(n_t, n_s, fc, bw):
    """pact_rf_bandpass against the FP64 oracle: random channel data, the
    channel-data size (8 channels compared), and a record shorter than the
    filter (n_s = 20 < 2K + 1)."""
    from oracle import rf_oracle as R
    fs = 40e6
    rng = np.random.default_rng(n_t + n_s)
    x = rng.standard_normal((n_t, n_s)).astype(np.float32)
    y = pact.rf_bandpass(torch.as_tensor(x, device="cuda"), fs, fc, bw).cpu().numpy()
    rows = np.arange(n_t) if n_t <= 16 else rng.choice(n_t, 8, replace=False)
    ref = R.rf_bandpass(torch.as_tensor(x[rows].astype(np.float64)), fs, fc, bw).numpy()
    err = np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


def test_rf_bandpass_rejects_bad_arguments():
    x = torch.zeros((4, 64), device="cuda")
    for args in ((40e6, 25e6, 0.5), (40e6, 5e6, 0.0), (40e6, 5e6, 3.0), (0.0, 5e6, 0.5), (40e6, 1e3, 0.01)):
        with pytest.raises(pact.PactError):
            pact.rf_bandpass(x, *args)
    with pytest.raises(pact.PactError):
        pact.rf_bandpass(x, 40e6, 5e6, 0.5, out=x)
