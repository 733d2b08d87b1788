"""GPU (libpact, through the C ABI) vs the FP64 oracle, element by element on
the same seeded inputs.

Tolerances (relative L2 unless stated), from the FP32 arithmetic:
  delays w, patches X_hat, loss, spectra, transfer functions: 1e-4
  gradients dL/dw and dL/dsos: 2e-3
  DAS stack: 5e-4 (|r' - r_n| carries ~1 ulp of FP32 at the ring radius,
  i.e. ~1e-4 of a sample for a 40 MHz / 1500 m/s sampling; the parity RF is
  band-limited so the tap error stays below that fraction of the signal)
"""
import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs, pact
from paper_2409_10876_gb300.recovery import McDeconvLoss, PGRecovery, SosToDelays, recover

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a, np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def cpu(t):
    return t.detach().cpu().numpy()


def rand_Y(shape, seed):
    z = np.random.default_rng(seed).standard_normal(shape + (2,)).astype(np.float32)
    return z[..., 0] + 1j * z[..., 1]


def to_dev_c(y):
    return torch.as_tensor(np.ascontiguousarray(y.astype(np.complex64)), device=DEV)


CASES = {
    "tiny_p16_m4": lambda: inputs.config_tiny(p=16, m=4),
    "tiny_p8_m1": lambda: inputs.config_tiny(p=8, m=1),
    "tiny_p12_m3": lambda: inputs.config_tiny(p=12, m=3, grid=3),
    "small_p32_m8": inputs.config_small,
    "tiny_nt48": lambda: inputs.config_tiny(p=16, m=4, n_t=48),     # N_t not a multiple of 32: warp-per-ray kernels
}


# ------------------------------------------------------------------ Eq. 3 and its adjoint

@pytest.mark.parametrize("name", list(CASES) + ["tiny_g200", "tiny_g512"])
def test_sos_to_delays(name):
    cfg = ADJ_CASES[name]() if name in ADJ_CASES else CASES[name]()
    for seed in (0, 1):
        case = inputs.make_case(cfg, seed)
        pb = pact.Problem(cfg, DEV)
        w = pact.sos_to_delays(pb, torch.as_tensor(case["sos_true"], device=DEV))
        ref = O.wavefront_errors(O.geom(cfg), case["sos_true"], case["centres"]).numpy()
        assert rel(cpu(w), ref) <= 1e-4


def test_sos_to_delays_uniform_is_zero_and_background():
    cfg = inputs.config_small()
    pb = pact.Problem(cfg, DEV)
    w = pact.sos_to_delays(pb, torch.full((cfg.sos_g, cfg.sos_g), cfg.v0, device=DEV))
    assert float(w.abs().max()) == 0.0
    cfg2 = cfg.replace(v_bg=1510.0)
    pb2 = pact.Problem(cfg2, DEV)
    sos = torch.full((cfg.sos_g, cfg.sos_g), 1510.0, device=DEV)
    w2 = pact.sos_to_delays(pb2, sos)
    ref = O.wavefront_errors(O.geom(cfg2), np.full((cfg.sos_g, cfg.sos_g), 1510.0), cfg.centres()).numpy()
    assert rel(cpu(w2), ref) <= 1e-4


def test_sos_to_delays_full_size_sampled():
    cfg = inputs.config_full()
    case = inputs.make_case(cfg, 3)
    pb = pact.Problem(cfg, DEV)
    w = cpu(pact.sos_to_delays(pb, torch.as_tensor(case["sos_true"], device=DEV)))
    idx = [0, 13, 77, 143]                        # corner patches lie outside the mask
    ref = O.wavefront_errors(O.geom(cfg), case["sos_true"], case["centres"][idx]).numpy()
    assert rel(w[idx], ref) <= 1e-4


ADJ_CASES = {
    "tiny_p16_m4": CASES["tiny_p16_m4"],
    "small_p32_m8": CASES["small_p32_m8"],
    "tiny_nt48": CASES["tiny_nt48"],
    # grids whose excess rows and accumulator take several shared-memory bands
    "tiny_g200": lambda: inputs.config_tiny(p=16, m=4).replace(sos_g=200),
    "tiny_g512": lambda: inputs.config_tiny(p=16, m=4).replace(sos_g=512),
}


@pytest.mark.parametrize("name", list(ADJ_CASES))
def test_sos_to_delays_adj(name):
    cfg = ADJ_CASES[name]()
    case = inputs.make_case(cfg, 2)
    pb = pact.Problem(cfg, DEV)
    r = np.random.default_rng(5).standard_normal((cfg.n_patches, cfg.n_t)).astype(np.float32)
    sos = torch.as_tensor(case["sos_true"], device=DEV)
    g = cpu(pact.sos_to_delays_adj(pb, sos, torch.as_tensor(r, device=DEV)))
    ref = O.sos_to_delays_adj(O.geom(cfg), case["sos_true"], case["centres"], r).numpy()
    assert rel(g, ref) <= 2e-3
    # fixed-point shared sums: the same bits on every call
    g_again = cpu(pact.sos_to_delays_adj(pb, sos, torch.as_tensor(r, device=DEV)))
    assert np.array_equal(g, g_again)
    # accumulate adds
    base = torch.ones((cfg.sos_g, cfg.sos_g), device=DEV)
    g2 = cpu(pact.sos_to_delays_adj(pb, sos, torch.as_tensor(r, device=DEV), base, accumulate=True))
    assert rel(g2, ref + 1.0) <= 2e-3


@pytest.mark.parametrize("sos_g", [None, 200])
def test_rays_with_mask_beyond_the_node_hull(sos_g):
    """A mask disk larger than the SOS grid's field of view: samples beyond the
    node hull take the edge-clamped SOS (the kernels' clamped paths; with a
    200² grid the adjoint also runs in several row bands)."""
    cfg = inputs.config_tiny(p=16, m=4)
    if sos_g:
        cfg = cfg.replace(sos_g=sos_g)
    gd = cfg.geometry_dict()
    gd["mask_radius"] = 0.7 * cfg.fov
    pb = pact.Problem(cfg, DEV)
    pb.geom.mask_radius = gd["mask_radius"]
    case = inputs.make_case(cfg, 9)
    sos_np = case["sos_true"].copy()
    sos_np[0, :] += 30.0                              # the edge rows matter now
    sos_np[:, -1] -= 25.0
    sos = torch.as_tensor(sos_np, device=DEV)
    w = cpu(pact.sos_to_delays(pb, sos))
    ref = O.wavefront_errors(O.geom(gd), sos_np, case["centres"]).numpy()
    assert rel(w, ref) <= 1e-4
    r = np.random.default_rng(12).standard_normal((cfg.n_patches, cfg.n_t)).astype(np.float32)
    g = cpu(pact.sos_to_delays_adj(pb, sos, torch.as_tensor(r, device=DEV)))
    ref = O.sos_to_delays_adj(O.geom(gd), sos_np, case["centres"], r).numpy()
    assert rel(g, ref) <= 2e-3


def test_sos_to_delays_adj_full_size():
    cfg = inputs.config_full()
    case = inputs.make_case(cfg, 1)
    pb = pact.Problem(cfg, DEV)
    rng = np.random.default_rng(6)
    r = np.zeros((cfg.n_patches, cfg.n_t), np.float32)
    idx = [5, 70, 140]
    r[idx] = rng.standard_normal((len(idx), cfg.n_t))
    sos = torch.as_tensor(case["sos_true"], device=DEV)
    g = cpu(pact.sos_to_delays_adj(pb, sos, torch.as_tensor(r, device=DEV)))
    ref = O.sos_to_delays_adj(O.geom(cfg), case["sos_true"], case["centres"][idx], r[idx]).numpy()
    assert rel(g, ref) <= 2e-3


def test_sos_to_delays_and_adj_channel_data_size_sampled():
    """1024 x 1024 image, 3721 patches, 1024 transducers, 256 x 256 SOS grid
    (too large to stage in shared memory: the kernels read the grid from
    global memory and the adjoint scatters with global atomics)."""
    cfg = inputs.config_rf()
    case = inputs.make_case(cfg.replace(m=1), 6)
    pb = pact.Problem(cfg, DEV)
    sos = torch.as_tensor(case["sos_true"], device=DEV)
    w = cpu(pact.sos_to_delays(pb, sos))
    idx = [0, 61, 1860, 2999, 3720]
    ref = O.wavefront_errors(O.geom(cfg), case["sos_true"], case["centres"][idx]).numpy()
    assert rel(w[idx], ref) <= 1e-4
    rng = np.random.default_rng(7)
    r = np.zeros((cfg.n_patches, cfg.n_t), np.float32)
    idx = [100, 1900, 3600]
    r[idx] = rng.standard_normal((len(idx), cfg.n_t))
    g = cpu(pact.sos_to_delays_adj(pb, sos, torch.as_tensor(r, device=DEV)))
    ref = O.sos_to_delays_adj(O.geom(cfg), case["sos_true"], case["centres"][idx], r[idx]).numpy()
    assert rel(g, ref) <= 2e-3


# ------------------------------------------------------------------ Eq. 4-5

@pytest.mark.parametrize("name", list(CASES))
def test_psf_synth_and_forward_model(name):
    cfg = CASES[name]()
    rng = np.random.default_rng(7)
    w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng)
    d = cfg.delays()
    pb = pact.Problem(cfg, DEV)
    wt = torch.as_tensor(w, device=DEV)
    H = cpu(pact.psf_synth(pb, wt, d))
    Href = O.transfer_functions(O.geom(cfg), w.astype(np.float64), cfg.centres(), d).numpy()
    assert rel(H, Href) <= 1e-4
    X = rand_Y((cfg.n_patches, cfg.p, cfg.p // 2 + 1), 8)
    Y = cpu(pact.forward_model(pb, wt, d, to_dev_c(X)))
    assert rel(Y, Href * X.astype(np.complex64)[:, None]) <= 1e-4
    Y2 = cpu(pact.forward_model(pb, wt, d, to_dev_c(X), to_dev_c(np.ones_like(Y)), accumulate=True))
    assert rel(Y2, Href * X.astype(np.complex64)[:, None] + 1) <= 1e-4


@pytest.mark.parametrize("name", ["tiny_p16_m4", "small_p32_m8"])
def test_psf_synth_adj(name):
    cfg = CASES[name]()
    rng = np.random.default_rng(9)
    w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng)
    d = cfg.delays()
    G = rand_Y((cfg.n_patches, cfg.m, cfg.p, cfg.p // 2 + 1), 10)
    pb = pact.Problem(cfg, DEV)
    gw = cpu(pact.psf_synth_adj(pb, torch.as_tensor(w, device=DEV), d, to_dev_c(G)))
    wr = torch.tensor(w.astype(np.float64), requires_grad=True)
    H = O.transfer_functions(O.geom(cfg), wr, cfg.centres(), d)
    Gt = torch.as_tensor(G.astype(np.complex128))
    (ref,) = torch.autograd.grad((Gt.real * H.real + Gt.imag * H.imag).sum(), wr)
    assert rel(gw, ref.numpy()) <= 2e-3


# ------------------------------------------------------------------ Eq. 6-7 fused + adjoint

def _mcd_case(cfg, seed, d=None, realistic=False):
    rng = np.random.default_rng(seed)
    if realistic:
        case = inputs.make_case(cfg, seed)
        Y, _, _ = O.make_measurement(O.geom(cfg), case)
        Y = Y.numpy()
        w = O.wavefront_errors(O.geom(cfg), case["sos_init"], case["centres"]).numpy().astype(np.float32)
        w = (w + inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng, 1e-4)).astype(np.float32)
    else:
        Y = rand_Y((cfg.n_patches, cfg.m, cfg.p, cfg.p // 2 + 1), seed)
        w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng)
    d = cfg.delays() if d is None else np.asarray(d, np.float32)
    return Y.astype(np.complex64), w, d


def _scales(cfg, Y):
    """Loss and gradient scales of the data term (X_hat = 0): floors for cases
    whose exact loss or gradient is 0 (M = 1 with eps = 0)."""
    kx, ky, kmag, _, ck = (t.numpy() for t in O.kgrid(O.geom(cfg)))
    om = ck * kmag * 1e-3
    e = (np.abs(Y.astype(np.complex128)) ** 2).sum(1)
    return float((om * e).sum()), float((om * kmag * e).sum()) / np.sqrt(cfg.n_patches * cfg.n_t)


def _check_mcd(cfg, Y, w, d, eps, idx=None, tol_g=2e-3):
    pb = pact.Problem(cfg, DEV)
    out = pact.mc_deconv_loss(pb, torch.as_tensor(w, device=DEV), to_dev_c(Y), d, eps, want_grad=True,
                              want_xhat=True, want_loss_pp=True)
    torch.cuda.synchronize()
    sel = slice(None) if idx is None else idx
    cen = cfg.centres()[sel]
    L, lp, Xh, gw = O.mc_deconv_loss(O.geom(cfg), w[sel].astype(np.float64), torch.as_tensor(Y[sel]), cen, d, eps)
    l_sc, g_sc = _scales(cfg, Y[sel])
    if idx is None:
        assert abs(float(out["loss"].item()) - float(L)) <= 1e-4 * abs(float(L)) + 1e-7 * l_sc
    lpg = cpu(out["loss_pp"])[sel]
    assert np.linalg.norm(lpg - lp.numpy()) <= 1e-4 * np.linalg.norm(lp.numpy()) + 1e-7 * l_sc
    assert rel(cpu(out["Xhat"])[sel], Xh.numpy()) <= 1e-4
    if cfg.m == 1 and eps == 0.0:
        # exact gradient is 0 (zero residual); in FP32 it is rounding noise scaled
        # by 1/|H|, unbounded near the zeros of H -- nothing to compare
        return out
    gg = cpu(out["dL_dw"])[sel]
    assert np.linalg.norm(gg - gw.numpy()) <= tol_g * np.linalg.norm(gw.numpy()) + 1e-7 * g_sc
    return out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("eps", [1e-3, 0.0])
def test_mc_deconv_loss(name, eps):
    cfg = CASES[name]()
    Y, w, d = _mcd_case(cfg, 11)
    _check_mcd(cfg, Y, w, d, eps)


def test_mc_deconv_loss_realistic_small():
    cfg = inputs.config_small()
    Y, w, d = _mcd_case(cfg, 0, realistic=True)
    _check_mcd(cfg, Y, w, d, cfg.eps)
    _check_mcd(cfg, Y, w, d, 1e-8)          # FP64 denominator path


def test_mc_deconv_loss_nonuniform_delays_and_wide_channels():
    cfg = inputs.config_tiny(p=16, m=5)
    d = np.array([-7e-4, -2e-4, 0.0, 1.5e-4, 6e-4], np.float32)
    Y, w, _ = _mcd_case(cfg, 12)
    _check_mcd(cfg, Y, w, d, 1e-3)
    cfg64 = inputs.config_tiny(p=8, m=64)
    Y, w, d = _mcd_case(cfg64, 13)
    _check_mcd(cfg64, Y, w, d, 1e-3)
    cfg40 = inputs.config_tiny(p=10, m=40)
    Y, w, d = _mcd_case(cfg40, 14)
    _check_mcd(cfg40, Y, w, d, 1e-3)
    cfg16 = inputs.config_tiny(p=12, m=16)             # uniform delays: factorised phases
    Y, w, d = _mcd_case(cfg16, 22)
    _check_mcd(cfg16, Y, w, d, 1e-3)
    d16 = d.copy()
    d16[5] += 3e-6                                     # no longer uniform: one phase factor per channel
    _check_mcd(cfg16, Y, w, d16, 1e-3)


def test_mc_deconv_loss_full_size_sampled():
    """512x512 image, 144 patches of 80x80, 32 channels: the launch the benchmark
    times; the oracle checks a sample of patches."""
    cfg = inputs.config_full()
    Y, w, d = _mcd_case(cfg, 15)
    _check_mcd(cfg, Y, w, d, cfg.eps, idx=[0, 11, 72, 100, 143])


def test_mc_deconv_loss_channel_data_size_sampled():
    """3721 patches of 64 x 64, 32 channels, 1024 transducers: 2.0 GB of
    spectra, far beyond L2; the oracle checks a sample of patches."""
    cfg = inputs.config_rf()
    rng = np.random.default_rng(31)
    z = rng.standard_normal((cfg.n_patches, cfg.m, cfg.p, cfg.p // 2 + 1, 2), dtype=np.float32)
    Y = z.view(np.complex64)[..., 0]
    del z
    w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng)
    _check_mcd(cfg, Y, w, cfg.delays(), cfg.eps, idx=[0, 60, 1234, 1860, 3720])


_REALISTIC = {}


def _realistic_full(seed):
    """The benchmark problem's measurement spectra, Y = H(v_true) X + N (Eq. 5
    plus the seeded noise stack), made by the FP64 oracle."""
    if seed not in _REALISTIC:
        cfg = inputs.config_full()
        case = inputs.make_case(cfg, seed)
        Y, _, _ = O.make_measurement(O.geom(cfg), case)
        _REALISTIC[seed] = (cfg, case, Y.numpy().astype(np.complex64))
    return _REALISTIC[seed]


def _near_truth(cfg, case, seed, amp):
    """The true SOS plus a seeded perturbation of a few m/s (Gaussian ellipses
    from the input generator, shifted to zero background)."""
    rng = np.random.default_rng(seed)
    bump = inputs.sos_phantom(cfg.replace(sos_lo=cfg.v_bg - amp, sos_hi=cfg.v_bg + amp), rng) - cfg.v_bg
    return (case["sos_true"] + bump * case["mask"]).astype(np.float32)


@pytest.mark.parametrize("point", ["truth", "near_truth", "uniform"])
def test_mc_deconv_loss_realistic_full_size(point):
    """All 144 patches of the benchmark launch on realistic spectra, where the
    loss is small against the data energy (at the truth it is the noise floor):
    the regime in which the closed-form residual energy of the streaming kernel
    is least accurate.  Loss, per-patch loss, X_hat (1e-4) and dL/dw (2e-3)."""
    cfg, case, Y = _realistic_full(0)
    g = O.geom(cfg)
    sos = {"truth": case["sos_true"], "near_truth": None, "uniform": case["sos_init"]}[point]
    if sos is None:
        sos = _near_truth(cfg, case, 17, 3.0)
    w = O.wavefront_errors(g, sos.astype(np.float64), case["centres"]).numpy().astype(np.float32)
    _check_mcd(cfg, Y, w, cfg.delays(), cfg.eps)
    if point == "truth":
        _check_mcd(cfg, Y, w, cfg.delays(), 1e-8)        # FP64 denominators, explicit residual


def test_mc_deconv_loss_at_the_fp64_cold_end_point():
    """The held-out warm-start problem at the end point of the FP64 oracle's own
    1000-iteration cold recovery (tests/golden/make_cold_optimum.py): all 144
    patches, near a local optimum of Eq. 7, against the oracle."""
    import os
    cfg = inputs.config_held_out()
    path = os.path.join(os.path.dirname(__file__), "golden", f"cold_optimum_{cfg.name}_seed1000.npy")
    sos = np.load(path).astype(np.float64)
    case = inputs.make_case(cfg, 1000)
    g = O.geom(cfg)
    Y = O.make_measurement(g, case)[0].numpy().astype(np.complex64)
    w = O.wavefront_errors(g, sos, case["centres"]).numpy().astype(np.float32)
    _check_mcd(cfg, Y, w, cfg.delays(), cfg.eps)


def test_mc_deconv_loss_on_das_spectra_sampled():
    """Spectra made the way the channel-data workload makes them -- ring channel
    data (oracle) -> DAS (Eq. 1, oracle, at the pixels of the sampled patches)
    -> windowed patch DFT (oracle) -- on the 1024 x 1024 / 1024-element
    geometry with a sparse source image, for three patches; then the fused pass
    against the oracle at the true and at the uniform SOS."""
    from oracle import rf_oracle as R
    cfg = inputs.config_rf()
    case = inputs.make_case(cfg, 4)
    g = O.geom(cfg)
    rng = np.random.default_rng(8)
    ip = case["ip"].copy()
    on = np.argwhere(ip != 0)
    keep = on[rng.choice(len(on), size=min(400, len(on)), replace=False)]
    src = np.zeros_like(ip)
    src[keep[:, 0], keep[:, 1]] = ip[keep[:, 0], keep[:, 1]]
    rf = R.rf_synth(g, src, case["sos_true"], cfg.rf_fs, cfg.rf_t0, cfg.rf_ns, cfg.rf_sigma)
    idx = [1830, 1860, 1890]                               # patches near the centre row
    cen = case["centres"][idx]
    P = cfg.p
    rr, cc = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    stack = np.zeros((cfg.m, cfg.img_h, cfg.img_w))
    for ca, cb in cen:
        rows = (ca - P // 2 + rr).ravel()
        cols = (cb - P // 2 + cc).ravel()
        vals = R.das_at(g, rf, cfg.rf_fs, cfg.rf_t0, cfg.delays(), torch.as_tensor(rows), torch.as_tensor(cols))
        stack[:, rows, cols] = vals.numpy()
    Y = O.patch_spectra(g, torch.as_tensor(stack), cen).numpy().astype(np.complex64)
    sub = cfg.replace(centres_rows=(0,), centres_cols=(0,))
    for sos in (case["sos_true"], case["sos_init"]):
        w = O.wavefront_errors(g, sos.astype(np.float64), cen).numpy().astype(np.float32)
        _check_mcd_centres(sub, cen, Y, w, cfg.delays(), cfg.eps)


def _check_mcd_centres(cfg, cen, Y, w, d, eps):
    """_check_mcd for an explicit list of patch centres."""
    pb = pact.Problem(cfg, DEV, centres=np.asarray(cen, np.int32))
    out = pact.mc_deconv_loss(pb, torch.as_tensor(w, device=DEV), to_dev_c(Y), d, eps, want_grad=True,
                              want_xhat=True, want_loss_pp=True)
    torch.cuda.synchronize()
    L, lp, Xh, gw = O.mc_deconv_loss(O.geom(cfg), w.astype(np.float64), torch.as_tensor(Y), cen, d, eps)
    assert abs(float(out["loss"].item()) - float(L)) <= 1e-4 * abs(float(L))
    assert np.linalg.norm(cpu(out["loss_pp"]) - lp.numpy()) <= 1e-4 * np.linalg.norm(lp.numpy())
    assert rel(cpu(out["Xhat"]), Xh.numpy()) <= 1e-4
    assert rel(cpu(out["dL_dw"]), gw.numpy()) <= 2e-3


def test_mc_deconv_loss_adj_scale_and_accumulate():
    cfg = inputs.config_tiny(p=16, m=4)
    Y, w, d = _mcd_case(cfg, 16)
    pb = pact.Problem(cfg, DEV)
    wt, Yt = torch.as_tensor(w, device=DEV), to_dev_c(Y)
    g1 = pact.mc_deconv_loss(pb, wt, Yt, d, 1e-3)["dL_dw"]
    s = torch.tensor([2.5], device=DEV)
    g2 = pact.mc_deconv_loss_adj(pb, wt, Yt, d, 1e-3, dL_dloss=s)
    assert rel(cpu(g2), 2.5 * cpu(g1)) <= 1e-6
    g3 = pact.mc_deconv_loss_adj(pb, wt, Yt, d, 1e-3, dL_dw=torch.ones_like(g1), accumulate=True)
    assert rel(cpu(g3), cpu(g1) + 1) <= 1e-6


@pytest.mark.parametrize("eps", [1e-3, 1e-8])
def test_mc_deconv_loss_tabled_matches_per_call_tables(eps):
    """Prebuilt tables give the outputs of the per-call build (and the oracle);
    tables built for other delays poison the outputs with NaN."""
    cfg = inputs.config_small()
    Y, w, d = _mcd_case(cfg, 0, realistic=True)
    pb = pact.Problem(cfg, DEV)
    wt, Yt = torch.as_tensor(w, device=DEV), to_dev_c(Y)
    tab = pact.McdTables(pb, d)
    ref = pact.mc_deconv_loss(pb, wt, Yt, d, eps, want_xhat=True, want_loss_pp=True)
    for _ in range(2):
        out = pact.mc_deconv_loss(pb, wt, Yt, d, eps, want_xhat=True, want_loss_pp=True, tables=tab)
        assert float(out["loss"].item()) == float(ref["loss"].item())
        assert torch.equal(out["Xhat"], ref["Xhat"]) and torch.equal(out["loss_pp"], ref["loss_pp"])
        assert rel(cpu(out["dL_dw"]), cpu(ref["dL_dw"])) <= 1e-6
    L, _, _, gw = O.mc_deconv_loss(O.geom(cfg), w.astype(np.float64), torch.as_tensor(Y), cfg.centres(), d, eps)
    assert abs(float(out["loss"].item()) - float(L)) <= 1e-4 * float(L)
    assert rel(cpu(out["dL_dw"]), gw.numpy()) <= 2e-3
    other = pact.McdTables(pb, d * 1.01)
    bad = pact.mc_deconv_loss(pb, wt, Yt, d, eps, tables=other)
    assert np.isnan(float(bad["loss"].item())) and np.isnan(cpu(bad["dL_dw"])).any()


def test_mc_deconv_loss_overwrites_dl_dw_back_to_back():
    """dL/dw is overwritten whatever it held (the streaming kernel clears it
    itself, each CTA a share, before any CTA adds to it), also for calls
    queued back to back on one stream, where each call's kernel may start
    while the one before is finishing; with and without prebuilt tables, on a
    small case and on the full-size launch."""
    for cfg in (inputs.config_small(), inputs.config_full()):
        Y, w, d = _mcd_case(cfg, 5)
        pb = pact.Problem(cfg, DEV)
        wt, Yt = torch.as_tensor(w, device=DEV), to_dev_c(Y)
        tab = pact.McdTables(pb, d)
        ref = pact.mc_deconv_loss(pb, wt, Yt, d, cfg.eps)
        torch.cuda.synchronize()
        outs = []
        for k, fill in enumerate((float("nan"), 7.0, -1e30, float("inf"), 0.0, 3.0)):
            o = {"loss": torch.zeros(1, device=DEV), "dL_dw": torch.full((pb.n, pb.n_t), fill, device=DEV)}
            pact.mc_deconv_loss(pb, wt, Yt, d, cfg.eps, out=o, tables=tab if k % 2 == 0 else None)
            outs.append(o)
        torch.cuda.synchronize()
        g_ref = cpu(ref["dL_dw"])
        assert np.isfinite(g_ref).all() and np.abs(g_ref).max() > 0
        for o in outs:
            assert float(o["loss"].item()) == float(ref["loss"].item())      # fixed-order loss sums
            assert rel(cpu(o["dL_dw"]), g_ref) <= 1e-6


def test_accumulating_pass_behind_the_ray_kernel():
    """In a recovery iteration the fused pass adds to the dL/dw that the ray
    kernel ahead of it clears and reads the w that kernel writes, while the
    copies and channel sums of each CTA's first unit may run before that kernel
    has ended.  Queued back to back on one stream for three SOS fields, each
    pass equals a separate clearing call on the same w: bit-equal loss (fixed
    order sums) and dL/dw up to the order of the atomics; small case and the
    full-size launch."""
    for cfg in (inputs.config_small(), inputs.config_full()):
        case = inputs.make_case(cfg, 3)
        Y, _, d = _mcd_case(cfg, 8)
        pb = pact.Problem(cfg, DEV)
        Yt = to_dev_c(Y)
        tab = pact.McdTables(pb, d)
        tv_ws = pact._ws(pact.sos_to_delays_tv_workspace_size(pb), DEV)
        w = torch.empty(pb.n, pb.n_t, device=DEV)
        out = {"loss": torch.zeros(1, device=DEV), "dL_dw": torch.full((pb.n, pb.n_t), 5.0, device=DEV)}
        sos = [torch.as_tensor(case["sos_init"] + a * (case["sos_true"] - case["sos_init"]), device=DEV)
               for a in (0.3, 1.0, 0.6)]
        got = []
        torch.cuda.synchronize()
        for s in sos:
            pact.sos_to_delays_tv(pb, s, w, out["dL_dw"], cfg.tv_lambda, tv_ws)
            pact.mc_deconv_loss(pb, w, Yt, d, cfg.eps, out=out, tables=tab, accumulate=True)
            got.append((out["loss"].clone(), out["dL_dw"].clone()))
        torch.cuda.synchronize()
        for s, (loss, gw) in zip(sos, got):
            ref = pact.mc_deconv_loss(pb, pact.sos_to_delays(pb, s), Yt, d, cfg.eps)
            assert float(loss.item()) == float(ref["loss"].item())
            g_ref = cpu(ref["dL_dw"])
            assert np.isfinite(g_ref).all() and np.abs(g_ref).max() > 0
            assert rel(cpu(gw), g_ref) <= 1e-6


def test_mc_deconv_loss_misaligned_w_takes_the_general_path():
    """w not 16-byte aligned (the streaming kernel copies w rows in bulk): the
    two-pass kernel serves the call with the same results."""
    cfg = inputs.config_small()
    Y, w, d = _mcd_case(cfg, 0, realistic=True)
    pb = pact.Problem(cfg, DEV)
    big = torch.zeros(w.size + 1, dtype=torch.float32, device=DEV)
    big[1:] = torch.as_tensor(w.ravel(), device=DEV)
    w_odd = big[1:].view(w.shape)
    assert w_odd.data_ptr() % 16 != 0
    Yt = to_dev_c(Y)
    a = pact.mc_deconv_loss(pb, torch.as_tensor(w, device=DEV), Yt, d, cfg.eps, want_xhat=True)
    b = pact.mc_deconv_loss(pb, w_odd, Yt, d, cfg.eps, want_xhat=True)
    assert abs(float(a["loss"].item()) - float(b["loss"].item())) <= 1e-5 * float(a["loss"].item())
    assert rel(cpu(b["Xhat"]), cpu(a["Xhat"])) <= 1e-6
    assert rel(cpu(b["dL_dw"]), cpu(a["dL_dw"])) <= 1e-5


def test_mc_deconv_loss_noise_free_truth_is_minimum():
    """Y = H(w) X exactly, eps = 0: the loss at w is ~0 relative to a perturbed w."""
    cfg = inputs.config_small()
    pb = pact.Problem(cfg, DEV)
    rng = np.random.default_rng(17)
    w = inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng)
    X = rand_Y((cfg.n_patches, cfg.p, cfg.p // 2 + 1), 18)
    wt = torch.as_tensor(w, device=DEV)
    Y = pact.forward_model(pb, wt, cfg.delays(), to_dev_c(X))
    l0 = float(pact.mc_deconv_loss(pb, wt, Y, cfg.delays(), 0.0, want_grad=False)["loss"].item())
    l1 = float(pact.mc_deconv_loss(pb, wt + 5e-5, Y, cfg.delays(), 0.0, want_grad=False)["loss"].item())
    assert l0 <= 1e-6 * l1


# ------------------------------------------------------------------ Sec. S1.5 spectra, stitching

FFT_CASES = {
    "tiny_p8_m1": CASES["tiny_p8_m1"],
    "tiny_p12_m3": CASES["tiny_p12_m3"],
    "tiny_p16_m4": CASES["tiny_p16_m4"],
    "tiny_p18_m3": lambda: inputs.config_tiny(p=18, m=3),      # P = 2 mod 4: ragged row tiles
    "tiny_p4_m2": lambda: inputs.config_tiny(p=4, m=2),        # smallest patch: one folded pair
    "tiny_p128_m2": lambda: inputs.config_tiny(p=128, m=2),    # largest patch (3 row-pass tiles per thread),
                                                               # reaching past the 64 x 64 image (zero padding)
    "small_p32_m8": inputs.config_small,
}


@pytest.mark.parametrize("name", list(FFT_CASES))
def test_patch_fft(name):
    cfg = FFT_CASES[name]()
    case = inputs.make_case(cfg, 3)
    pb = pact.Problem(cfg, DEV)
    Y = cpu(pact.patch_fft(pb, torch.as_tensor(case["noise"], device=DEV)))
    ref = O.patch_spectra(O.geom(cfg), case["noise"], case["centres"]).numpy()
    assert rel(Y, ref) <= 1e-4


def test_patch_fft_full_size_sampled():
    cfg = inputs.config_full()
    case = inputs.make_case(cfg, 4)
    pb = pact.Problem(cfg, DEV)
    Y = cpu(pact.patch_fft(pb, torch.as_tensor(case["noise"][:4], device=DEV)))
    idx = [0, 50, 143]
    ref = O.patch_spectra(O.geom(cfg), case["noise"][:4], case["centres"][idx]).numpy()
    assert rel(Y[idx], ref) <= 1e-4


def test_patch_fft_channel_data_size_sampled():
    """64 x 64 patches of the 1024 x 1024 channel-data image (3721 patches at
    stride 16), four channels of noise: the first, last and middle patches and
    one on the top edge, checked against the oracle."""
    cfg = inputs.config_rf()
    pb = pact.Problem(cfg, DEV)
    stack = np.random.default_rng(23).standard_normal((4, cfg.img_h, cfg.img_w)).astype(np.float32)
    Y = cpu(pact.patch_fft(pb, torch.as_tensor(stack, device=DEV)))
    idx = [0, 60, 1860, 3720]
    ref = O.patch_spectra(O.geom(cfg), stack, cfg.centres()[idx]).numpy()
    assert rel(Y[idx], ref) <= 1e-4


@pytest.mark.parametrize("name", ["tiny_p16_m4", "small_p32_m8"])
def test_stitch(name):
    cfg = CASES[name]()
    pb = pact.Problem(cfg, DEV)
    X = rand_Y((cfg.n_patches, cfg.p, cfg.p // 2 + 1), 19)
    img = cpu(pact.stitch(pb, to_dev_c(X)))
    ref = O.stitch(O.geom(cfg), torch.as_tensor(X.astype(np.complex128)), cfg.centres()).numpy()
    assert rel(img, ref) <= 1e-4


def test_stitch_channels_matches_oracle_per_channel():
    """The delay stack of Eq. 5 from [N][M] patch spectra, all channels in one call."""
    cfg = inputs.config_small()
    pb = pact.Problem(cfg, DEV)
    Y = rand_Y((cfg.n_patches, cfg.m, cfg.p, cfg.p // 2 + 1), 21)
    st = cpu(pact.stitch_channels(pb, to_dev_c(Y)))
    assert st.shape == (cfg.m, cfg.img_h, cfg.img_w)
    for j in (0, 3, cfg.m - 1):
        ref = O.stitch(O.geom(cfg), torch.as_tensor(Y[:, j].astype(np.complex128)), cfg.centres()).numpy()
        assert rel(st[j], ref) <= 1e-4


# ------------------------------------------------------------------ Eq. 1

def test_das_stack():
    cfg = inputs.config_tiny(p=16, m=3).replace(img_h=48, img_w=40, n_t=32)
    pb = pact.Problem(cfg, DEV)
    fs, n_s, t0 = 40e6, 400, 2e-6
    t = np.arange(n_s) / fs
    rng = np.random.default_rng(20)
    rf = np.zeros((cfg.n_t, n_s))
    for n in range(cfg.n_t):                       # band-limited: a few Gaussian-windowed tones
        for _ in range(4):
            f0, tc = rng.uniform(1e6, 6e6), rng.uniform(t[0], t[-1])
            rf[n] += np.cos(2 * np.pi * f0 * (t - tc)) * np.exp(-((t - tc) / 4e-7) ** 2)
    rf = rf.astype(np.float32)
    d = np.array([-3e-4, 0.0, 4e-4], np.float32)
    st = cpu(pact.das_stack(pb, torch.as_tensor(rf, device=DEV), fs, t0, d))
    ref = O.das_stack(O.geom(cfg), rf, fs, t0, d).numpy()
    assert rel(st, ref) <= 5e-4


@pytest.mark.parametrize("m,h,w", [(32, 72, 100), (5, 72, 100), (8, 70, 100), (1, 37, 45), (64, 72, 100), (17, 9, 33)])
def test_das_stack_tiled_windows(m, h, w):
    """The tiled DAS path (each 32 x 8 pixel tile, warps over 8 x 4 pixel
    blocks, reads a staged window of samples per transducer): 0.05 mm pixels at
    40 MHz, ragged tiles and warp blocks (100 x 72, 100 x 70, 45 x 37, 33 x 9
    pixels) and a ragged last chunk of transducers (48), arrivals before the
    record start and after its end (zero there), uniform and non-uniform
    delays, channel counts with an exact kernel instance (8, 32, 64) and
    without (1, 5, 17)."""
    cfg = inputs.config_tiny(p=16, m=3).replace(img_h=h, img_w=w, dx=0.05e-3, n_t=48)
    pb = pact.Problem(cfg, DEV)
    fs, n_s, t0 = 40e6, 60, 5.5e-6
    rng = np.random.default_rng(23)
    rf = rng.standard_normal((cfg.n_t, n_s)).astype(np.float32)
    if m == 5:
        d = np.array([-6e-4, -1e-4, 0.0, 2.5e-4, 7e-4], np.float32)
    else:
        d = np.linspace(-7.5e-4, 7.5e-4, m).astype(np.float32) if m > 1 else np.array([2e-4], np.float32)
    st = cpu(pact.das_stack(pb, torch.as_tensor(rf, device=DEV), fs, t0, d))
    ref = O.das_stack(O.geom(cfg), rf, fs, t0, d).numpy()
    assert np.abs(ref).max() > 1.0          # (sample positions run from about -70 to 110: both ends are crossed)
    assert rel(st, ref) <= 5e-4


def test_das_stack_channel_data_size_sampled():
    """1024 transducers x 4096 samples at 40 MHz -> 32 x 1024 x 1024 (the
    channel-data workload's launch), checked at sampled pixels."""
    from oracle import rf_oracle as R
    cfg = inputs.config_rf()
    pb = pact.Problem(cfg, DEV)
    rng = np.random.default_rng(24)
    rf = rng.standard_normal((cfg.n_t, cfg.rf_ns)).astype(np.float32)
    d = cfg.delays()
    st = pact.das_stack(pb, torch.as_tensor(rf, device=DEV), cfg.rf_fs, cfg.rf_t0, d)
    rows = np.array([0, 1, 7, 8, 300, 511, 512, 777, 1016, 1023])
    cols = np.array([0, 31, 32, 500, 1023, 64, 513, 95, 1000, 1])
    got = st[:, torch.as_tensor(rows, device=DEV), torch.as_tensor(cols, device=DEV)].cpu().numpy()
    ref = R.das_at(O.geom(cfg), rf, cfg.rf_fs, cfg.rf_t0, d, torch.as_tensor(rows), torch.as_tensor(cols)).numpy()
    assert rel(got, ref) <= 5e-4


# ------------------------------------------------------------------ TV, Adam

def test_tv():
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 5)
    pb = pact.Problem(cfg, DEV)
    sos = torch.as_tensor(case["sos_true"], device=DEV)
    val = torch.zeros(1, device=DEV)
    grad = torch.zeros_like(sos)
    pact.tv(pb, sos, 1e-4, val, grad)
    s = torch.tensor(case["sos_true"].astype(np.float64), requires_grad=True)
    T = 1e-4 * O.tv(s)
    (gref,) = torch.autograd.grad(T, s)
    assert abs(float(val.item()) - float(T.detach())) <= 1e-5 * float(T.detach())
    assert rel(cpu(grad), gref.numpy()) <= 1e-6


def test_adam_matches_oracle_and_counter():
    rng = np.random.default_rng(21)
    n = 1000
    p0 = rng.standard_normal(n).astype(np.float32)
    mask = (rng.uniform(size=n) > 0.3).astype(np.uint8)
    p, m, v = (torch.as_tensor(x, device=DEV) for x in (p0.copy(), np.zeros(n, np.float32), np.zeros(n, np.float32)))
    p2, m2, v2 = p.clone(), m.clone(), v.clone()
    cnt = torch.zeros(2, dtype=torch.int32, device=DEV)
    rp, rm, rv = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.standard_normal(n).astype(np.float32)
        gt = torch.as_tensor(g, device=DEV)
        pact.adam_step(p, gt, m, v, t, 0.05, mask=torch.as_tensor(mask, device=DEV))
        pact.adam_step(p2, gt, m2, v2, 99, 0.05, mask=torch.as_tensor(mask, device=DEV), step_counter=cnt)
        rp, rm, rv = (x.numpy() for x in O.adam_step(rp, g, rm, rv, t, 0.05, mask=mask))
    assert rel(cpu(p), rp) <= 1e-6
    assert rel(cpu(p2), rp) <= 1e-6
    assert cnt.tolist() == [5, 0]


def test_adam_counter_with_many_ctas_in_a_graph():
    """The step count advances once per call also when the update spans many
    CTAs (the last one to finish advances it), eagerly and on graph replays."""
    rng = np.random.default_rng(22)
    n = 600_000
    p0 = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    p, m, v = (torch.as_tensor(x, device=DEV) for x in (p0.copy(), np.zeros(n, np.float32), np.zeros(n, np.float32)))
    gt = torch.as_tensor(g, device=DEV)
    cnt = torch.zeros(2, dtype=torch.int32, device=DEV)
    pact.adam_step(p, gt, m, v, 1, 1e-3, step_counter=cnt)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        pact.adam_step(p, gt, m, v, 1, 1e-3, step_counter=cnt)
    for _ in range(6):
        graph.replay()
    torch.cuda.synchronize()
    assert cnt.tolist() == [7, 0]        # capture does not run the kernel: 1 eager + 6 replays
    rp, rm, rv = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 8):
        rp, rm, rv = (x.numpy() for x in O.adam_step(rp, g, rm, rv, t, 1e-3))
    assert rel(cpu(p), rp) <= 1e-6


# ------------------------------------------------------------------ recovery loop, graphs, autograd

def test_recovery_iteration_matches_oracle():
    """One full iteration (Eq. 3-7 + TV + Adam) equals the oracle's, and the
    50-step FP32 loss curve tracks the FP64 oracle's."""
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 0)
    g = O.geom(cfg)
    Y64, _, _ = O.make_measurement(g, case)
    pb = pact.Problem(cfg, DEV)
    rec = PGRecovery(pb, to_dev_c(Y64.numpy()), case["d"], cfg.eps, cfg.tv_lambda, cfg.lr,
                     torch.as_tensor(case["sos_init"]), torch.as_tensor(case["mask"]))
    rec.step()
    L0, _, _, gs = O.objective(g, case["sos_init"], Y64, case["centres"], case["d"], cfg.eps, cfg.tv_lambda)
    assert abs(rec.loss() - float(L0)) <= 1e-4 * float(L0)
    sos1, _, _ = O.adam_step(case["sos_init"], gs, np.zeros_like(gs), np.zeros_like(gs), 1, cfg.lr,
                             mask=case["mask"])
    assert rel(cpu(rec.sos) - case["sos_init"], sos1.numpy() - case["sos_init"]) <= 1e-3
    hist = [rec.loss()] + rec.run(49, record_every=1)
    _, ref = O.recover(g, case, Y64, 50, cfg.lr, cfg.eps, cfg.tv_lambda)
    assert rel(np.array(hist), np.array(ref)) <= 1e-2


def test_graph_replay_equals_eager():
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 1)
    Y64, _, _ = O.make_measurement(O.geom(cfg), case)
    pb = pact.Problem(cfg, DEV)
    args = (pb, to_dev_c(Y64.numpy()), case["d"], cfg.eps, cfg.tv_lambda, cfg.lr,
            torch.as_tensor(case["sos_init"]), torch.as_tensor(case["mask"]))
    a, b = PGRecovery(*args), PGRecovery(*args)
    b.capture()
    ha = a.run(6, record_every=1)
    hb = b.run(6, record_every=1)
    assert np.allclose(ha, hb, rtol=1e-5)
    assert rel(cpu(a.sos), cpu(b.sos)) <= 1e-5      # atomics reorder FP32 sums


def test_recover_reads_back_every_iteration():
    """The public end-to-end call (host stack upload, patch spectra, graph
    replays with each loss read back one iteration behind) gives the loss
    history and the SOS of the same recovery stepped eagerly."""
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 2)
    pb = pact.Problem(cfg, DEV)
    rng = np.random.default_rng(4)
    stack = torch.as_tensor(rng.standard_normal((cfg.m, cfg.img_h, cfg.img_w)).astype(np.float32)).pin_memory()
    args = (case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, torch.as_tensor(case["sos_init"]), torch.as_tensor(case["mask"]))
    for iters in (1, 2, 17, 60):
        r = recover(pb, stack, *args, iters)
        rec = PGRecovery(pb, pact.patch_fft(pb, stack.to(DEV)), *args)
        ref = rec.run(iters, record_every=1)
        assert len(r.hist) == iters and np.all(np.isfinite(r.hist)) and not r.restarts
        assert np.allclose(r.hist, ref, rtol=1e-4)          # atomics reorder FP32 sums
        assert r.sos.device.type == "cpu" and r.image.device.type == "cpu"
        assert rel(r.sos.numpy(), cpu(rec.sos)) <= 1e-4
        assert r.xhat.shape == (cfg.n_patches, cfg.p, cfg.p // 2 + 1)
        assert r.image.shape == (cfg.img_h, cfg.img_w)
        img = pact.stitch(pb, r.xhat)
        assert rel(r.image.numpy(), cpu(img)) <= 1e-6


def test_recover_restores_after_a_non_finite_loss():
    """A learning rate far too large drives the SOS to non-physical values
    (negative speeds: the rays return NaN); the loss check restores the last
    good state with a smaller learning rate until the losses stay finite."""
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 2)
    pb = pact.Problem(cfg, DEV)
    rng = np.random.default_rng(4)
    stack = torch.as_tensor(rng.standard_normal((cfg.m, cfg.img_h, cfg.img_w)).astype(np.float32)).pin_memory()
    r = recover(pb, stack, case["d"], cfg.eps, cfg.tv_lambda, 1e5, torch.as_tensor(case["sos_init"]),
                torch.as_tensor(case["mask"]), 80, snapshot_every=10)
    assert r.restarts and len(r.hist) == 80 and np.all(np.isfinite(r.hist))
    assert r.restarts[-1][2] < 1e5


def test_recover_raises_on_non_finite_input():
    """NaN in the host stack: every loss is non-finite, the restarts cannot
    help and the call raises with PACT_ERR_NONFINITE."""
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 2)
    pb = pact.Problem(cfg, DEV)
    stack = torch.zeros((cfg.m, cfg.img_h, cfg.img_w), dtype=torch.float32)
    stack[0, 64, 64] = float("nan")
    with pytest.raises(pact.PactError) as e:
        recover(pb, stack.pin_memory(), case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, torch.as_tensor(case["sos_init"]),
                torch.as_tensor(case["mask"]), 20, max_restarts=2)
    assert e.value.status == pact.PACT_ERR_NONFINITE


def test_autograd_functions():
    cfg = inputs.config_tiny(p=16, m=4)
    case = inputs.make_case(cfg, 2)
    pb = pact.Problem(cfg, DEV)
    Y, _, d = _mcd_case(cfg, 22)
    Yt = to_dev_c(Y)
    sos = torch.as_tensor(case["sos_true"], device=DEV).requires_grad_(True)
    w = SosToDelays.apply(pb, sos)
    L = McDeconvLoss.apply(pb, w, Yt, d, 1e-3)
    (3.0 * L).backward()
    _, _, _, gref = O.objective(O.geom(cfg), case["sos_true"], torch.as_tensor(Y.astype(np.complex128)),
                                case["centres"], d, 1e-3, 0.0)
    assert rel(cpu(sos.grad), 3.0 * gref.numpy()) <= 2e-3


@pytest.mark.parametrize("kind", ["pixel_grid", "siren"])
def test_checkpoint_resume_reproduces_the_loss_curve(tmp_path, kind):
    """Run 20 iterations; save after 10; a fresh recovery resumed from the file
    runs the last 10 with the same losses (the fused pass's float atomics may
    reorder sums: 1e-5) and ends at the same parameters."""
    from paper_2409_10876_gb300 import checkpoint
    from paper_2409_10876_gb300.recovery import SirenRecovery
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 5)
    pb = pact.Problem(cfg, DEV)
    Y = to_dev_c(O.make_measurement(O.geom(cfg), case)[0].numpy())

    def make():
        if kind == "siren":
            return SirenRecovery(pb, Y, case["d"], cfg.eps, inputs.SIREN_LR, inputs.siren_init(0), case["mask"])
        return PGRecovery(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, torch.as_tensor(case["sos_init"]),
                          torch.as_tensor(case["mask"]))

    h = checkpoint.config_hash(cfg, kind=kind)
    a = make()
    a.capture()
    first = a.run(10, record_every=1)
    path = str(tmp_path / "ck.npz")
    a.checkpoint(path, 10, 5, h)
    rest = a.run(10, record_every=1)
    b = make()
    meta = b.resume(path, h)
    assert meta["iteration"] == 10 and meta["seed"] == 5
    b.capture()
    again = b.run(10, record_every=1)
    assert np.all(np.isfinite(first + rest))
    assert np.allclose(again, rest, rtol=1e-5)
    pa, pb_ = (cpu(r.params if kind == "siren" else r.sos) for r in (a, b))
    assert rel(pb_, pa) <= 1e-5
    with pytest.raises(checkpoint.CheckpointError):
        make().resume(path, checkpoint.config_hash(cfg, kind="other"))
