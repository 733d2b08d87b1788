"""Neural-field SOS on BF16 tensor cores (pact_nf_forward / pact_nf_backward)
vs the FP64 oracle.

Tolerances: BF16 keeps 8 significant bits (relative rounding 2^-9); features,
weights and the activations of 4 hidden layers of width 128 are rounded, so
the field deviation v - v_bg and the gradients are compared at relative L2
3e-2 / 5e-2 (the FP32 path of the pixel grid keeps its 1e-4 / 2e-3)."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs, pact
from paper_2409_10876_gb300.recovery import NFRecovery

pytestmark = pytest.mark.gpu

FWD_TOL = 3e-2
GRAD_TOL = 5e-2


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _params(seed, w5_scale=30.0):
    p = inputs.nf_init(seed).astype(np.float32)
    sh = dict((n, s) for n, s in inputs.nf_shapes())
    off = 0
    for name, shape in inputs.nf_shapes():
        n = int(np.prod(shape))
        if name == "w5":
            p[off:off + n] *= w5_scale          # a field that varies by tens of m/s
        off += n
    return p


def _oracle_args(cfg):
    return (O.geom(cfg), inputs.nf_shapes(), inputs.nf_frequencies(), inputs.sos_mask(cfg),
            inputs.NF_V_MID, inputs.NF_V_HALF)


@pytest.mark.parametrize("cfg", [inputs.config_small(), inputs.config_full()], ids=["G32", "G128"])
def test_nf_forward_matches_oracle(cfg):
    pb = pact.Problem(cfg, "cuda")
    prm = _params(1)
    nf = pact.NeuralField(pb, prm, inputs.sos_mask(cfg))
    v = pact.nf_forward(nf).cpu().numpy()
    pact.nf_status(nf)
    g, sh, f, mask, vm, vh = _oracle_args(cfg)
    ref = O.nf_sos(g, O._t(prm), sh, f, mask, vm, vh).numpy()
    assert np.all(v[mask == 0] == cfg.v_bg)
    assert _rel(v - cfg.v_bg, ref - cfg.v_bg) <= FWD_TOL
    assert np.abs(v - ref).max() <= 2.0           # m/s


@pytest.mark.parametrize("cfg", [inputs.config_small(), inputs.config_full()], ids=["G32", "G128"])
def test_nf_backward_matches_oracle_vjp(cfg):
    pb = pact.Problem(cfg, "cuda")
    prm = _params(2)
    nf = pact.NeuralField(pb, prm, inputs.sos_mask(cfg))
    pact.nf_forward(nf)
    up = np.random.default_rng(3).standard_normal((cfg.sos_g, cfg.sos_g)).astype(np.float32)
    gp = pact.nf_backward(nf, torch.as_tensor(up, device="cuda")).cpu().numpy()
    pact.nf_status(nf)
    g, sh, f, mask, vm, vh = _oracle_args(cfg)
    p64 = O._t(prm).clone().requires_grad_(True)
    (ref,) = torch.autograd.grad((O.nf_sos(g, p64, sh, f, mask, vm, vh) * O._t(up)).sum(), p64)
    assert _rel(gp, ref.numpy()) <= GRAD_TOL
    # accumulate adds
    gp2 = pact.nf_backward(nf, torch.as_tensor(up, device="cuda"), torch.ones(prm.size, device="cuda"),
                           accumulate=True).cpu().numpy()
    assert _rel(gp2 - 1.0, gp) <= 1e-5


@pytest.mark.parametrize("G", [40, 72])
def test_nf_ragged_node_count_and_every_parameter_group(G):
    """Node counts that are not a multiple of the 128-node CTA tile (1600 and
    5184 nodes: the last CTA holds 64 rows past the grid, which must enter no
    sum): the field against the oracle, and the gradient of every parameter
    group on its own (a mis-placed weight block or a bias sum over the wrong
    rows shows up in its group, even where the whole vector would hide it)."""
    cfg = dataclasses.replace(inputs.config_small(), sos_g=G)
    pb = pact.Problem(cfg, "cuda")
    prm = _params(4)
    mask = inputs.sos_mask(cfg)
    nf = pact.NeuralField(pb, prm, mask)
    v = pact.nf_forward(nf).cpu().numpy()
    g, sh, f, _, vm, vh = _oracle_args(cfg)
    ref = O.nf_sos(g, O._t(prm), sh, f, mask, vm, vh).numpy()
    assert np.all(v[mask == 0] == cfg.v_bg)
    assert _rel(v - cfg.v_bg, ref - cfg.v_bg) <= FWD_TOL
    up = np.random.default_rng(5).standard_normal((G, G)).astype(np.float32)
    gp = pact.nf_backward(nf, torch.as_tensor(up, device="cuda")).cpu().numpy()
    pact.nf_status(nf)
    p64 = O._t(prm).clone().requires_grad_(True)
    (gr,) = torch.autograd.grad((O.nf_sos(g, p64, sh, f, mask, vm, vh) * O._t(up)).sum(), p64)
    gr = gr.numpy()
    assert _rel(gp, gr) <= GRAD_TOL
    off = 0
    for name, shape in inputs.nf_shapes():
        n = int(np.prod(shape))
        assert _rel(gp[off:off + n], gr[off:off + n]) <= 2 * GRAD_TOL, name
        off += n


def test_nf_objective_gradient_end_to_end():
    """NF -> rays -> fused deconvolution/loss/adjoint -> ray adjoint -> NF
    backward, all in libpact, vs the oracle's autograd gradient of Eq. 7."""
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 0)
    g, sh, f, mask, vm, vh = _oracle_args(cfg)
    Y64, _, _ = O.make_measurement(g, case)
    pb = pact.Problem(cfg, "cuda")
    prm = _params(4)
    nf = pact.NeuralField(pb, prm, mask)
    Y = torch.as_tensor(Y64.numpy().astype(np.complex64), device="cuda")
    sos = pact.nf_forward(nf)
    w = pact.sos_to_delays(pb, sos)
    out = pact.mc_deconv_loss(pb, w, Y, case["d"], cfg.eps)
    gs = pact.sos_to_delays_adj(pb, sos, out["dL_dw"])
    gp = pact.nf_backward(nf, gs).cpu().numpy()
    pact.nf_status(nf)
    L, _, gref = O.nf_objective(g, prm, sh, f, mask, vm, vh, Y64, case["centres"], case["d"], cfg.eps)
    assert abs(float(out["loss"].item()) - float(L)) <= FWD_TOL * float(L)
    assert _rel(gp, gref.numpy()) <= GRAD_TOL


def test_nf_recovery_loop_descends_and_graph_matches_eager():
    """The neural-field recovery iteration (Sec. 3.3 with lambda = 0) lowers the
    loss, its first loss equals the oracle's, and the captured CUDA graph
    replays the eager iteration."""
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 1)
    g, sh, f, mask, vm, vh = _oracle_args(cfg)
    Y64, _, _ = O.make_measurement(g, case)
    Y = torch.as_tensor(Y64.numpy().astype(np.complex64), device="cuda")
    pb = pact.Problem(cfg, "cuda")
    prm = inputs.nf_init(6)
    a = NFRecovery(pb, Y, case["d"], cfg.eps, 5e-3, prm, mask)
    b = NFRecovery(pb, Y, case["d"], cfg.eps, 5e-3, prm, mask)
    b.capture()
    ha = a.run(20, record_every=1)
    hb = b.run(20, record_every=1)
    L0, _, _ = O.nf_objective(g, prm.astype(np.float64), sh, f, mask, vm, vh, Y64, case["centres"], case["d"],
                              cfg.eps, False)
    assert abs(ha[0] - float(L0)) <= FWD_TOL * float(L0)
    assert ha[-1] < 0.9 * ha[0]
    assert np.allclose(ha, hb, rtol=1e-3)


# ------------------------------------------------------------------ the paper's SIREN field (FP32)

def _siren_params(seed, w2_scale=20.0):
    p = inputs.siren_init(seed)
    p[768:1024] *= w2_scale                   # a field that varies by tens of m/s
    return p


@pytest.mark.parametrize("cfg", [inputs.config_small(), inputs.config_full()], ids=["G32", "G128"])
def test_siren_forward_and_backward_match_oracle(cfg):
    pb = pact.Problem(cfg, "cuda")
    mask = inputs.sos_mask(cfg)
    prm = _siren_params(1)
    sf = pact.SirenField(pb, prm, mask, inputs.SIREN_OMEGA0)
    v = pact.siren_forward(sf).cpu().numpy()
    g = O.geom(cfg)
    sh = inputs.siren_shapes()
    p64 = O._t(prm).clone().requires_grad_(True)
    ref = O.siren_sos(g, p64, sh, mask, inputs.SIREN_OMEGA0)
    assert np.all(v[~mask] == cfg.v_bg)
    assert _rel(v - 1500.0, ref.detach().numpy() - 1500.0) <= 1e-4
    up = np.random.default_rng(2).standard_normal((cfg.sos_g, cfg.sos_g)).astype(np.float32)
    gp = pact.siren_backward(sf, torch.as_tensor(up, device="cuda")).cpu().numpy()
    (gref,) = torch.autograd.grad((ref * O._t(up)).sum(), p64)
    assert _rel(gp, gref.numpy()) <= 1e-4
    gp2 = pact.siren_backward(sf, torch.as_tensor(up, device="cuda"), torch.as_tensor(gp, device="cuda"),
                              accumulate=True).cpu().numpy()
    assert _rel(gp2, 2.0 * gp) <= 1e-6


def test_siren_objective_gradient_end_to_end_and_recovery():
    """SIREN -> rays -> fused pass -> ray adjoint -> SIREN backward vs the
    oracle's autograd gradient of Eq. 7; the captured recovery loop descends."""
    from paper_2409_10876_gb300.recovery import SirenRecovery
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 0)
    g = O.geom(cfg)
    mask = inputs.sos_mask(cfg)
    Y64, _, _ = O.make_measurement(g, case)
    pb = pact.Problem(cfg, "cuda")
    prm = _siren_params(4)
    sf = pact.SirenField(pb, prm, mask, inputs.SIREN_OMEGA0)
    Y = torch.as_tensor(Y64.numpy().astype(np.complex64), device="cuda")
    sos = pact.siren_forward(sf)
    w = pact.sos_to_delays(pb, sos)
    out = pact.mc_deconv_loss(pb, w, Y, case["d"], cfg.eps)
    gs = pact.sos_to_delays_adj(pb, sos, out["dL_dw"])
    gp = pact.siren_backward(sf, gs).cpu().numpy()
    L, _, gref = O.siren_objective(g, prm.astype(np.float64), inputs.siren_shapes(), mask, inputs.SIREN_OMEGA0, Y64,
                                   case["centres"], case["d"], cfg.eps)
    assert abs(float(out["loss"].item()) - float(L)) <= 1e-4 * float(L)
    assert _rel(gp, gref.numpy()) <= 2e-3
    rec = SirenRecovery(pb, Y, case["d"], cfg.eps, inputs.SIREN_LR, inputs.siren_init(6), mask)
    rec.capture()
    h = rec.run(60, record_every=1)
    assert np.all(np.isfinite(h)) and h[-1] < 0.9 * h[0]


@pytest.mark.parametrize("seed", [0, 1])
def test_nf_field_recovers_on_the_benchmark_workload(seed):
    """The Fourier-feature MLP field at its learning rate (inputs.NF_LR), 1000
    Adam iterations from a uniform 1500 m/s field on phantoms 0 and 1 of the
    benchmark workload: no node's tanh output saturates, the loss falls, and
    on phantom 1 the field reaches the data loss of the true SOS (the noise
    floor) with an SOS error of a few m/s."""
    from paper_2409_10876_gb300.recovery import measurement_spectra
    cfg = inputs.config_full()
    pb = pact.Problem(cfg, "cuda")
    case = inputs.make_case(cfg, seed)
    Y = measurement_spectra(pb, case, "cuda")
    rec = NFRecovery(pb, Y, case["d"], cfg.eps, inputs.NF_LR, inputs.nf_init(seed), case["mask"])
    rec.capture()
    hist = rec.run(1000, record_every=250)
    m = case["mask"].astype(bool)
    sos = rec.sos.cpu().numpy().astype(np.float64)
    t = (sos[m] - inputs.NF_V_MID) / inputs.NF_V_HALF
    assert np.all(np.isfinite(hist)) and np.abs(t).max() < 0.99
    assert min(hist[1:]) < 0.6 * hist[0]
    if seed == 1:
        w_true = pact.sos_to_delays(pb, torch.as_tensor(case["sos_true"], device="cuda"))
        floor = float(pact.mc_deconv_loss(pb, w_true, Y, case["d"], cfg.eps, want_grad=False)["loss"].item())
        rms = float(np.sqrt(np.mean((sos[m] - case["sos_true"][m]) ** 2)))
        # Adam at a constant rate oscillates about the optimum: the best recorded loss
        assert min(hist[1:]) < 1.05 * floor and rms < 3.0, (hist, floor, rms)
