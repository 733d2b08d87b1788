"""Warm-start CNN on BF16 tensor cores (pact_cnn_*) vs the FP64 oracle.

Tolerances: inputs, weights and the activations of five layers are BF16
(relative rounding 2^-9 each), accumulation is FP32; the predicted field
deviation v - v_mid and the parameter gradients are compared at relative L2
3e-2 and 5e-2 (each parameter group at 1e-1)."""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as C
from paper_2409_10876_gb300 import inputs, pact

pytestmark = pytest.mark.gpu

FWD_TOL = 3e-2
GRAD_TOL = 5e-2
GROUP_TOL = 1e-1


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _params(m, seed, head=40.0):
    p = inputs.cnn_init(seed, m)
    p[-65:-1] *= head                         # a head whose output varies by tens of m/s
    return p


def _inputs(cfg, batch, seed):
    """Pooled BF16 inputs built on the host: random stacks through the oracle's
    pooling, rounded to BF16 by torch on the CPU.  Returns (NHWC padded for the
    GPU, NCHW float64 for the oracle)."""
    rng = np.random.default_rng(seed)
    m, cp = cfg.m, pact.cnn_input_channels(cfg.m)
    xs = []
    for _ in range(batch):
        st = rng.standard_normal((m, cfg.img_h, cfg.img_w))
        xs.append(C.pool_stack(st).to(torch.bfloat16))
    x = torch.stack(xs)                                        # [B][m][G][G] bf16
    nhwc = torch.zeros((batch, cfg.sos_g, cfg.sos_g, cp), dtype=torch.bfloat16)
    nhwc[..., :m] = x.permute(0, 2, 3, 1)
    return nhwc.contiguous().cuda(), x.to(torch.float64)


def _groups(m):
    out, o = [], 0
    for name, shape in inputs.cnn_shapes(m):
        n = int(np.prod(shape))
        out.append((name, o, o + n))
        o += n
    return out


CFGS = {"full_m32": inputs.config_full, "small_m8": inputs.config_small}


@pytest.mark.parametrize("name", list(CFGS))
def test_cnn_forward_matches_oracle(name):
    cfg = CFGS[name]()
    pb = pact.Problem(cfg, "cuda")
    mask = inputs.sos_mask(cfg)
    prm = _params(cfg.m, 1)
    net = pact.WarmStartCNN(pb, cfg.m, 2, prm, mask)
    xg, xo = _inputs(cfg, 2, 2)
    v = pact.cnn_forward(net, xg).cpu().numpy()
    pact.cnn_status(net)
    ref = C.cnn_sos(prm.astype(np.float64), inputs.cnn_shapes(cfg.m), inputs.CNN_CONVS, xo, mask,
                    inputs.CNN_V_MID, inputs.CNN_V_HALF, cfg.v_bg).numpy()
    assert np.all(v[:, ~mask] == cfg.v_bg)
    assert ref[:, mask].std() > 5.0                      # the case exercises the head
    assert _rel(v[:, mask] - inputs.CNN_V_MID, ref[:, mask] - inputs.CNN_V_MID) <= FWD_TOL
    assert np.abs(v - ref).max() <= 3.0                  # m/s


@pytest.mark.parametrize("name", list(CFGS))
def test_cnn_loss_and_gradient_match_oracle(name):
    cfg = CFGS[name]()
    pb = pact.Problem(cfg, "cuda")
    mask = inputs.sos_mask(cfg)
    prm = _params(cfg.m, 3)
    B = 2
    net = pact.WarmStartCNN(pb, cfg.m, B, prm, mask)
    xg, xo = _inputs(cfg, B, 4)
    rng = np.random.default_rng(5)
    vt = np.stack([inputs.sos_phantom(inputs.config_cnn().replace(sos_g=cfg.sos_g, img_h=cfg.img_h, img_w=cfg.img_w,
                                                                  dx=cfg.dx), rng) for _ in range(B)])
    vt_d = torch.as_tensor(vt.astype(np.float32), device="cuda")
    sos = pact.cnn_forward(net, xg)
    loss, dsos = pact.cnn_mse(net, sos, vt_d, inputs.CNN_V_SCALE)
    g = pact.cnn_backward(net, xg, dsos).cpu().numpy()
    pact.cnn_status(net)
    L, gref = C.cnn_loss(prm.astype(np.float64), inputs.cnn_shapes(cfg.m), inputs.CNN_CONVS, xo, vt, mask,
                         inputs.CNN_V_MID, inputs.CNN_V_HALF, cfg.v_bg, inputs.CNN_V_SCALE)
    gref = gref.numpy()
    assert abs(float(loss.item()) - float(L)) <= 2 * FWD_TOL * float(L)
    assert _rel(g, gref) <= GRAD_TOL
    for gname, a, b in _groups(cfg.m):
        assert _rel(g[a:b], gref[a:b]) <= GROUP_TOL, gname
    # accumulate adds (onto a copy of the gradient: doubling is exact in FP32)
    g2 = pact.cnn_backward(net, xg, dsos, torch.as_tensor(g, device="cuda"), accumulate=True).cpu().numpy()
    assert _rel(g2, 2.0 * g) <= 1e-6


def test_cnn_pool_stack_matches_oracle():
    cfg = inputs.config_full()
    pb = pact.Problem(cfg, "cuda")
    st = np.random.default_rng(6).standard_normal((cfg.m, cfg.img_h, cfg.img_w)).astype(np.float32)
    x = pact.cnn_pool_stack(pb, torch.as_tensor(st, device="cuda")).float().cpu().numpy()
    ref = C.pool_stack(st.astype(np.float64)).numpy().transpose(1, 2, 0)
    assert x.shape == (cfg.sos_g, cfg.sos_g, 32)
    assert _rel(x, ref) <= 4e-3                          # BF16 rounding of the output


def test_cnn_training_steps_fit_a_small_batch():
    """Adam on the CNN's own kernels (forward, MSE, backward, pact_adam_step)
    lowers the training loss on a fixed batch of generated phantoms."""
    cfg = inputs.config_small()
    pb = pact.Problem(cfg, "cuda")
    mask = inputs.sos_mask(cfg)
    B = 4
    net = pact.WarmStartCNN(pb, cfg.m, B, inputs.cnn_init(7, cfg.m), mask)
    xg, _ = _inputs(cfg, B, 8)
    rng = np.random.default_rng(9)
    vt = np.stack([inputs.sos_phantom(cfg.replace(sos_kind="ellipses", sos_lo=1400.0, sos_hi=1650.0), rng)
                   for _ in range(B)]).astype(np.float32)
    vt_d = torch.as_tensor(vt, device="cuda")
    m1, m2 = torch.zeros_like(net.params), torch.zeros_like(net.params)
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    hist = []
    for _ in range(60):
        sos = pact.cnn_forward(net, xg)
        loss, dsos = pact.cnn_mse(net, sos, vt_d, inputs.CNN_V_SCALE)
        g = pact.cnn_backward(net, xg, dsos)
        pact.adam_step(net.params, g, m1, m2, 1, 2e-3, 0.9, 0.999, 1e-8, step_counter=cnt)
        hist.append(float(loss.item()))
    pact.cnn_status(net)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.5 * hist[0]
