"""What the trained warm-start network gains over the plain method alone.

A CNN is trained on the GPU (library kernels only) on stacks that the forward
model generates from random SOS fields.  On held-out problems the recovery
started from its prediction (warmstart.recover_warm: the warm branch refined
by the plain method, with the plain method from the uniform start as judge and
fallback) must reach 1.01 times the cold run's best loss (1000 iterations from
uniform 1500 m/s) on every problem -- directly, or through the cold branch when
the warm start settles in a worse basin (seen on two or three of six problems
with this small training set) -- and in far fewer iterations overall."""
import numpy as np
import pytest
import torch

from paper_2409_10876_gb300 import inputs, pact, warmstart
from paper_2409_10876_gb300.recovery import measurement_spectra, synthesize_stack

pytestmark = pytest.mark.gpu


def test_warm_start_reaches_the_cold_optimum_sooner():
    cfg = inputs.config_small()
    pb = pact.Problem(cfg, "cuda")
    mask = inputs.sos_mask(cfg)
    gen = warmstart.StackGenerator(pb, cfg, n_ip=2, n_noise=2, seed=1)
    S = 2048
    X = torch.empty((S, cfg.sos_g, cfg.sos_g, pact.cnn_input_channels(cfg.m)), dtype=torch.bfloat16, device="cuda")
    V = torch.empty((S, cfg.sos_g, cfg.sos_g), dtype=torch.float32, device="cuda")
    gen.fill(X, V)
    net = pact.WarmStartCNN(pb, cfg.m, 32, inputs.cnn_init(0, cfg.m), mask)
    hist = warmstart.train(net, X, V, epochs=12, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0]
    net1 = pact.WarmStartCNN(pb, cfg.m, 1, net.params.cpu().numpy(), mask)
    mask_d = torch.as_tensor(mask.astype(np.uint8), device="cuda")
    held_out = cfg.replace(sos_kind="ellipses", sos_lo=1400.0, sos_hi=1650.0)
    results = []
    for seed in range(100, 106):
        case = inputs.make_case(held_out, seed)
        Y = measurement_spectra(pb, case, "cuda")
        v_warm = warmstart.predict(net1, pb, synthesize_stack(pb, case, "cuda"))
        v_cold = torch.full((cfg.sos_g, cfg.sos_g), cfg.v_bg, dtype=torch.float32, device="cuda")
        _, _, h_cold, _ = warmstart.time_to_target(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, v_cold, mask_d,
                                                   -1.0, 1000)
        target = 1.01 * min(h_cold)
        it_cold = 5 * (next(k for k, L in enumerate(h_cold) if L <= target) + 1)   # the loss is read every 5
        r = warmstart.recover_warm(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, v_warm, mask_d, 2000,
                                   target=target)
        assert r["reached_s"] is not None, (seed, r["best"], target, r["fallback"])
        results.append((seed, it_cold, r["iters"]["W"] + r["iters"]["C"], r["branch"], r["fallback"]))
    # every problem reaches the cold optimum (warm, or through the cold branch
    # when the warm start settles in a worse basin), and the warm start saves
    # most of the iterations overall
    tot_cold = sum(r[1] for r in results)
    tot_warm = sum(r[2] for r in results)
    assert tot_warm <= 0.6 * tot_cold, results
    assert sum(r[3] == "warm" for r in results) >= 3, results
