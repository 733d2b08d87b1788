"""Pins of the FP64 warm-start CNN oracle against brute force, library routines
other than the ones it uses, closed forms and finite differences."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

from oracle import cnn_oracle as C
from paper_2409_10876_gb300 import inputs

SH = inputs.cnn_shapes(4)
CONVS = inputs.CNN_CONVS


def _x(seed, b=2, m=4, n=16):
    return torch.as_tensor(np.random.default_rng(seed).standard_normal((b, m, n, n)))


def test_conv_step_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 5, 6))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    p = {"W1": torch.as_tensor(w), "b1": torch.as_tensor(b)}
    got = C.cnn_features(p, torch.as_tensor(x), ((2, 3, False),))[0].numpy()
    ref = np.zeros((3, 5, 6))
    for o in range(3):
        for r in range(5):
            for c in range(6):
                s = b[o]
                for i in range(2):
                    for dy in range(3):
                        for dx in range(3):
                            rr, cc = r + dy - 1, c + dx - 1
                            if 0 <= rr < 5 and 0 <= cc < 6:
                                s += w[o, i, dy, dx] * x[0, i, rr, cc]
                ref[o, r, c] = max(s, 0.0)
    assert np.allclose(got, ref, atol=1e-12)


def test_avg_pool_step_is_block_mean():
    x = _x(1, b=1, m=3, n=8)
    p = {"W1": torch.zeros(3, 3, 3, 3, dtype=torch.float64), "b1": torch.zeros(3, dtype=torch.float64)}
    for k in range(3):
        p["W1"][k, k, 1, 1] = 1.0                  # identity convolution
    got = C.cnn_features(p, x, ((3, 3, True),))
    ref = torch.relu(x).reshape(1, 3, 4, 2, 4, 2).mean(dim=(3, 5))
    assert torch.allclose(got, ref, atol=1e-14)


def test_upsample4_matches_library_bilinear_and_keeps_affine_fields():
    v = torch.as_tensor(np.random.default_rng(2).standard_normal((2, 8, 8)))
    ref = Fn.interpolate(v[:, None], scale_factor=4, mode="bilinear", align_corners=False)[:, 0]
    assert torch.allclose(C.upsample4(v), ref, atol=1e-13)
    ii, jj = torch.meshgrid(torch.arange(8.0, dtype=torch.float64), torch.arange(8.0, dtype=torch.float64),
                            indexing="ij")
    a = (3.0 + 0.5 * ii - 0.25 * jj)[None]
    up = C.upsample4(a)[0]
    q = (torch.arange(32.0, dtype=torch.float64) + 0.5) / 4 - 0.5
    exact = 3.0 + 0.5 * q[:, None] - 0.25 * q[None, :]
    inner = slice(2, 30)                              # away from the clamped border
    assert torch.allclose(up[inner, inner], exact[inner, inner], atol=1e-13)


def test_pool_stack_constant_and_scale_invariance():
    s = np.full((3, 16, 16), 2.5)
    assert torch.allclose(C.pool_stack(s), torch.ones(3, 4, 4, dtype=torch.float64))
    r = np.random.default_rng(3).standard_normal((3, 16, 16))
    assert torch.allclose(C.pool_stack(r), C.pool_stack(7.0 * r), atol=1e-12)
    blk = r.reshape(3, 4, 4, 4, 4).mean(axis=(2, 4))
    assert np.allclose(C.pool_stack(r).numpy() * np.sqrt((blk ** 2).mean()), blk)


def test_zero_weights_give_constant_head_output():
    prm = np.zeros(inputs.cnn_param_count(4))
    prm[-1] = 0.3
    mask = np.zeros((16, 16), np.uint8)
    mask[4:12, 4:12] = 1
    v = C.cnn_sos(prm, SH, CONVS, _x(4, n=16), mask, 1525.0, 125.0, 1500.0)
    assert v.shape == (2, 16, 16)
    assert torch.allclose(v[:, 4:12, 4:12], torch.full((2, 8, 8), 1525.0 + 125.0 * np.tanh(0.3), dtype=torch.float64))
    assert torch.all(v[:, :4] == 1500.0)


def test_init_starts_near_v_start():
    prm = inputs.cnn_init(0, 4)
    mask = np.ones((16, 16), np.uint8)
    v = C.cnn_sos(prm.astype(np.float64), SH, CONVS, _x(5, n=16), mask, 1525.0, 125.0, 1500.0)
    assert abs(float(v.mean()) - 1500.0) < 5.0


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    prm = inputs.cnn_init(1, 4).astype(np.float64)
    prm[-2 - 64:-1] *= 50.0                           # a head that actually moves v
    x = _x(7, n=16)
    mask = np.ones((16, 16), np.uint8)
    mask[0] = 0
    v_true = 1500.0 + 40.0 * rng.standard_normal((2, 16, 16))
    args = (SH, CONVS, x, v_true, mask, 1525.0, 125.0, 1500.0)
    L, g = C.cnn_loss(prm, *args)
    idx = rng.choice(prm.size, 24, replace=False)
    h = 1e-6
    for k in idx:
        pp, pm = prm.copy(), prm.copy()
        pp[k] += h
        pm[k] -= h
        fd = (float(C.cnn_loss(pp, *args, want_grad=False)[0]) - float(C.cnn_loss(pm, *args, want_grad=False)[0])) / (2 * h)
        gk = float(g[k].item())
        assert abs(fd - gk) <= 1e-6 * max(1.0, abs(fd)) + 1e-7 * float(g.abs().max()), (k, fd, gk)
