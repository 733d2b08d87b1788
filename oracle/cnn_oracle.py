"""FP64 CPU oracle of the warm-start CNN (learned SOS initialiser).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module; the
product path never calls it and shares no code with it.

The paper recovers the SOS by test-time optimisation alone (Sec. 3.3); the
warm start is a learned addition: a small convolutional network maps the
delay stack of Eq. 1 / Eq. 5 (the "focal stack" of Sec. 3.2) to an SOS map
from which the plain optimisation starts.  What it computes, literally:

* input: the M x H x W delay stack averaged over 4 x 4 pixel blocks and
  divided by its root-mean-square value                     -> pool_stack
* five 3x3 convolutions (zero padding 1) with ReLU; 2x2 average pooling
  after the first two                                        -> cnn_features
* a 1x1 head z = w6 . h + b6 and v32 = v_mid + v_half tanh(z)   (32 x 32)
* bilinear upsampling x4 to the 128 x 128 node grid, sample positions
  (q + 0.5) / 4 - 0.5 clamped to the grid, and v_bg outside the SOS mask
                                                             -> upsample4, cnn_sos
* training loss: mean over samples and mask nodes of ((v - v_true) / 100)^2
                                                             -> cnn_loss

Library routines serve as steps (conv2d, avg_pool2d); gradients come from
autograd and are pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn

DT = torch.float64


def _t(x, dtype=DT):
    if isinstance(x, torch.Tensor):
        return x.to(dtype)
    return torch.as_tensor(np.asarray(x), dtype=dtype)


def unflatten(params, shapes):
    out, o = {}, 0
    for name, shape in shapes:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def pool_stack(stack, f: int = 4) -> torch.Tensor:
    """[M][H][W] delay stack -> [M][H/f][W/f]: f x f block means divided by the
    root-mean-square of the pooled stack."""
    s = _t(stack)
    m, h, w = s.shape
    p = s.reshape(m, h // f, f, w // f, f).mean(dim=(2, 4))
    rms = torch.sqrt((p * p).mean())
    return p / (rms + 1e-12)


def cnn_features(p, x, convs) -> torch.Tensor:
    """Hidden activations after the five convolutions: x [B][C][128][128] ->
    [B][64][32][32]."""
    h = x
    for l, (_, _, pool) in enumerate(convs, start=1):
        h = torch.relu(Fn.conv2d(h, p[f"W{l}"], p[f"b{l}"], padding=1))
        if pool:
            h = Fn.avg_pool2d(h, 2)
    return h


def upsample4(v) -> torch.Tensor:
    """Bilinear x4 upsampling [B][n][n] -> [B][4n][4n]: output node q samples
    input position (q + 0.5)/4 - 0.5, clamped to [0, n - 1]."""
    n = v.shape[-1]
    q = torch.arange(4 * n, dtype=DT)
    src = torch.clamp((q + 0.5) / 4.0 - 0.5, 0.0, n - 1.0)
    i0 = torch.floor(src).long()
    i1 = torch.clamp(i0 + 1, max=n - 1)
    t = src - i0.to(DT)
    rows = v[:, i0, :] * (1 - t)[None, :, None] + v[:, i1, :] * t[None, :, None]
    return rows[:, :, i0] * (1 - t)[None, None, :] + rows[:, :, i1] * t[None, None, :]


def cnn_sos(params, shapes, convs, x, mask, v_mid: float, v_half: float, v_bg: float):
    """SOS maps [B][4n][4n] predicted from pooled stacks x [B][C][H][W];
    params may require grad."""
    p = unflatten(_t(params) if not isinstance(params, torch.Tensor) else params, shapes)
    h = cnn_features(p, _t(x), convs)
    z = torch.einsum("bchw,c->bhw", h, p["w6"]) + p["b6"][0]
    v = upsample4(v_mid + v_half * torch.tanh(z))
    m = _t(mask) > 0
    return torch.where(m[None], v, torch.full_like(v, v_bg))


def cnn_loss(params, shapes, convs, x, v_true, mask, v_mid, v_half, v_bg, v_scale: float = 100.0,
             want_grad: bool = True):
    """Training loss mean_{b, mask} ((v_b - v_true_b) / v_scale)^2 and its
    gradient with respect to the flat parameters."""
    prm = _t(params).clone().requires_grad_(want_grad)
    v = cnn_sos(prm, shapes, convs, x, mask, v_mid, v_half, v_bg)
    m = _t(mask) > 0
    r = (v - _t(v_true)) / v_scale
    L = (r * r)[:, m].mean()
    if not want_grad:
        return L.detach(), None
    (g,) = torch.autograd.grad(L, prm)
    return L.detach(), g
