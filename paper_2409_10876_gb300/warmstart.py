"""Warm-start SOS from a learned network, refined by the plain method.

The paper's recovery (Sec. 3.3) starts every optimisation from a uniform SOS.
Here a small CNN (pact_cnn_*, BF16 tensor cores) predicts a starting SOS map
from the delay stack, and the plain pixel-grid optimisation refines it and
has the last word: the warm start only changes where Adam starts.

Training data are generated on the GPU by the library's own forward model:
a random SOS field (1-6 Gaussian ellipses, 1400-1650 m/s) gives the
wavefront errors (Eq. 2-3); a vessel-tree initial pressure gives patch
spectra X; Y = H(v) X (Eq. 5) is stitched channel by channel into the delay
stack (Sec. S1.4), a seeded noise stack is added, and the stack is pooled
into the network input.  The target is the SOS field itself.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import inputs, pact
from .recovery import PGRecovery


class StackGenerator:
    """Seeded synthetic (pooled stack, SOS) pairs for one problem geometry.

    `n_ip` vessel-tree images are drawn once on the host; each is used in its
    eight orientations (rotations by 90 degrees and mirror images), so the
    generator holds 8 n_ip clean spectra X.  `n_noise` seeded noise stacks are
    kept on the device and drawn at random per sample."""

    def __init__(self, pb: "pact.Problem", cfg: "inputs.Config", n_ip: int = 4, n_noise: int = 2, seed: int = 0):
        self.pb, self.cfg = pb, cfg
        self.d = cfg.delays()
        self.rng = np.random.Generator(np.random.PCG64(seed))
        dev = pb.device
        self.X = []
        for _ in range(n_ip):
            ip = inputs.ip_phantom(cfg, self.rng)
            for k in range(4):
                for flip in (False, True):
                    img = np.rot90(ip, k)
                    img = img[:, ::-1] if flip else img
                    t = torch.as_tensor(np.ascontiguousarray(img, np.float32), device=dev)[None]
                    self.X.append(pact.patch_fft(pb, t)[:, 0].contiguous())
        self.noise = [torch.as_tensor(self.rng.standard_normal((cfg.m, cfg.img_h, cfg.img_w), np.float32)
                                      * np.float32(cfg.noise_sigma), device=dev) for _ in range(n_noise)]
        self.sos_cfg = inputs.config_cnn().replace(img_h=cfg.img_h, img_w=cfg.img_w, dx=cfg.dx, sos_g=cfg.sos_g,
                                                   n_t=cfg.n_t, ring_radius=cfg.ring_radius)
        self.ws_stitch = pact._ws(pact.load().pact_stitch_channels_workspace_size(pb.gp(), pb.pp(), cfg.m), dev)
        self.ws_pool = pact._ws(pact.load().pact_cnn_pool_workspace_size(pb.gp(), cfg.m), dev)
        self.Yc = torch.empty(pb.spectra_shape(cfg.m), dtype=torch.complex64, device=dev)
        self.stack = torch.empty((cfg.m, cfg.img_h, cfg.img_w), dtype=torch.float32, device=dev)
        self.w = torch.empty((pb.n, pb.n_t), dtype=torch.float32, device=dev)

    def sos(self) -> np.ndarray:
        return inputs.sos_phantom(self.sos_cfg, self.rng).astype(np.float32)

    def stack_of(self, sos: torch.Tensor, X: torch.Tensor, noise: torch.Tensor) -> torch.Tensor:
        """Delay stack [M, H, W] of Eq. 5: stitch(H(v) X) + noise."""
        pb = self.pb
        pact.sos_to_delays(pb, sos, self.w)
        pact.forward_model(pb, self.w, self.d, X, self.Yc)
        pact.stitch_channels(pb, self.Yc, self.stack, ws=self.ws_stitch)
        self.stack += noise
        return self.stack

    def fill(self, x_out: torch.Tensor, v_out: torch.Tensor, first: int = 0) -> None:
        """Writes samples first .. len(x_out)-1 of a dataset: x_out [S, G, G, Cp]
        BF16, v_out [S, G, G] float32."""
        for s in range(first, x_out.shape[0]):
            v = torch.as_tensor(self.sos(), device=self.pb.device)
            X = self.X[int(self.rng.integers(len(self.X)))]
            nz = self.noise[int(self.rng.integers(len(self.noise)))]
            st = self.stack_of(v, X, nz)
            pact.cnn_pool_stack(self.pb, st, x_out[s], ws=self.ws_pool)
            v_out[s].copy_(v)


def train(net: "pact.WarmStartCNN", x_all: torch.Tensor, v_all: torch.Tensor, epochs: int, lr: float = 1e-3,
          seed: int = 0, graph: bool = True, log=None):
    """Adam on the network parameters over shuffled batches of (x_all, v_all),
    every step on the library's kernels (forward, loss, backward, Adam), one
    captured CUDA graph per step.  Returns the per-epoch mean losses."""
    dev = net.params.device
    B = net.batch
    S = x_all.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    xb = torch.empty((B,) + tuple(x_all.shape[1:]), dtype=x_all.dtype, device=dev)
    vb = torch.empty((B,) + tuple(v_all.shape[1:]), dtype=v_all.dtype, device=dev)
    m1, m2 = torch.zeros_like(net.params), torch.zeros_like(net.params)
    cnt = torch.zeros(2, dtype=torch.int32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    grad = torch.zeros_like(net.params)
    sos = torch.empty_like(vb)
    dsos = torch.empty_like(vb)
    lsum = torch.zeros(1, dtype=torch.float32, device=dev)

    def step():
        pact.cnn_forward(net, xb, sos)
        pact.cnn_mse(net, sos, vb, inputs.CNN_V_SCALE, loss, dsos)
        pact.cnn_backward(net, xb, dsos, grad)
        pact.adam_step(net.params, grad, m1, m2, 1, lr, 0.9, 0.999, 1e-8, step_counter=cnt)
        lsum.add_(loss)

    g = None
    if graph:
        xb.copy_(x_all[:B])
        vb.copy_(v_all[:B])
        st0 = [t.clone() for t in (net.params, m1, m2, cnt)]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()
        torch.cuda.current_stream().wait_stream(s)
        for dst, src in zip((net.params, m1, m2, cnt), st0):
            dst.copy_(src)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
    hist = []
    nb = S // B
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(S)[:nb * B], device=dev)
        lsum.zero_()
        for b in range(nb):
            idx = perm[b * B:(b + 1) * B]
            torch.index_select(x_all, 0, idx, out=xb)
            torch.index_select(v_all, 0, idx, out=vb)
            if g is not None:
                g.replay()
            else:
                step()
        hist.append(float(lsum.item()) / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    pact.cnn_status(net)
    return hist


def predict(net1: "pact.WarmStartCNN", pb: "pact.Problem", stack: torch.Tensor) -> torch.Tensor:
    """Warm-start SOS [G, G] of one delay stack (network with batch 1)."""
    x = pact.cnn_pool_stack(pb, stack)[None]
    return pact.cnn_forward(net1, x)[0]


def time_to_target(pb, Y, d, eps, lam, lr, sos0, mask, target: float, max_iters: int, check_every: int = 5):
    """Runs the plain recovery (one CUDA graph per iteration) from sos0 until
    the loss is at most `target`; returns (iterations, GPU seconds, loss
    history).  The loss is read every `check_every` iterations."""
    rec = PGRecovery(pb, Y, d, eps, lam, lr, sos0, mask)
    rec.capture()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    it, hist = 0, []
    reached = None
    while it < max_iters:
        for _ in range(check_every):
            rec.iterate()
        it += check_every
        L = rec.loss()
        hist.append(L)
        if L <= target:
            reached = it
            break
    ev1.record()
    torch.cuda.synchronize()
    return reached, ev0.elapsed_time(ev1) * 1e-3, hist, rec
