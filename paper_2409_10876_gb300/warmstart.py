"""Warm-start SOS from a learned network, refined by the plain method.

The paper's recovery (Sec. 3.3) starts every optimisation from a uniform SOS.
Here a small CNN (pact_cnn_*, BF16 tensor cores) predicts a starting SOS map
from the delay stack, and the plain pixel-grid optimisation refines it and
has the last word: the warm start only changes where Adam starts.

Training data are generated on the GPU by the library's own forward model:
a random SOS field (1-6 Gaussian ellipses, 1400-1650 m/s) gives the
wavefront errors (Eq. 2-3); a vessel-tree initial pressure gives patch
spectra X; Y = H(v) X (Eq. 5) is stitched channel by channel into the delay
stack (Sec. S1.5), a seeded noise stack is added, and the stack is pooled
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
        assert self.sos_cfg.sos_kind == "ellipses"
        self.ws_stitch = pact._ws(pact.load().pact_stitch_channels_workspace_size(pb.gp(), pb.pp(), cfg.m), dev)
        self.ws_pool = pact._ws(pact.load().pact_cnn_pool_workspace_size(pb.gp(), cfg.m), dev)
        self.Yc = torch.empty(pb.spectra_shape(cfg.m), dtype=torch.complex64, device=dev)
        self.stack = torch.empty((cfg.m, cfg.img_h, cfg.img_w), dtype=torch.float32, device=dev)
        self.w = torch.empty((pb.n, pb.n_t), dtype=torch.float32, device=dev)

    def stack_of(self, sos: torch.Tensor, X: torch.Tensor, noise: torch.Tensor) -> torch.Tensor:
        """Delay stack [M, H, W] of Eq. 5: stitch(H(v) X) + noise."""
        pb = self.pb
        pact.sos_to_delays(pb, sos, self.w)
        pact.forward_model(pb, self.w, self.d, X, self.Yc)
        pact.stitch_channels(pb, self.Yc, self.stack, ws=self.ws_stitch)
        self.stack += noise
        return self.stack

    def fill(self, x_out: torch.Tensor, v_out: torch.Tensor, first: int = 0, chunk: int = 512) -> None:
        """Writes samples first .. len(x_out)-1 of a dataset: x_out [S, G, G, Cp]
        BF16, v_out [S, G, G] float32.  The phantoms' parameters are drawn on
        the host (seeded) and the phantoms evaluated on the device in chunks."""
        S = x_out.shape[0]
        dev = self.pb.device
        for c0 in range(first, S, chunk):
            c1 = min(S, c0 + chunk)
            params, picks = [], []
            for _ in range(c0, c1):
                params.append(inputs.ellipse_params(self.sos_cfg, self.rng))
                picks.append((int(self.rng.integers(len(self.X))), int(self.rng.integers(len(self.noise)))))
            V = inputs.ellipse_phantoms_batch(self.sos_cfg, params, dev)
            for k, s in enumerate(range(c0, c1)):
                xi, ni = picks[k]
                st = self.stack_of(V[k], self.X[xi], self.noise[ni])
                pact.cnn_pool_stack(self.pb, st, x_out[s], ws=self.ws_pool)
            v_out[c0:c1].copy_(V)


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


def recover_warm(pb, Y, d, eps, lam, lr, v_warm, mask, iters: int, target: float = None, ratio: int = 4,
                 check_every: int = 5, window: int = 50, tol: float = 2e-3):
    """Warm-started plain recovery with the plain method as judge and fallback.

    Two recoveries run side by side on the GPU (each one CUDA graph per
    iteration): W from the network's SOS `v_warm`, C from the uniform SOS of
    the paper's method (Sec. 3.3).  The self-supervised loss (Eq. 7) judges
    them; no ground truth is used:
      * if the loss at the warm start is not below the loss at the uniform
        start, W is dropped at once (fallback to C);
      * while W improves it takes `ratio` iterations for each one of C;
      * once W's loss improves by less than `tol` (relative) over `window`
        of its iterations, W pauses and C takes every iteration;
      * C stops when it too has settled above W's best loss; W is dropped if
        C goes below its best loss.
    `iters` bounds the iterations of both branches together.  With `target`,
    the run stops as soon as either branch's loss is at most `target`.
    Returns a dict: 'sos' (the better branch's SOS), 'branch', 'fallback'
    (why W was dropped, or None), 'iters' {W, C}, 'hist' [(seconds, W its,
    C its, W loss, C loss)], 'reached_s' (seconds to target, or None)."""
    dev = Y.device
    W = PGRecovery(pb, Y, d, eps, lam, lr, v_warm, mask)
    C = PGRecovery(pb, Y, d, eps, lam, lr, torch.full_like(v_warm, pb.cfg.v_bg), mask)
    W.capture()
    C.capture()
    torch.cuda.synchronize(dev)
    its = {"W": 0, "C": 0}
    best = {"W": float("inf"), "C": float("inf")}
    track = {"W": [], "C": []}                    # (iterations, loss) per branch
    state = {"W": "run", "C": "run"}              # run | paused | dropped | settled
    fallback, hist, reached = None, [], None

    def settled(b):
        tr = track[b]
        if not tr:
            return False
        old = next((L for k, L in reversed(tr) if k <= tr[-1][0] - window), None)
        return old is not None and old - tr[-1][1] < tol * abs(old)

    t0 = time.perf_counter()
    while its["W"] + its["C"] < iters:
        share = {"W": check_every if state["W"] == "run" else 0,
                 "C": (max(1, check_every // ratio) if state["W"] == "run" else check_every)
                 if state["C"] == "run" else 0}
        if share["W"] + share["C"] == 0:
            break
        for b, rec in (("W", W), ("C", C)):
            for _ in range(share[b]):
                rec.iterate()
            its[b] += share[b]
        lw, lc = W.loss(), C.loss()
        el = time.perf_counter() - t0
        hist.append((el, its["W"], its["C"], lw, lc))
        for b, L in (("W", lw), ("C", lc)):
            if share[b]:
                track[b].append((its[b], L))
                if np.isfinite(L):
                    best[b] = min(best[b], L)
        if target is not None and reached is None and min(best.values()) <= target:
            reached = el
            break
        if fallback is None and len(hist) == 1 and not (lw < lc):      # losses of the first iterations:
            fallback = "the loss at the warm start is not below the loss at the uniform start"
        if fallback is None and not np.isfinite(lw):
            fallback = "non-finite loss on the warm branch"
            best["W"] = float("inf")             # its state is no longer usable
        if fallback is not None:
            state["W"] = "dropped"
        if state["W"] == "run" and settled("W"):
            state["W"] = "paused"
        if state["W"] != "dropped" and best["C"] < best["W"]:
            state["W"] = "dropped"
            fallback = fallback or "the cold branch went below the warm branch's best loss"
        if state["W"] != "run" and state["C"] == "run" and settled("C") and best["C"] >= best["W"]:
            state["C"] = "settled"
    branch = "W" if best["W"] <= best["C"] else "C"
    rec = W if branch == "W" else C
    return {"sos": rec.sos.clone(), "branch": "warm" if branch == "W" else "cold", "fallback": fallback,
            "iters": dict(its), "best": dict(best), "hist": hist, "reached_s": reached,
            "seconds": time.perf_counter() - t0}
