"""Recovery loop on the GPU (Sec. 3.3) and autograd wrappers.

``PGRecovery`` runs the plain method with the pixel-grid SOS: every iteration
is  sos_to_delays (Eq. 3) -> fused mc_deconv_loss + adjoint (Eq. 4-7) ->
sos_to_delays_adj -> TV value/subgradient -> Adam, all in libpact kernels,
captured once into a CUDA graph and replayed.  The loss stays on the device
and is read back only when asked.

``SosToDelays`` and ``McDeconvLoss`` expose the forward calls and their
hand-written adjoints to torch.autograd for users who compose the forward
model with their own parametrisations.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import checkpoint, pact


class SosToDelays(torch.autograd.Function):
    """w = sos_to_delays(sos) (Eq. 3); backward = pact_sos_to_delays_adj."""

    @staticmethod
    def forward(ctx, pb, sos):
        ctx.pb = pb
        ctx.save_for_backward(sos)
        return pact.sos_to_delays(pb, sos.contiguous())

    @staticmethod
    def backward(ctx, gw):
        (sos,) = ctx.saved_tensors
        return None, pact.sos_to_delays_adj(ctx.pb, sos.contiguous(), gw.contiguous())


class McDeconvLoss(torch.autograd.Function):
    """Eq. 6-7 data term as a function of w; backward = pact_mc_deconv_loss_adj
    (X_hat recomputed, never stored)."""

    @staticmethod
    def forward(ctx, pb, w, Y, d, eps):
        ctx.pb, ctx.d, ctx.eps = pb, np.asarray(d, np.float32), float(eps)
        ctx.save_for_backward(w, Y)
        out = pact.mc_deconv_loss(pb, w.contiguous(), Y, d, eps, want_grad=False)
        return out["loss"].reshape(())

    @staticmethod
    def backward(ctx, gl):
        w, Y = ctx.saved_tensors
        gw = pact.mc_deconv_loss_adj(ctx.pb, w.contiguous(), Y, ctx.d, ctx.eps,
                                     dL_dloss=gl.reshape(1).float().contiguous())
        return None, gw, None, None, None


class PGRecovery:
    """Plain method, pixel-grid SOS (Sec. 3.3), one CUDA graph per iteration."""

    def __init__(self, pb: "pact.Problem", Y: torch.Tensor, d, eps: float, lam: float, lr: float,
                 sos_init: torch.Tensor, mask: torch.Tensor = None, betas=(0.9, 0.999), adam_eps=1e-8):
        dev = Y.device
        self.pb, self.Y, self.d = pb, Y, np.asarray(d, np.float32)
        self.eps, self.lam, self.lr, self.betas, self.adam_eps = float(eps), float(lam), float(lr), betas, adam_eps
        self.m = int(Y.shape[1])
        self.sos = sos_init.to(dev, torch.float32).contiguous().clone()
        self.mask = None if mask is None else mask.to(dev, torch.uint8).contiguous()
        self.adam_m = torch.zeros_like(self.sos)
        self.adam_v = torch.zeros_like(self.sos)
        self.counter = torch.zeros(2, dtype=torch.int32, device=dev)
        self.w = torch.empty((pb.n, pb.n_t), dtype=torch.float32, device=dev)
        self.grad = torch.empty_like(self.sos)
        self.out = {"loss": torch.zeros(1, dtype=torch.float32, device=dev),
                    "dL_dw": torch.zeros((pb.n, pb.n_t), dtype=torch.float32, device=dev)}
        self.tables = pact.McdTables(pb, self.d, dev)       # geometry/delay tables, built once
        self.ws_mcd = pact._ws(self.tables.scratch_bytes, dev)
        self.ws_adj = pact._ws(pact.sos_to_delays_adj_workspace_size(pb), dev)
        self.ws_tv = pact._ws(pact.sos_to_delays_tv_workspace_size(pb), dev) if self.lam != 0.0 else None
        self.graph = None

    # one iteration, enqueued on the current stream: four kernels -- rays (with
    # the clearing of dL/dw and the TV terms), the fused pass, the ray adjoint,
    # and one tail kernel (partial-grid sum + TV subgradient + Adam).  `mark(k)`,
    # if given, is called between the parts (k = 0 start, 1 after the rays, 2
    # after the fused pass, 4 after the ray adjoint and Adam, 3 end).
    def step(self, mark=None):
        pb = self.pb
        mark = mark or (lambda k: None)
        mark(0)
        if self.ws_tv is not None:
            pact.sos_to_delays_tv(pb, self.sos, self.w, self.out["dL_dw"], self.lam, self.ws_tv)
        else:
            pact.sos_to_delays(pb, self.sos, self.w, clear=self.out["dL_dw"])
        mark(1)
        pact.mc_deconv_loss(pb, self.w, self.Y, self.d, self.eps, want_grad=True, out=self.out, ws=self.ws_mcd,
                            tables=self.tables, accumulate=True)
        mark(2)
        pact.sos_to_delays_adj_adam(pb, self.sos, self.out["dL_dw"], self.adam_m, self.adam_v, self.lr,
                                    self.betas[0], self.betas[1], self.adam_eps, mask=self.mask,
                                    step_counter=self.counter, tv_ws=self.ws_tv, loss=self.out["loss"],
                                    grad=self.grad, ws=self.ws_adj)
        mark(4)
        mark(3)

    def state(self):
        return [t.clone() for t in (self.sos, self.adam_m, self.adam_v, self.counter)]

    def set_state(self, st):
        for dst, src in zip((self.sos, self.adam_m, self.adam_v, self.counter), st):
            dst.copy_(src)

    STATE_NAMES = ("sos", "adam_m", "adam_v", "counter")

    def checkpoint(self, path: str, iteration: int, seed: int, cfg_hash: str) -> None:
        """Saves the state a run needs to continue (parameters, Adam moments and
        step counter), with the iteration, the seed and the configuration hash."""
        arrays = {n: t.detach().cpu().numpy() for n, t in zip(self.STATE_NAMES, self.state())}
        checkpoint.save(path, arrays, {"iteration": int(iteration), "seed": int(seed), "config_hash": cfg_hash,
                                       "lr": self.lr, "lam": self.lam, "eps": self.eps, "kind": type(self).__name__})

    def resume(self, path: str, cfg_hash: str) -> dict:
        """Restores a checkpoint made by checkpoint() for the same configuration
        hash and recovery kind; returns its metadata (iteration, seed, ...)."""
        arrays, meta = checkpoint.load(path, cfg_hash)
        if meta.get("kind") != type(self).__name__:
            raise checkpoint.CheckpointError(f"{path}: a {meta.get('kind')} checkpoint, not {type(self).__name__}")
        cur = self.state()
        st = []
        for n, t in zip(self.STATE_NAMES, cur):
            a = arrays.get(n)
            if a is None or tuple(a.shape) != tuple(t.shape) or str(a.dtype) != str(t.dtype).replace("torch.", ""):
                raise checkpoint.CheckpointError(f"{path}: array {n} missing or of another shape/type")
            st.append(torch.as_tensor(a))
        self.set_state([x.to(t.device) for x, t in zip(st, cur)])
        return meta

    def capture(self):
        """Captures one iteration into a CUDA graph (after one eager warm-up
        iteration whose effect on the state is undone)."""
        st0 = self.state()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.set_state(st0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g
        torch.cuda.synchronize()
        return g

    def iterate(self):
        if self.graph is None:
            self.step()
        else:
            self.graph.replay()

    def run(self, iters: int, record_every: int = 0):
        hist = []
        for it in range(iters):
            self.iterate()
            if record_every and (it % record_every == 0 or it == iters - 1):
                hist.append(self.loss())
        return hist

    def loss(self) -> float:
        """Eq. 7 at the SOS the last iteration started from: data term + lambda TV."""
        return float(self.out["loss"].item())


class NFRecovery(PGRecovery):
    """Neural-field SOS (Sec. 3.3, lambda = 0): Adam on the field's parameters;
    every iteration is nf_forward -> sos_to_delays -> fused deconvolution/loss/
    adjoint -> sos_to_delays_adj -> nf_backward -> Adam, one CUDA graph."""

    STATE_NAMES = ("params", "adam_m", "adam_v", "counter")

    def __init__(self, pb: "pact.Problem", Y: torch.Tensor, d, eps: float, lr: float, params,
                 mask=None, betas=(0.9, 0.999), adam_eps=1e-8, v_mid: float = 1525.0, v_half: float = 125.0):
        dev = Y.device
        self.nf = pact.NeuralField(pb, params, mask, v_mid, v_half)
        super().__init__(pb, Y, d, eps, 0.0, lr, torch.zeros(pb.g, pb.g), None, betas, adam_eps)
        self.params = self.nf.params
        self.adam_m = torch.zeros_like(self.params)
        self.adam_v = torch.zeros_like(self.params)
        self.gparams = torch.zeros_like(self.params)

    def step(self):
        pb = self.pb
        pact.nf_forward(self.nf, self.sos)
        pact.sos_to_delays(pb, self.sos, self.w, clear=self.out["dL_dw"])
        pact.mc_deconv_loss(pb, self.w, self.Y, self.d, self.eps, want_grad=True, out=self.out, ws=self.ws_mcd,
                            tables=self.tables, accumulate=True)
        pact.sos_to_delays_adj(pb, self.sos, self.out["dL_dw"], self.grad, accumulate=False, ws=self.ws_adj)
        pact.nf_backward(self.nf, self.grad, self.gparams)
        pact.adam_step(self.params, self.gparams, self.adam_m, self.adam_v, 1, self.lr, self.betas[0],
                       self.betas[1], self.adam_eps, step_counter=self.counter)

    def state(self):
        return [t.clone() for t in (self.params, self.adam_m, self.adam_v, self.counter)]

    def set_state(self, st):
        for dst, src in zip((self.params, self.adam_m, self.adam_v, self.counter), st):
            dst.copy_(src)


class SirenRecovery(PGRecovery):
    """The paper's neural field (SIREN, Sec. 3.3, lambda = 0): Adam on its 1027
    parameters; every iteration is siren_forward -> sos_to_delays -> fused
    deconvolution/loss/adjoint -> sos_to_delays_adj -> siren_backward -> Adam,
    one CUDA graph."""

    STATE_NAMES = ("params", "adam_m", "adam_v", "counter")

    def __init__(self, pb: "pact.Problem", Y: torch.Tensor, d, eps: float, lr: float, params, mask=None,
                 betas=(0.9, 0.999), adam_eps=1e-8, omega0: float = 30.0):
        self.sf = pact.SirenField(pb, params, mask, omega0)
        super().__init__(pb, Y, d, eps, 0.0, lr, torch.zeros(pb.g, pb.g), None, betas, adam_eps)
        self.params = self.sf.params
        self.adam_m = torch.zeros_like(self.params)
        self.adam_v = torch.zeros_like(self.params)
        self.gparams = torch.zeros_like(self.params)

    def step(self):
        pb = self.pb
        pact.siren_forward(self.sf, self.sos)
        pact.sos_to_delays(pb, self.sos, self.w, clear=self.out["dL_dw"])
        pact.mc_deconv_loss(pb, self.w, self.Y, self.d, self.eps, want_grad=True, out=self.out, ws=self.ws_mcd,
                            tables=self.tables, accumulate=True)
        pact.sos_to_delays_adj(pb, self.sos, self.out["dL_dw"], self.grad, accumulate=False, ws=self.ws_adj)
        pact.siren_backward(self.sf, self.grad, self.gparams)
        pact.adam_step(self.params, self.gparams, self.adam_m, self.adam_v, 1, self.lr, self.betas[0],
                       self.betas[1], self.adam_eps, step_counter=self.counter)

    def state(self):
        return [t.clone() for t in (self.params, self.adam_m, self.adam_v, self.counter)]

    def set_state(self, st):
        for dst, src in zip((self.params, self.adam_m, self.adam_v, self.counter), st):
            dst.copy_(src)


def synthesize_stack(pb: "pact.Problem", case: dict, device) -> torch.Tensor:
    """Delay stack [M, H, W] made by the forward model (Eq. 5) from the
    ground-truth SOS and IP: every channel j is the stitch of the patches
    H_ij(v_true) X_i, plus the seeded noise stack.  All arithmetic in libpact."""
    d = case["d"]
    sos = torch.as_tensor(case["sos_true"], device=device)
    w_true = pact.sos_to_delays(pb, sos)
    X = pact.patch_fft(pb, torch.as_tensor(case["ip"], device=device)[None])[:, 0].contiguous()
    Yc = pact.forward_model(pb, w_true, d, X)
    noise = torch.as_tensor(case["noise"], device=device)
    stack = torch.empty_like(noise)
    ws = pact._ws(pact.stitch_workspace_size(pb), device)
    for j in range(len(d)):
        pact.stitch(pb, Yc[:, j].contiguous(), stack[j], ws=ws)
    stack += noise
    return stack


def measurement_spectra(pb: "pact.Problem", case: dict, device) -> torch.Tensor:
    """Patch spectra of the synthetic measurement, Y = H(v_true) X + N (Eq. 5 per
    patch, N the windowed spectra of the seeded noise stack)."""
    sos = torch.as_tensor(case["sos_true"], device=device)
    w_true = pact.sos_to_delays(pb, sos)
    X = pact.patch_fft(pb, torch.as_tensor(case["ip"], device=device)[None])[:, 0].contiguous()
    Y = pact.patch_fft(pb, torch.as_tensor(case["noise"], device=device))
    return pact.forward_model(pb, w_true, case["d"], X, Y, accumulate=True)


def channel_data_stack(pb: "pact.Problem", case: dict, device, spread: float = 0.0, ring_dr: float = 0.0,
                       ws=None, bandpass=None) -> torch.Tensor:
    """Delay stack [M, H, W] made end to end from synthetic ring channel data:
    pact_rf_synth (straight-ray times of flight through the ground-truth SOS,
    differentiated pulses from the ground-truth IP; optional spreading and
    ring-radius mismatch), optionally a transducer band-limit
    (bandpass = (fc, frac_bw), pact_rf_bandpass), then DAS (Eq. 1) at the M
    delays."""
    cfg = pb.cfg
    rf = pact.rf_synth(pb, torch.as_tensor(case["ip"], device=device), torch.as_tensor(case["sos_true"], device=device),
                       cfg.rf_fs, cfg.rf_t0, cfg.rf_ns, cfg.rf_sigma, spread, ring_dr, ws=ws)
    if bandpass is not None:
        rf = pact.rf_bandpass(rf, cfg.rf_fs, bandpass[0], bandpass[1])
    return pact.das_stack(pb, rf, cfg.rf_fs, cfg.rf_t0, case["d"])


@dataclasses.dataclass
class Recovered:
    """Result of recover(): the SOS [G, G] and the stitched initial-pressure
    image [H, W] (host tensors when asked for), the loss of every iteration,
    the deconvolved patches X_hat (device) and the restarts that the loss
    checks triggered, as (iteration, reason, new learning rate)."""
    sos: torch.Tensor
    hist: list
    xhat: torch.Tensor
    image: torch.Tensor
    restarts: list


def recover(pb: "pact.Problem", stack_host: torch.Tensor, d, eps: float, lam: float, lr: float,
            sos_init: torch.Tensor, mask: torch.Tensor, iters: int, graph: bool = True, to_host: bool = True,
            snapshot_every: int = 50, explode: float = 1e3, lr_decay: float = 0.1, max_restarts: int = 8):
    """Public end-to-end API: upload a delay stack (host, ideally pinned), form
    the patch spectra, run `iters` recovery iterations reading the loss back
    after each, and return the recovered SOS, the stitched image (Sec. S1.5)
    and the loss history (a Recovered).  With `to_host` the SOS and the image
    are copied to pinned host memory before the call returns.

    Each iteration's loss is copied to pinned host memory behind it on the
    stream and read while the next iteration runs, so the read-back does not
    stall the GPU.  Every loss is checked: a non-finite loss, or one above
    `explode` times the first, restores the last state whose loss was good
    (a device snapshot taken every `snapshot_every` iterations; the initial
    state and the last four are kept, and a restart that fails again within
    one interval goes one snapshot further back), multiplies the learning
    rate by `lr_decay` and continues from there; after `max_restarts`
    restarts the call raises PactError (PACT_ERR_NONFINITE)."""
    dev = pb.device
    stack = stack_host.to(dev, non_blocking=True)
    Y = pact.patch_fft(pb, stack)
    rec = PGRecovery(pb, Y, d, eps, lam, lr, sos_init, mask)
    if graph:
        rec.capture()
    hist, restarts = [], []
    host = torch.empty(2, dtype=torch.float32, pin_memory=True)      # one slot per iteration in flight
    done = [torch.cuda.Event(), torch.cuda.Event()]
    stream = torch.cuda.current_stream(dev)
    goods = [(0, rec.state())]                    # (iteration, state) whose loss was checked, oldest first
    pending = None                                # snapshot whose loss is not read yet
    L0 = None
    it = 0

    def bad(L):
        return not np.isfinite(L) or (L0 is not None and L > explode * abs(L0))

    def restart(at, reason):
        nonlocal it, pending
        if len(restarts) >= max_restarts:
            raise pact.PactError(f"recover: {reason} at iteration {at}; {max_restarts} restarts did not help",
                                 pact.PACT_ERR_NONFINITE)
        torch.cuda.synchronize(dev)
        # a state whose loss was finite can still be non-physical (a negative
        # speed gives a NaN gradient): if the last restart from it failed
        # within one snapshot interval, go one snapshot further back
        if restarts and len(goods) > 1 and at - goods[-1][0] <= snapshot_every:
            goods.pop()
        rec.lr *= lr_decay
        rec.set_state(goods[-1][1])
        if graph:
            rec.capture()
        restarts.append((at, reason, rec.lr))
        del hist[goods[-1][0]:]
        it, pending = goods[-1][0], None

    while it < iters:
        if it % snapshot_every == 0:
            pending = (it, rec.state())
        rec.iterate()
        slot = it & 1
        host[slot:slot + 1].copy_(rec.out["loss"], non_blocking=True)
        done[slot].record(stream)
        if it > len(hist):                        # the previous iteration's loss, copied meanwhile
            done[slot ^ 1].synchronize()
            L = float(host[slot ^ 1])
            L0 = L if L0 is None and np.isfinite(L) else L0
            if bad(L):
                restart(it - 1, "non-finite loss" if not np.isfinite(L) else "exploding loss")
                continue
            hist.append(L)
            if pending is not None and pending[0] == it - 1:
                goods.append(pending)
                del goods[1:-4]                   # the initial state and the last four
                pending = None
        it += 1
        if it == iters:                           # the last iteration's loss
            done[(iters - 1) & 1].synchronize()
            L = float(host[(iters - 1) & 1])
            L0 = L if L0 is None and np.isfinite(L) else L0
            if bad(L):
                restart(iters - 1, "non-finite loss" if not np.isfinite(L) else "exploding loss")
                continue
            hist.append(L)
    w = pact.sos_to_delays(pb, rec.sos)
    Xh = pact.mc_deconv_loss(pb, w, Y, d, eps, want_grad=False, want_xhat=True)["Xhat"]
    image = pact.stitch(pb, Xh)
    sos = rec.sos
    if to_host:
        sos_h = torch.empty(sos.shape, dtype=sos.dtype, pin_memory=True)
        img_h = torch.empty(image.shape, dtype=image.dtype, pin_memory=True)
        sos_h.copy_(sos, non_blocking=True)
        img_h.copy_(image, non_blocking=True)
        torch.cuda.synchronize(dev)
        sos, image = sos_h, img_h
    return Recovered(sos, hist, Xh, image, restarts)
