"""Python binding of libpact (include/pact.h): argument marshalling only.

Every function here checks tensor devices, dtypes and shapes, allocates the
outputs it is not given (PyTorch owns device memory) and calls the C entry
point of the same name on the current PyTorch CUDA stream.  All arithmetic
of the method runs in the CUDA kernels of libpact; there is no CPU path.
If the library is not built, or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

from . import build as _build

_LIB = None


# status codes of include/pact.h
PACT_OK, PACT_ERR_INVALID_ARG, PACT_ERR_SHAPE, PACT_ERR_CUDA, PACT_ERR_TIMEOUT, PACT_ERR_NONFINITE, \
    PACT_ERR_UNSUPPORTED = range(7)


class PactError(RuntimeError):
    """A libpact call failed; `status` is its pact_status code (or None)."""

    def __init__(self, msg, status=None):
        super().__init__(msg)
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_int), ("ring_radius", ctypes.c_float), ("ring_phase", ctypes.c_float),
                ("v0", ctypes.c_float), ("v_bg", ctypes.c_float), ("img_h", ctypes.c_int),
                ("img_w", ctypes.c_int), ("dx", ctypes.c_float), ("sos_g", ctypes.c_int),
                ("sos_dx", ctypes.c_float), ("mask_radius", ctypes.c_float), ("ray_step", ctypes.c_float)]


class _PatchesC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("p", ctypes.c_int), ("centres", ctypes.c_void_p),
                ("window_fwhm", ctypes.c_float)]


class RfParams(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_float), ("t0", ctypes.c_float), ("n_s", ctypes.c_int),
                ("sigma", ctypes.c_float), ("spread", ctypes.c_float), ("ring_dr", ctypes.c_float)]


_VP, _I, _F, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
_GP = ctypes.POINTER(Geometry)
_PP = ctypes.POINTER(_PatchesC)

_SIGS = {
    "pact_version": ([], ctypes.c_char_p),
    "pact_last_error_message": ([], ctypes.c_char_p),
    "pact_das_stack": ([_GP, _VP, _I, _F, _F, _VP, _I, _VP, _VP], _I),
    "pact_rf_synth_workspace_size": ([_GP, _I], _SZ),
    "pact_rf_synth": ([_GP, _VP, _VP, ctypes.POINTER(RfParams), _VP, _VP, _SZ, _VP], _I),
    "pact_rf_bandpass": ([_VP, _VP, _I, _I, _F, _F, _F, _VP], _I),
    "pact_patch_fft": ([_GP, _PP, _VP, _I, _VP, _VP], _I),
    "pact_sos_to_delays": ([_GP, _PP, _VP, _VP, _VP], _I),
    "pact_sos_to_delays_clear": ([_GP, _PP, _VP, _VP, _VP, _SZ, _VP], _I),
    "pact_sos_to_delays_tv_workspace_size": ([_GP, _PP], _SZ),
    "pact_sos_to_delays_tv": ([_GP, _PP, _VP, _VP, _VP, _SZ, _F, _VP, _SZ, _VP], _I),
    "pact_sos_to_delays_adj_adam": ([_GP, _PP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _F, _F, _F, _F, _VP,
                                     _VP, _SZ, _VP], _I),
    "pact_sos_to_delays_adj_workspace_size": ([_GP, _PP], _SZ),
    "pact_sos_to_delays_adj": ([_GP, _PP, _VP, _VP, _VP, _I, _VP, _SZ, _VP], _I),
    "pact_psf_synth": ([_GP, _PP, _VP, _VP, _I, _VP, _VP], _I),
    "pact_psf_synth_adj": ([_GP, _PP, _VP, _VP, _I, _VP, _VP, _I, _VP], _I),
    "pact_forward_model": ([_GP, _PP, _VP, _VP, _I, _VP, _VP, _I, _VP], _I),
    "pact_mc_deconv_loss_workspace_size": ([_GP, _PP, _I], _SZ),
    "pact_mc_deconv_loss": ([_GP, _PP, _VP, _VP, _VP, _I, _F, _VP, _VP, _VP, _VP, _VP, _SZ, _VP], _I),
    "pact_mc_deconv_loss_noalloc": ([_GP, _PP, _VP, _VP, _VP, _I, _F, _VP, _VP, _VP, _VP, _VP], _I),
    "pact_mc_deconv_tables_size": ([_GP, _PP, _I], _SZ),
    "pact_mc_deconv_loss_tabled_workspace_size": ([_GP, _PP, _I], _SZ),
    "pact_mc_deconv_tables": ([_GP, _PP, _VP, _I, _VP, _SZ, _VP], _I),
    "pact_mc_deconv_loss_tabled": ([_GP, _PP, _VP, _VP, _VP, _I, _F, _VP, _SZ, _VP, _VP, _VP, _VP, _I, _VP, _SZ,
                                    _VP], _I),
    "pact_mc_deconv_loss_adj": ([_GP, _PP, _VP, _VP, _VP, _I, _F, _VP, _VP, _I, _VP, _SZ, _VP], _I),
    "pact_mc_deconv_status": ([_GP, _PP, _I, _VP, _VP, _VP], _I),
    "pact_mc_deconv_inject_stall": ([_GP, _PP, _I, _VP, _VP, _VP], _I),
    "pact_set_wait_limit_ns": ([ctypes.c_ulonglong], _I),
    "pact_get_wait_limit_ns": ([], ctypes.c_ulonglong),
    "pact_tv": ([_GP, _VP, _F, _VP, _VP, _I, _VP], _I),
    "pact_adam_step": ([_I, _VP, _VP, _VP, _VP, _I, _VP, _F, _F, _F, _F, _VP, _VP], _I),
    "pact_stitch_workspace_size": ([_GP, _PP], _SZ),
    "pact_stitch": ([_GP, _PP, _VP, _VP, _VP, _SZ, _VP], _I),
    "pact_stitch_channels_workspace_size": ([_GP, _PP, _I], _SZ),
    "pact_stitch_channels": ([_GP, _PP, _I, _VP, _VP, _VP, _SZ, _VP], _I),
    "pact_nf_param_count": ([], _I),
    "pact_nf_workspace_size": ([_GP], _SZ),
    "pact_nf_forward": ([_GP, _VP, _VP, _F, _F, _VP, _VP, _SZ, _VP], _I),
    "pact_nf_backward": ([_GP, _VP, _VP, _F, _F, _VP, _VP, _I, _VP, _SZ, _VP], _I),
    "pact_nf_status": ([_GP, _VP, _SZ, ctypes.POINTER(ctypes.c_int), _VP], _I),
    "pact_siren_param_count": ([], _I),
    "pact_siren_workspace_size": ([_GP], _SZ),
    "pact_siren_forward": ([_GP, _VP, _VP, _F, _VP, _VP, _SZ, _VP], _I),
    "pact_siren_backward": ([_GP, _VP, _VP, _F, _VP, _VP, _I, _VP, _SZ, _VP], _I),
    "pact_cnn_param_count": ([_I], _I),
    "pact_cnn_input_channels": ([_I], _I),
    "pact_cnn_pool_workspace_size": ([_GP, _I], _SZ),
    "pact_cnn_pool_stack": ([_GP, _VP, _I, _VP, _VP, _SZ, _VP], _I),
    "pact_cnn_workspace_size": ([_GP, _I, _I], _SZ),
    "pact_cnn_forward": ([_GP, _I, _I, _VP, _VP, _VP, _F, _F, _VP, _VP, _SZ, _VP], _I),
    "pact_cnn_backward": ([_GP, _I, _I, _VP, _VP, _VP, _F, _VP, _VP, _I, _VP, _SZ, _VP], _I),
    "pact_cnn_mse": ([_GP, _I, _VP, _VP, _VP, _I, _F, _VP, _VP, _VP, _VP], _I),
    "pact_cnn_status": ([_GP, _I, _I, _VP, _SZ, ctypes.POINTER(ctypes.c_int), _VP], _I),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libpact.so (building it first if allowed); raises if impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise PactError(f"libpact is not built ({path}); run paper_2409_10876_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        msg = load().pact_last_error_message().decode()
        raise PactError(f"{what} failed (status {status}): {msg}", status)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise PactError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise PactError(f"{name} must be {dtype} (got {t.dtype})")
    if not t.is_contiguous():
        raise PactError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise PactError(f"{name} must have shape {tuple(shape)} (got {tuple(t.shape)})")
    return t


def _host_f32(d):
    a = np.ascontiguousarray(np.asarray(d, dtype=np.float32).ravel())
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ problem description

class Problem:
    """Geometry + patch set of one workload, with the patch centres on the device."""

    def __init__(self, cfg, device="cuda", centres=None):
        self.cfg = cfg
        gd = cfg.geometry_dict()
        self.geom = Geometry(gd["n_t"], gd["ring_radius"], gd["ring_phase"], gd["v0"], gd["v_bg"],
                             gd["img_h"], gd["img_w"], gd["dx"], gd["sos_g"], gd["sos_dx"],
                             gd["mask_radius"], gd["ray_step"])
        cen = cfg.centres() if centres is None else np.asarray(centres, np.int32)
        self.centres = torch.as_tensor(np.ascontiguousarray(cen, dtype=np.int32), device=device)
        self.patches = _PatchesC(int(cen.shape[0]), int(cfg.p), self.centres.data_ptr(), gd["window_fwhm"])
        self.n = int(cen.shape[0])
        self.p = int(cfg.p)
        self.f = self.p * (self.p // 2 + 1)
        self.n_t = int(cfg.n_t)
        self.g = int(cfg.sos_g)
        self.device = torch.device(device)

    def gp(self):
        return ctypes.byref(self.geom)

    def pp(self):
        return ctypes.byref(self.patches)

    def spectra_shape(self, m):
        return (self.n, m, self.p, self.p // 2 + 1)


def _empty(shape, dtype, dev):
    return torch.empty(shape, dtype=dtype, device=dev)


def _ws(nbytes: int, dev) -> torch.Tensor:
    # 256-byte alignment: PyTorch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


# ------------------------------------------------------------------ entry points

def das_stack(pb: Problem, rf, fs: float, t0: float, d, stack=None):
    """Eq. 1: DAS stack [M, H, W] from channel data rf [N_t, n_s]."""
    L = load()
    rf = _dev(rf, "rf", torch.float32)
    dh, dp = _host_f32(d)
    m = dh.size
    if stack is None:
        stack = _empty((m, pb.cfg.img_h, pb.cfg.img_w), torch.float32, rf.device)
    _dev(stack, "stack", torch.float32, (m, pb.cfg.img_h, pb.cfg.img_w))
    _check(L.pact_das_stack(pb.gp(), _ptr(rf), rf.shape[1], fs, t0, dp, m, _ptr(stack), _stream()), "das_stack")
    return stack


def rf_synth_workspace_size(pb: Problem, pixels_per_pass: int) -> int:
    return int(load().pact_rf_synth_workspace_size(pb.gp(), int(pixels_per_pass)))


def rf_synth(pb: Problem, p0, sos, fs: float, t0: float, n_s: int, sigma: float, spread: float = 0.0,
             ring_dr: float = 0.0, rf=None, ws=None, pixels_per_pass: int = 65536):
    """Synthetic ring channel data rf [N_t, n_s] of the initial pressure p0 [H, W]
    with straight-ray times of flight through the SOS grid [G, G] (the input of
    Eq. 1).  The workspace (made if None) sets the pixels per pass."""
    L = load()
    cfg = pb.cfg
    p0 = _dev(p0, "p0", torch.float32, (cfg.img_h, cfg.img_w))
    sos = _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    if rf is None:
        rf = _empty((pb.n_t, int(n_s)), torch.float32, p0.device)
    _dev(rf, "rf", torch.float32, (pb.n_t, int(n_s)))
    if ws is None:
        ws = _ws(rf_synth_workspace_size(pb, min(int(pixels_per_pass), cfg.img_h * cfg.img_w)), p0.device)
    rp = RfParams(float(fs), float(t0), int(n_s), float(sigma), float(spread), float(ring_dr))
    _check(L.pact_rf_synth(pb.gp(), _ptr(p0), _ptr(sos), ctypes.byref(rp), _ptr(rf), _ptr(ws), ws.numel(),
                           _stream()), "rf_synth")
    return rf



def rf_bandpass(rf, fs: float, fc: float, frac_bw: float, out=None):
    """Channel data [N_t, n_s] filtered along time by the transducer band-limit
    (zero-phase Gaussian-windowed cosine at fc, half-amplitude width frac_bw fc)."""
    L = load()
    rf = _dev(rf, "rf", torch.float32)
    if rf.dim() != 2:
        raise ValueError("rf must be [N_t, n_s]")
    if out is None:
        out = torch.empty_like(rf)
    _dev(out, "out", torch.float32, tuple(rf.shape))
    _check(L.pact_rf_bandpass(_ptr(rf), _ptr(out), rf.shape[0], rf.shape[1], float(fs), float(fc), float(frac_bw),
                              _stream()), "rf_bandpass")
    return out

def patch_fft(pb: Problem, stack, Y=None):
    """Sec. S1.5: windowed patch spectra Y [N, M, P, P/2+1] (complex64)."""
    L = load()
    stack = _dev(stack, "stack", torch.float32)
    m = stack.shape[0]
    if Y is None:
        Y = _empty(pb.spectra_shape(m), torch.complex64, stack.device)
    _dev(Y, "Y", torch.complex64, pb.spectra_shape(m))
    _check(L.pact_patch_fft(pb.gp(), pb.pp(), _ptr(stack), m, _ptr(Y), _stream()), "patch_fft")
    return Y


def sos_to_delays(pb: Problem, sos, w=None, clear=None):
    """Eq. 3: wavefront errors w [N, N_t] from the SOS grid [G, G].  `clear`
    (a float32 CUDA tensor, e.g. the dL/dw buffer a following accumulating
    fused pass adds to) is set to zero in the same launch."""
    L = load()
    sos = _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    if w is None:
        w = _empty((pb.n, pb.n_t), torch.float32, sos.device)
    _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    if clear is None:
        _check(L.pact_sos_to_delays(pb.gp(), pb.pp(), _ptr(sos), _ptr(w), _stream()), "sos_to_delays")
    else:
        clear = _dev(clear, "clear", torch.float32)
        _check(L.pact_sos_to_delays_clear(pb.gp(), pb.pp(), _ptr(sos), _ptr(w), _ptr(clear), clear.numel(),
                                          _stream()), "sos_to_delays_clear")
    return w


def sos_to_delays_tv_workspace_size(pb: Problem) -> int:
    return int(load().pact_sos_to_delays_tv_workspace_size(pb.gp(), pb.pp()))


def sos_to_delays_tv(pb: Problem, sos, w, clear, lam: float, tv_ws):
    """Eq. 3 with `clear` zeroed, plus lam times the TV terms of Eq. 7 at `sos`
    into `tv_ws` (uint8 CUDA tensor of sos_to_delays_tv_workspace_size bytes)
    for the sos_to_delays_adj_adam call of the same iteration."""
    L = load()
    sos = _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    clear = _dev(clear, "clear", torch.float32)
    _check(L.pact_sos_to_delays_tv(pb.gp(), pb.pp(), _ptr(sos), _ptr(w), _ptr(clear), clear.numel(), float(lam),
                                   _ptr(tv_ws), tv_ws.numel(), _stream()), "sos_to_delays_tv")
    return w


def sos_to_delays_adj_adam(pb: Problem, sos, dL_dw, m, v, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, mask=None,
                           step_counter=None, step: int = 1, tv_ws=None, loss=None, grad=None, ws=None):
    """Adjoint of Eq. 3, the TV subgradient from `tv_ws` (if given) and one
    in-place Adam step on `sos` in two launches; `grad` (if given) receives
    the gradient, `loss` (if given, with tv_ws) gets lam TV added."""
    L = load()
    sos = _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    dL_dw = _dev(dL_dw, "dL_dw", torch.float32, (pb.n, pb.n_t))
    for t, nm in ((m, "m"), (v, "v")):
        _dev(t, nm, torch.float32, (pb.g, pb.g))
    if grad is not None:
        _dev(grad, "grad", torch.float32, (pb.g, pb.g))
    if mask is not None:
        _dev(mask, "mask", torch.uint8, (pb.g, pb.g))
    if step_counter is not None:
        _dev(step_counter, "step_counter", torch.int32, (2,))
    if ws is None:
        ws = _ws(sos_to_delays_adj_workspace_size(pb), sos.device)
    _check(L.pact_sos_to_delays_adj_adam(pb.gp(), pb.pp(), _ptr(sos), _ptr(dL_dw), _ptr(tv_ws), _ptr(loss),
                                         _ptr(grad), _ptr(m), _ptr(v), int(step), _ptr(step_counter), float(lr),
                                         float(beta1), float(beta2), float(eps), _ptr(mask), _ptr(ws), ws.numel(),
                                         _stream()), "sos_to_delays_adj_adam")
    return sos


def sos_to_delays_adj_workspace_size(pb: Problem) -> int:
    return int(load().pact_sos_to_delays_adj_workspace_size(pb.gp(), pb.pp()))


def sos_to_delays_adj(pb: Problem, sos, dL_dw, dL_dsos=None, accumulate=False, ws=None):
    """Adjoint of Eq. 3: dL/dsos [G, G] from dL/dw [N, N_t]."""
    L = load()
    sos = _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    dL_dw = _dev(dL_dw, "dL_dw", torch.float32, (pb.n, pb.n_t))
    if dL_dsos is None:
        dL_dsos = torch.zeros((pb.g, pb.g), dtype=torch.float32, device=sos.device)
    _dev(dL_dsos, "dL_dsos", torch.float32, (pb.g, pb.g))
    if ws is None:
        ws = _ws(sos_to_delays_adj_workspace_size(pb), sos.device)
    _check(L.pact_sos_to_delays_adj(pb.gp(), pb.pp(), _ptr(sos), _ptr(dL_dw), _ptr(dL_dsos), int(accumulate),
                                    _ptr(ws), ws.numel(), _stream()), "sos_to_delays_adj")
    return dL_dsos


def psf_synth(pb: Problem, w, d, H=None):
    """Eq. 4: transfer functions H [N, M, P, P/2+1] (complex64)."""
    L = load()
    w = _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    dh, dp = _host_f32(d)
    if H is None:
        H = _empty(pb.spectra_shape(dh.size), torch.complex64, w.device)
    _dev(H, "H", torch.complex64, pb.spectra_shape(dh.size))
    _check(L.pact_psf_synth(pb.gp(), pb.pp(), _ptr(w), dp, dh.size, _ptr(H), _stream()), "psf_synth")
    return H


def psf_synth_adj(pb: Problem, w, d, dL_dH, dL_dw=None, accumulate=False):
    """Adjoint of Eq. 4; dL_dH holds (dL/dRe, dL/dIm) pairs (PyTorch convention)."""
    L = load()
    w = _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    dh, dp = _host_f32(d)
    dL_dH = _dev(dL_dH, "dL_dH", torch.complex64, pb.spectra_shape(dh.size))
    if dL_dw is None:
        dL_dw = torch.zeros((pb.n, pb.n_t), dtype=torch.float32, device=w.device)
    _dev(dL_dw, "dL_dw", torch.float32, (pb.n, pb.n_t))
    _check(L.pact_psf_synth_adj(pb.gp(), pb.pp(), _ptr(w), dp, dh.size, _ptr(dL_dH), _ptr(dL_dw), int(accumulate),
                                _stream()), "psf_synth_adj")
    return dL_dw


def forward_model(pb: Problem, w, d, X, Y=None, accumulate=False):
    """Eq. 5: Y_ij (+)= H_ij X_i."""
    L = load()
    w = _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    dh, dp = _host_f32(d)
    X = _dev(X, "X", torch.complex64, (pb.n, pb.p, pb.p // 2 + 1))
    if Y is None:
        Y = _empty(pb.spectra_shape(dh.size), torch.complex64, w.device)
        accumulate = False
    _dev(Y, "Y", torch.complex64, pb.spectra_shape(dh.size))
    _check(L.pact_forward_model(pb.gp(), pb.pp(), _ptr(w), dp, dh.size, _ptr(X), _ptr(Y), int(accumulate),
                                _stream()), "forward_model")
    return Y


def mc_deconv_loss_workspace_size(pb: Problem, m: int) -> int:
    return int(load().pact_mc_deconv_loss_workspace_size(pb.gp(), pb.pp(), int(m)))


def mc_deconv_loss(pb: Problem, w, Y, d, eps: float, want_grad=True, want_xhat=False, want_loss_pp=False,
                   out=None, ws=None, tables: "McdTables" = None, accumulate=False):
    """Eq. 6-7 fused (+ adjoint when want_grad).  Returns a dict with
    'loss' [1], and 'dL_dw' [N, N_t], 'Xhat' [N, P, P/2+1], 'loss_pp' [N] as asked.
    `out` may hold preallocated tensors under the same keys; `tables` (built
    for the same problem and delays) skips the per-call table build."""
    L = load()
    w = _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    Y = _dev(Y, "Y", torch.complex64)
    m = Y.shape[1]
    _dev(Y, "Y", torch.complex64, pb.spectra_shape(m))
    dh, dp = _host_f32(d)
    if dh.size != m:
        raise PactError(f"delay list has {dh.size} entries but Y has {m} channels")
    out = {} if out is None else out
    dev = w.device
    if "loss" not in out:
        out["loss"] = torch.zeros(1, dtype=torch.float32, device=dev)
    if want_grad and "dL_dw" not in out:
        out["dL_dw"] = _empty((pb.n, pb.n_t), torch.float32, dev)
    if want_xhat and "Xhat" not in out:
        out["Xhat"] = _empty((pb.n, pb.p, pb.p // 2 + 1), torch.complex64, dev)
    if want_loss_pp and "loss_pp" not in out:
        out["loss_pp"] = _empty((pb.n,), torch.float32, dev)
    if tables is not None:
        if ws is None:
            ws = _ws(tables.scratch_bytes, dev)
        _check(L.pact_mc_deconv_loss_tabled(pb.gp(), pb.pp(), _ptr(w), _ptr(Y), dp, m, float(eps), _ptr(tables.buf),
                                            tables.buf.numel(), _ptr(out["loss"]),
                                            _ptr(out.get("loss_pp") if want_loss_pp else None),
                                            _ptr(out.get("Xhat") if want_xhat else None),
                                            _ptr(out.get("dL_dw") if want_grad else None), int(accumulate),
                                            _ptr(ws), ws.numel(), _stream()), "mc_deconv_loss_tabled")
        return out
    if accumulate:
        raise PactError("accumulate needs prebuilt tables (pact_mc_deconv_loss_tabled)")
    if ws is None:
        ws = _ws(mc_deconv_loss_workspace_size(pb, m), dev)
    _check(L.pact_mc_deconv_loss(pb.gp(), pb.pp(), _ptr(w), _ptr(Y), dp, m, float(eps), _ptr(out["loss"]),
                                 _ptr(out.get("loss_pp") if want_loss_pp else None),
                                 _ptr(out.get("Xhat") if want_xhat else None),
                                 _ptr(out.get("dL_dw") if want_grad else None), _ptr(ws), ws.numel(), _stream()),
           "mc_deconv_loss")
    return out


class McdTables:
    """Prebuilt tables of the fused pass for fixed (geometry, patches, delays):
    build once, pass to mc_deconv_loss(..., tables=...) every iteration."""

    def __init__(self, pb: Problem, d, device=None):
        L = load()
        self.d, dp = _host_f32(d)
        self.m = int(self.d.size)
        dev = pb.device if device is None else device
        self.buf = _ws(int(L.pact_mc_deconv_tables_size(pb.gp(), pb.pp(), self.m)), dev)
        self.scratch_bytes = int(L.pact_mc_deconv_loss_tabled_workspace_size(pb.gp(), pb.pp(), self.m))
        _check(L.pact_mc_deconv_tables(pb.gp(), pb.pp(), dp, self.m, _ptr(self.buf), self.buf.numel(), _stream()),
               "mc_deconv_tables")


def mc_deconv_status(pb: Problem, m: int, tables: Optional["McdTables"] = None, ws=None) -> None:
    """Raises PactError (status PACT_ERR_TIMEOUT) if a bounded wait of a fused
    pass using these tables (or this workspace) gave up since the last check;
    clears the flag.  Synchronises the stream."""
    L = load()
    _check(L.pact_mc_deconv_status(pb.gp(), pb.pp(), int(m), _ptr(tables.buf if tables is not None else None),
                                   _ptr(ws), _stream()), "mc_deconv_status")


def mc_deconv_inject_stall(pb: Problem, tables: "McdTables") -> None:
    """Test hook: the next streaming fused pass with these tables withholds a
    pipeline-stage release, runs into the wait limit and reports a timeout."""
    L = load()
    _check(L.pact_mc_deconv_inject_stall(pb.gp(), pb.pp(), tables.m, _ptr(tables.buf), None, _stream()),
           "mc_deconv_inject_stall")


def set_wait_limit_ns(ns: int) -> None:
    """Bound on every device-side wait of later launches (0 = default 200 ms)."""
    _check(load().pact_set_wait_limit_ns(int(ns)), "set_wait_limit_ns")


def wait_limit_ns() -> int:
    return int(load().pact_get_wait_limit_ns())


def mc_deconv_loss_noalloc(pb: Problem, w, Y, d, eps: float, want_grad=True, want_xhat=False, want_loss_pp=False,
                           out=None):
    """mc_deconv_loss for callers that cannot allocate device memory: the
    library uses its built-in scratch array (PACT_NOALLOC_SCRATCH_BYTES) instead
    of a workspace.  Outputs must be preallocated in `out` if the caller cannot
    let this binding allocate them; missing ones are allocated here."""
    L = load()
    w = _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    Y = _dev(Y, "Y", torch.complex64)
    m = Y.shape[1]
    _dev(Y, "Y", torch.complex64, pb.spectra_shape(m))
    dh, dp = _host_f32(d)
    if dh.size != m:
        raise PactError(f"delay list has {dh.size} entries but Y has {m} channels")
    out = {} if out is None else out
    dev = w.device
    if "loss" not in out:
        out["loss"] = torch.zeros(1, dtype=torch.float32, device=dev)
    if want_grad and "dL_dw" not in out:
        out["dL_dw"] = _empty((pb.n, pb.n_t), torch.float32, dev)
    if want_xhat and "Xhat" not in out:
        out["Xhat"] = _empty((pb.n, pb.p, pb.p // 2 + 1), torch.complex64, dev)
    if want_loss_pp and "loss_pp" not in out:
        out["loss_pp"] = _empty((pb.n,), torch.float32, dev)
    _check(L.pact_mc_deconv_loss_noalloc(pb.gp(), pb.pp(), _ptr(w), _ptr(Y), dp, m, float(eps), _ptr(out["loss"]),
                                         _ptr(out.get("loss_pp") if want_loss_pp else None),
                                         _ptr(out.get("Xhat") if want_xhat else None),
                                         _ptr(out.get("dL_dw") if want_grad else None), _stream()),
           "mc_deconv_loss_noalloc")
    return out


def mc_deconv_loss_adj(pb: Problem, w, Y, d, eps: float, dL_dloss=None, dL_dw=None, accumulate=False, ws=None):
    """dL_dw (+)= dL_dloss * d(loss)/dw (standalone adjoint of mc_deconv_loss)."""
    L = load()
    w = _dev(w, "w", torch.float32, (pb.n, pb.n_t))
    Y = _dev(Y, "Y", torch.complex64)
    m = Y.shape[1]
    dh, dp = _host_f32(d)
    if dL_dw is None:
        dL_dw = torch.zeros((pb.n, pb.n_t), dtype=torch.float32, device=w.device)
    if dL_dloss is not None:
        dL_dloss = _dev(dL_dloss.reshape(1).contiguous(), "dL_dloss", torch.float32)
    if ws is None:
        ws = _ws(mc_deconv_loss_workspace_size(pb, m), w.device)
    _check(L.pact_mc_deconv_loss_adj(pb.gp(), pb.pp(), _ptr(w), _ptr(Y), dp, m, float(eps), _ptr(dL_dloss),
                                     _ptr(dL_dw), int(accumulate), _ptr(ws), ws.numel(), _stream()),
           "mc_deconv_loss_adj")
    return dL_dw


def tv(pb: Problem, sos, lam: float, value=None, grad=None, accumulate=False):
    """Eq. 7 TV term: value (+)= lam TV(sos), grad (+)= lam dTV/dsos."""
    L = load()
    sos = _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    _check(L.pact_tv(pb.gp(), _ptr(sos), float(lam), _ptr(value), _ptr(grad), int(accumulate), _stream()), "tv")
    return value, grad


def adam_step(param, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, mask=None,
              step_counter=None):
    """One in-place Adam update of `param` (Sec. 3.3).  With `step_counter`
    (int32 CUDA tensor [2], zeros initially; [0] counts the steps) the step
    count is read from and advanced on the device, so the call can be
    replayed from a CUDA graph."""
    L = load()
    for t, nm in ((param, "param"), (grad, "grad"), (m, "m"), (v, "v")):
        _dev(t, nm, torch.float32, tuple(param.shape))
    if mask is not None:
        _dev(mask, "mask", torch.uint8, tuple(param.shape))
    if step_counter is not None:
        _dev(step_counter, "step_counter", torch.int32, (2,))
    _check(L.pact_adam_step(param.numel(), _ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(step),
                            _ptr(step_counter), float(lr),
                            float(beta1), float(beta2), float(eps), _ptr(mask), _stream()), "adam_step")
    return param


def stitch_workspace_size(pb: Problem) -> int:
    return int(load().pact_stitch_workspace_size(pb.gp(), pb.pp()))


def stitch(pb: Problem, Xhat, image=None, ws=None):
    """Sec. S1.5: stitched image [H, W] from deconvolved patches."""
    L = load()
    Xhat = _dev(Xhat, "Xhat", torch.complex64, (pb.n, pb.p, pb.p // 2 + 1))
    if image is None:
        image = _empty((pb.cfg.img_h, pb.cfg.img_w), torch.float32, Xhat.device)
    if ws is None:
        ws = _ws(stitch_workspace_size(pb), Xhat.device)
    _check(L.pact_stitch(pb.gp(), pb.pp(), _ptr(Xhat), _ptr(image), _ptr(ws), ws.numel(), _stream()), "stitch")
    return image


def stitch_channels(pb: Problem, Y, stack=None, ws=None):
    """Sec. S1.5 for every channel: delay stack [M, H, W] from patch spectra
    [N, M, P, P/2+1]."""
    L = load()
    Y = _dev(Y, "Y", torch.complex64)
    m = int(Y.shape[1])
    _dev(Y, "Y", torch.complex64, pb.spectra_shape(m))
    if stack is None:
        stack = _empty((m, pb.cfg.img_h, pb.cfg.img_w), torch.float32, Y.device)
    _dev(stack, "stack", torch.float32, (m, pb.cfg.img_h, pb.cfg.img_w))
    if ws is None:
        ws = _ws(L.pact_stitch_channels_workspace_size(pb.gp(), pb.pp(), m), Y.device)
    _check(L.pact_stitch_channels(pb.gp(), pb.pp(), m, _ptr(Y), _ptr(stack), _ptr(ws), ws.numel(), _stream()),
           "stitch_channels")
    return stack


# ------------------------------------------------------------------ neural-field SOS (BF16 tensor cores)

def nf_param_count() -> int:
    return int(load().pact_nf_param_count())


def nf_workspace_size(pb: Problem) -> int:
    return int(load().pact_nf_workspace_size(pb.gp()))


class NeuralField:
    """Device state of the neural-field SOS: FP32 parameters and the workspace
    that carries activations from forward to backward."""

    def __init__(self, pb: Problem, params, mask=None, v_mid: float = 1525.0, v_half: float = 125.0):
        self.pb = pb
        self.params = torch.as_tensor(np.asarray(params, np.float32), device=pb.device).contiguous()
        if self.params.numel() != nf_param_count():
            raise PactError(f"neural field has {nf_param_count()} parameters, got {self.params.numel()}")
        self.mask = None if mask is None else torch.as_tensor(np.asarray(mask, np.uint8), device=pb.device).contiguous()
        self.v_mid, self.v_half = float(v_mid), float(v_half)
        self.ws = _ws(nf_workspace_size(pb), pb.device)


def nf_forward(nf: NeuralField, sos=None):
    """SOS [G, G] from the neural field (activations kept for nf_backward)."""
    L = load()
    pb = nf.pb
    if sos is None:
        sos = _empty((pb.g, pb.g), torch.float32, pb.device)
    _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    _check(L.pact_nf_forward(pb.gp(), _ptr(nf.params), _ptr(nf.mask), nf.v_mid, nf.v_half, _ptr(sos), _ptr(nf.ws),
                             nf.ws.numel(), _stream()), "nf_forward")
    return sos


def nf_backward(nf: NeuralField, dL_dsos, dL_dparams=None, accumulate=False):
    """dL/dparams from dL/dsos for the parameters of the last nf_forward."""
    L = load()
    pb = nf.pb
    dL_dsos = _dev(dL_dsos, "dL_dsos", torch.float32, (pb.g, pb.g))
    if dL_dparams is None:
        dL_dparams = torch.zeros_like(nf.params)
    _dev(dL_dparams, "dL_dparams", torch.float32, tuple(nf.params.shape))
    _check(L.pact_nf_backward(pb.gp(), _ptr(nf.params), _ptr(nf.mask), nf.v_mid, nf.v_half, _ptr(dL_dsos),
                              _ptr(dL_dparams), int(accumulate), _ptr(nf.ws), nf.ws.numel(), _stream()), "nf_backward")
    return dL_dparams


def nf_status(nf: NeuralField) -> None:
    """Raises if a tensor-core wait of the neural-field kernels gave up (synchronises)."""
    L = load()
    st = ctypes.c_int(0)
    _check(L.pact_nf_status(nf.pb.gp(), _ptr(nf.ws), nf.ws.numel(), ctypes.byref(st), _stream()), "nf_status")


# ------------------------------------------------------------------ the paper's SIREN field

class SirenField:
    """Device state of the paper's neural field (SIREN, 1027 parameters)."""

    def __init__(self, pb: Problem, params, mask=None, omega0: float = 30.0):
        L = load()
        self.pb = pb
        self.params = torch.as_tensor(np.asarray(params, np.float32), device=pb.device).contiguous()
        if self.params.numel() != int(L.pact_siren_param_count()):
            raise PactError(f"the field has {int(L.pact_siren_param_count())} parameters, got {self.params.numel()}")
        self.mask = None if mask is None else torch.as_tensor(np.asarray(mask, np.uint8), device=pb.device).contiguous()
        self.omega0 = float(omega0)
        self.ws = _ws(L.pact_siren_workspace_size(pb.gp()), pb.device)


def siren_forward(sf: SirenField, sos=None):
    """SOS [G, G] from the SIREN field (its output kept for siren_backward)."""
    L = load()
    pb = sf.pb
    if sos is None:
        sos = _empty((pb.g, pb.g), torch.float32, pb.device)
    _dev(sos, "sos", torch.float32, (pb.g, pb.g))
    _check(L.pact_siren_forward(pb.gp(), _ptr(sf.params), _ptr(sf.mask), sf.omega0, _ptr(sos), _ptr(sf.ws),
                                sf.ws.numel(), _stream()), "siren_forward")
    return sos


def siren_backward(sf: SirenField, dL_dsos, dL_dparams=None, accumulate=False):
    """dL/dparams from dL/dsos for the parameters of the last siren_forward."""
    L = load()
    pb = sf.pb
    dL_dsos = _dev(dL_dsos, "dL_dsos", torch.float32, (pb.g, pb.g))
    if dL_dparams is None:
        dL_dparams = torch.zeros_like(sf.params)
    _dev(dL_dparams, "dL_dparams", torch.float32, tuple(sf.params.shape))
    _check(L.pact_siren_backward(pb.gp(), _ptr(sf.params), _ptr(sf.mask), sf.omega0, _ptr(dL_dsos), _ptr(dL_dparams),
                                 int(accumulate), _ptr(sf.ws), sf.ws.numel(), _stream()), "siren_backward")
    return dL_dparams


# ------------------------------------------------------------------ warm-start CNN

def cnn_param_count(m: int) -> int:
    return int(load().pact_cnn_param_count(int(m)))


def cnn_input_channels(m: int) -> int:
    return int(load().pact_cnn_input_channels(int(m)))


def cnn_pool_stack(pb: Problem, stack, x=None, ws=None):
    """Pooled, RMS-normalised BF16 network input [G, G, Cp] of one delay stack
    [M, 4G, 4G]; `x` may be a slice of a larger BF16 dataset tensor."""
    L = load()
    stack = _dev(stack, "stack", torch.float32)
    m = int(stack.shape[0])
    _dev(stack, "stack", torch.float32, (m, pb.cfg.img_h, pb.cfg.img_w))
    cp = cnn_input_channels(m)
    if x is None:
        x = _empty((pb.g, pb.g, cp), torch.bfloat16, pb.device)
    _dev(x, "x", torch.bfloat16, (pb.g, pb.g, cp))
    if ws is None:
        ws = _ws(L.pact_cnn_pool_workspace_size(pb.gp(), m), pb.device)
    _check(L.pact_cnn_pool_stack(pb.gp(), _ptr(stack), m, _ptr(x), _ptr(ws), ws.numel(), _stream()), "cnn_pool_stack")
    return x


class WarmStartCNN:
    """Device state of the warm-start network for a fixed batch size: FP32
    parameters and the workspace that carries activations from forward to
    backward."""

    def __init__(self, pb: Problem, m: int, batch: int, params, mask=None, v_mid: float = 1525.0,
                 v_half: float = 125.0):
        L = load()
        self.pb, self.m, self.batch = pb, int(m), int(batch)
        self.params = torch.as_tensor(np.asarray(params, np.float32), device=pb.device).contiguous()
        if self.params.numel() != cnn_param_count(m):
            raise PactError(f"the network has {cnn_param_count(m)} parameters, got {self.params.numel()}")
        self.mask = None if mask is None else torch.as_tensor(np.asarray(mask, np.uint8), device=pb.device).contiguous()
        self.mask_count = pb.g * pb.g if mask is None else int(np.count_nonzero(np.asarray(mask)))
        self.v_mid, self.v_half = float(v_mid), float(v_half)
        self.cp = cnn_input_channels(m)
        self.ws = _ws(L.pact_cnn_workspace_size(pb.gp(), self.m, self.batch), pb.device)
        self.scratch = torch.empty(max(self.batch, 64), dtype=torch.float32, device=pb.device)

    def _x(self, x):
        return _dev(x, "x", torch.bfloat16, (self.batch, self.pb.g, self.pb.g, self.cp))


def cnn_forward(net: WarmStartCNN, x, sos=None):
    """SOS maps [batch, G, G] predicted from pooled inputs x [batch, G, G, Cp]."""
    L = load()
    pb = net.pb
    x = net._x(x)
    if sos is None:
        sos = _empty((net.batch, pb.g, pb.g), torch.float32, pb.device)
    _dev(sos, "sos", torch.float32, (net.batch, pb.g, pb.g))
    _check(L.pact_cnn_forward(pb.gp(), net.m, net.batch, _ptr(net.params), _ptr(x), _ptr(net.mask), net.v_mid,
                              net.v_half, _ptr(sos), _ptr(net.ws), net.ws.numel(), _stream()), "cnn_forward")
    return sos


def cnn_backward(net: WarmStartCNN, x, dL_dsos, dL_dparams=None, accumulate=False):
    """dL/dparams for the inputs of the last cnn_forward."""
    L = load()
    pb = net.pb
    x = net._x(x)
    dL_dsos = _dev(dL_dsos, "dL_dsos", torch.float32, (net.batch, pb.g, pb.g))
    if dL_dparams is None:
        dL_dparams = torch.zeros_like(net.params)
    _dev(dL_dparams, "dL_dparams", torch.float32, tuple(net.params.shape))
    _check(L.pact_cnn_backward(pb.gp(), net.m, net.batch, _ptr(net.params), _ptr(x), _ptr(net.mask), net.v_half,
                               _ptr(dL_dsos), _ptr(dL_dparams), int(accumulate), _ptr(net.ws), net.ws.numel(),
                               _stream()), "cnn_backward")
    return dL_dparams


def cnn_mse(net: WarmStartCNN, sos, sos_true, scale: float = 100.0, loss=None, dL_dsos=None, want_grad=True):
    """Training loss mean ((sos - sos_true) / scale)^2 over samples and mask
    nodes (device [1]) and, when asked, its gradient [batch, G, G]."""
    L = load()
    pb = net.pb
    sos = _dev(sos, "sos", torch.float32, (net.batch, pb.g, pb.g))
    sos_true = _dev(sos_true, "sos_true", torch.float32, (net.batch, pb.g, pb.g))
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=pb.device)
    if want_grad and dL_dsos is None:
        dL_dsos = _empty((net.batch, pb.g, pb.g), torch.float32, pb.device)
    _check(L.pact_cnn_mse(pb.gp(), net.batch, _ptr(sos), _ptr(sos_true), _ptr(net.mask), net.mask_count, float(scale),
                          _ptr(loss), _ptr(dL_dsos if want_grad else None), _ptr(net.scratch), _stream()), "cnn_mse")
    return loss, dL_dsos


def cnn_status(net: WarmStartCNN) -> None:
    """Raises if a tensor-core wait of the network kernels gave up (synchronises)."""
    L = load()
    st = ctypes.c_int(0)
    _check(L.pact_cnn_status(net.pb.gp(), net.m, net.batch, _ptr(net.ws), net.ws.numel(), ctypes.byref(st), _stream()),
           "cnn_status")
