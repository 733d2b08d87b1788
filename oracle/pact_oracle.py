"""FP64 CPU oracle of the per-iteration forward model and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never calls it and
shares no code with it; the only common module is the seeded input generator
``paper_2409_10876_gb300.inputs``, which holds no arithmetic of the method.

Everything here is a literal FP64 evaluation of the paper's definitions:

* Eq. 1   delay-and-sum (DAS) image for an extra delay d      -> das_stack
* Sec. S1.5 Gaussian-windowed patches, orthonormal 2-D DFT     -> patch_spectra
* Eq. 2-3 straight-ray wavefront error w = int (1 - v0/v) dl   -> wavefront_errors
* Eq. 4   wavefront transfer function H_i(k; d, v)             -> transfer_functions
* Eq. 5   multi-channel forward model Y_i = H_i X_i            -> forward_spectra
* Eq. 6   pseudo-inverse multi-channel deconvolution           -> deconvolve
* Eq. 7   |k|-weighted aberrated-image-matching loss + TV      -> data_loss, tv, objective
* Sec. 3.3 Adam on the SOS parameters                          -> adam_step
* Sec. S1.5 stitching: place patches, divide by summed windows  -> stitch
* Sec. 3.3 neural fields: the Fourier-feature MLP               -> nf_sos
  and the paper's SIREN (256 sine features, no hidden layer)    -> siren_sos

The DFT is an explicit matrix product (no FFT routine).  The gradients of
the objective come from PyTorch autograd through these FP64 definitions,
the same differentiation route the paper takes (Sec. 3.3), and are pinned
independently by central finite differences in the tests.

Readings where the paper is silent or ambiguous (each is listed in the
design notes of the repository):

* ``T`` in Eq. 6 is the conjugate transpose; a regulariser eps is added to
  the channel sum: X = sum_j conj(H_j) Y_j / (sum_j |H_j|^2 + eps).
* Eq. 4 is used in the sign that follows from Eq. 1 under the forward DFT
  kernel exp(-j k.rho): H = 1/2 (exp(+j|k|(d - w(ang k))) + exp(-j|k|(d - w(ang k + pi)))),
  i.e. the complex conjugate of the printed form.
* k is angular (rad/m); |k| in the loss weight is in rad/mm; the loss is
  summed over the rfft half-spectrum with weight 2 on columns other than
  k_x = 0 and Nyquist.
* w at direction phi is the linear interpolation, in ring angle, of the
  per-transducer values at the point where the ray from the patch centre in
  direction phi meets the ring.
* Ray integral: midpoint rule with step h inside the SOS mask disk (last
  partial step weighted by its true length); outside the mask the integrand
  is (1 - v0/v_bg).  v is bilinear in the node values, clamped at the edge.
"""
from __future__ import annotations

import math
from types import SimpleNamespace
from typing import Optional, Sequence

import numpy as np
import torch

DT = torch.float64
CT = torch.complex128


def geom(cfg) -> SimpleNamespace:
    """Geometry numbers as a namespace (accepts an inputs.Config or a dict)."""
    d = cfg.geometry_dict() if hasattr(cfg, "geometry_dict") else dict(cfg)
    return SimpleNamespace(**d)


def _t(x, dtype=DT):
    if isinstance(x, torch.Tensor):
        return x.to(dtype)
    return torch.as_tensor(np.asarray(x), dtype=dtype)


# --------------------------------------------------------------------------
# geometry (Eq. 1 notation: r_n transducer positions, r' image positions)
# --------------------------------------------------------------------------

def transducers(g) -> torch.Tensor:
    """r_n = R (cos a_n, sin a_n), a_n = 2 pi n / N_t + phase.  [N_t, 2]"""
    a = 2.0 * math.pi * torch.arange(g.n_t, dtype=DT) / g.n_t + g.ring_phase
    return torch.stack([g.ring_radius * torch.cos(a), g.ring_radius * torch.sin(a)], dim=1)


def pixel_xy(g, rows, cols):
    """Pixel (row a, col b) sits at x = (b - (W-1)/2) dx, y = (a - (H-1)/2) dx."""
    rows = _t(rows)
    cols = _t(cols)
    return (cols - (g.img_w - 1) / 2.0) * g.dx, (rows - (g.img_h - 1) / 2.0) * g.dx


def centre_xy(g, centres) -> torch.Tensor:
    """Patch-centre positions r'_i [N, 2] from (row, col) pixel indices."""
    c = _t(centres)
    x, y = pixel_xy(g, c[:, 0], c[:, 1])
    return torch.stack([x, y], dim=1)


# --------------------------------------------------------------------------
# Eq. 1: delay-and-sum
# --------------------------------------------------------------------------

def das_stack(g, rf, fs: float, t0: float, d) -> torch.Tensor:
    """y(r'; d_j) = sum_n S((|r' - r_n| - d_j)/v0, n) for every pixel and delay.

    S is sampled at rate fs starting at time t0 and linearly interpolated,
    zero outside the recorded samples.  Returns [M, H, W].
    """
    rf = _t(rf)
    d = _t(d)
    n_t, n_s = rf.shape
    rn = transducers(g)
    rows = torch.arange(g.img_h, dtype=DT)
    cols = torch.arange(g.img_w, dtype=DT)
    x, y = pixel_xy(g, rows[:, None], cols[None, :])
    out = torch.zeros(d.shape[0], g.img_h, g.img_w, dtype=DT)
    pad = torch.cat([torch.zeros(n_t, 1, dtype=DT), rf, torch.zeros(n_t, 1, dtype=DT)], dim=1)
    for n in range(n_t):
        dist = torch.sqrt((x - rn[n, 0]) ** 2 + (y - rn[n, 1]) ** 2)
        for j in range(d.shape[0]):
            q = ((dist - d[j]) / g.v0 - t0) * fs
            q0 = torch.floor(q)
            f = q - q0
            i0 = q0.long() + 1                       # +1: offset into the zero-padded row
            ok0 = (i0 >= 0) & (i0 <= n_s + 1)
            ok1 = (i0 + 1 >= 0) & (i0 + 1 <= n_s + 1)
            s0 = torch.where(ok0, pad[n, i0.clamp(0, n_s + 1)], torch.zeros((), dtype=DT))
            s1 = torch.where(ok1, pad[n, (i0 + 1).clamp(0, n_s + 1)], torch.zeros((), dtype=DT))
            out[j] += (1.0 - f) * s0 + f * s1
    return out


# --------------------------------------------------------------------------
# Sec. S1.5: Gaussian-windowed patches and their spectra
# --------------------------------------------------------------------------

def window(g) -> torch.Tensor:
    """Gaussian window exp(-|rho|^2 / (2 sigma^2)), FWHM = 2 sqrt(2 ln 2) sigma,
    rho measured from the patch centre (local index P/2).  [P, P]"""
    sig = g.window_fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    o = (torch.arange(g.p, dtype=DT) - g.p // 2) * g.dx
    return torch.exp(-(o[:, None] ** 2 + o[None, :] ** 2) / (2.0 * sig * sig))


def crop(g, stack, centres) -> torch.Tensor:
    """P x P crops of a [M, H, W] stack, rows c_a - P/2 .. c_a + P/2 - 1 (zero
    outside the image).  Returns [N, M, P, P]."""
    stack = _t(stack)
    c = np.asarray(centres)
    P = g.p
    out = torch.zeros(len(c), stack.shape[0], P, P, dtype=DT)
    for i, (ca, cb) in enumerate(c):
        r0, c0 = int(ca) - P // 2, int(cb) - P // 2
        ra, rb = max(r0, 0), min(r0 + P, g.img_h)
        ca_, cb_ = max(c0, 0), min(c0 + P, g.img_w)
        if ra < rb and ca_ < cb_:
            out[i, :, ra - r0:rb - r0, ca_ - c0:cb_ - c0] = stack[:, ra:rb, ca_:cb_]
    return out


def dft_matrix(P: int, sign: int = -1) -> torch.Tensor:
    """F[u, a] = exp(sign * 2 pi j u a / P)."""
    u = torch.arange(P, dtype=DT)
    return torch.exp(sign * 2j * math.pi * torch.outer(u, u).to(CT) / P)


def rfft2_ortho(x) -> torch.Tensor:
    """Y[u, v] = (1/P) sum_{a,b} x[a, b] exp(-2 pi j (u a + v b) / P), v = 0..P/2."""
    x = _t(x).to(CT)
    P = x.shape[-1]
    Fm = dft_matrix(P)
    return Fm @ x @ Fm[: P // 2 + 1].transpose(0, 1) / P


def irfft2_ortho(X) -> torch.Tensor:
    """Inverse of rfft2_ortho for Hermitian-symmetric spectra: the full spectrum
    is implied by X[-u, -v] = conj(X[u, v]); the imaginary parts of the k_x = 0
    and Nyquist columns are dropped, as a real signal requires."""
    X = X.to(CT)
    P = X.shape[-2]
    Z = dft_matrix(P, +1) @ X                       # inverse along rows (complex)
    b = torch.arange(P, dtype=DT)
    v = torch.arange(P // 2 + 1, dtype=DT)
    E = torch.exp(2j * math.pi * torch.outer(v, b).to(CT) / P)   # [P/2+1, P]
    wgt = torch.full((P // 2 + 1,), 2.0, dtype=DT)
    wgt[0] = 1.0
    wgt[P // 2] = 1.0
    return (torch.real(Z[..., :, :, None] * E[None, :, :]) * wgt[:, None]).sum(-2) / P


def patch_spectra(g, stack, centres) -> torch.Tensor:
    """Y_ij(k) of every windowed patch i and channel j: [N, M, P, P/2+1]."""
    return rfft2_ortho(crop(g, stack, centres) * window(g))


def kgrid(g):
    """Angular frequencies of the half-spectrum bins.

    Returns kx, ky [P, P/2+1] (rad/m, fftfreq order along rows), |k|, the
    angle atan2(ky, kx) (0 at k = 0) and the half-spectrum weight c_k."""
    P = g.p
    u = torch.arange(P, dtype=DT)
    fy = torch.where(u < P / 2, u, u - P) / (P * g.dx)
    fx = torch.arange(P // 2 + 1, dtype=DT) / (P * g.dx)
    ky = (2.0 * math.pi * fy)[:, None].expand(P, P // 2 + 1)
    kx = (2.0 * math.pi * fx)[None, :].expand(P, P // 2 + 1)
    kmag = torch.sqrt(kx * kx + ky * ky)
    phi = torch.atan2(ky, kx)
    phi = torch.where(kmag == 0, torch.zeros_like(phi), phi)
    ck = torch.full((P // 2 + 1,), 2.0, dtype=DT)
    ck[0] = 1.0
    ck[P // 2] = 1.0
    return kx, ky, kmag, phi, ck[None, :].expand(P, P // 2 + 1)


# --------------------------------------------------------------------------
# Eq. 2-3: straight-ray wavefront errors
# --------------------------------------------------------------------------

def sos_bilinear(g, sos, x, y) -> torch.Tensor:
    """Bilinear interpolation of the node values; node (p, q) sits at
    x = (q - (G-1)/2) sos_dx, y = (p - (G-1)/2) sos_dx; clamped at the edge."""
    G = g.sos_g
    fx = (x / g.sos_dx + (G - 1) / 2.0).clamp(0.0, G - 1.0)
    fy = (y / g.sos_dx + (G - 1) / 2.0).clamp(0.0, G - 1.0)
    ix = torch.floor(fx).clamp(0, G - 2)
    iy = torch.floor(fy).clamp(0, G - 2)
    tx = fx - ix
    ty = fy - iy
    ix = ix.long()
    iy = iy.long()
    v00 = sos[iy, ix]
    v01 = sos[iy, ix + 1]
    v10 = sos[iy + 1, ix]
    v11 = sos[iy + 1, ix + 1]
    return (1 - ty) * ((1 - tx) * v00 + tx * v01) + ty * ((1 - tx) * v10 + tx * v11)


def ray_quadrature(g, start, end):
    """Midpoint-rule samples of the segments start -> end clipped to the mask.

    Returns sample positions px, py [R, S], weights [R, S] (metres) and the
    length of each segment outside the mask [R]."""
    L = torch.linalg.norm(end - start, dim=1)
    e = (end - start) / L[:, None]
    ce = (start * e).sum(1)
    disc = ce * ce - ((start * start).sum(1) - g.mask_radius ** 2)
    hit = disc > 0
    sq = torch.sqrt(disc.clamp(min=0.0))
    s_in = (-ce - sq).clamp(min=torch.zeros_like(L), max=L)
    s_out = (-ce + sq).clamp(min=torch.zeros_like(L), max=L)
    chord = torch.where(hit, (s_out - s_in).clamp(min=0.0), torch.zeros_like(L))
    h = g.ray_step
    nfull = torch.floor(chord / h)
    rem = chord - nfull * h
    S = int(nfull.max().item()) + 1 if len(L) else 1
    m = torch.arange(S, dtype=DT)[None, :]
    full = m < nfull[:, None]
    last = m == nfull[:, None]
    s = torch.where(full, s_in[:, None] + (m + 0.5) * h, s_in[:, None] + nfull[:, None] * h + 0.5 * rem[:, None])
    wgt = torch.where(full, torch.full_like(s, h), torch.where(last, rem[:, None].expand_as(s), torch.zeros_like(s)))
    px = start[:, 0:1] + s * e[:, 0:1]
    py = start[:, 1:2] + s * e[:, 1:2]
    return px, py, wgt, L - chord


def wavefront_errors(g, sos, centres, chunk: int = 8) -> torch.Tensor:
    """Eq. 3: w_{i,n} = int_{r'_i}^{r_n} (1 - v0 / v(l)) dl, [N, N_t] metres.

    ``sos`` may require grad; the result is differentiable in it."""
    sos = sos if isinstance(sos, torch.Tensor) else _t(sos)
    c = centre_xy(g, centres)
    rn = transducers(g)
    out = []
    for i0 in range(0, c.shape[0], chunk):
        cc = c[i0:i0 + chunk]
        start = cc[:, None, :].expand(-1, g.n_t, -1).reshape(-1, 2)
        end = rn[None, :, :].expand(cc.shape[0], -1, -1).reshape(-1, 2)
        px, py, wgt, outside = ray_quadrature(g, start, end)
        v = sos_bilinear(g, sos, px, py)
        wi = (wgt * (1.0 - g.v0 / v)).sum(1) + outside * (1.0 - g.v0 / g.v_bg)
        out.append(wi.reshape(cc.shape[0], g.n_t))
    return torch.cat(out, 0)


# --------------------------------------------------------------------------
# Eq. 4: wavefront transfer functions
# --------------------------------------------------------------------------

def wavefront_at(g, w, cxy, phi) -> torch.Tensor:
    """w_i evaluated at ray direction phi from patch centre r'_i: the ray meets
    the ring at ring angle alpha; linear interpolation of the transducer
    values in alpha (cyclic).  w [N, N_t], cxy [N, 2], phi [...] -> [N, ...]"""
    ex = torch.cos(phi)[None]
    ey = torch.sin(phi)[None]
    cx = cxy[:, 0].reshape(-1, *([1] * phi.dim()))
    cy = cxy[:, 1].reshape(-1, *([1] * phi.dim()))
    ce = cx * ex + cy * ey
    s = -ce + torch.sqrt(ce * ce - (cx * cx + cy * cy) + g.ring_radius ** 2)
    alpha = torch.atan2(cy + s * ey, cx + s * ex) - g.ring_phase
    t = torch.remainder(alpha / (2.0 * math.pi / g.n_t), float(g.n_t))
    n1 = torch.floor(t)
    f = t - n1
    n1 = n1.long() % g.n_t
    n2 = (n1 + 1) % g.n_t
    flat = w.reshape(w.shape[0], -1)
    idx1 = n1.reshape(w.shape[0], -1)
    idx2 = n2.reshape(w.shape[0], -1)
    w1 = torch.gather(flat, 1, idx1).reshape(n1.shape)
    w2 = torch.gather(flat, 1, idx2).reshape(n1.shape)
    return (1.0 - f) * w1 + f * w2


def transfer_functions(g, w, centres, d) -> torch.Tensor:
    """Eq. 4 (sign derived from Eq. 1 for the forward DFT):
    H_ij(k) = 1/2 (exp(+j|k|(d_j - w_i(ang k))) + exp(-j|k|(d_j - w_i(ang k + pi)))).
    Returns [N, M, P, P/2+1]."""
    _, _, kmag, phi, _ = kgrid(g)
    cxy = centre_xy(g, centres)
    w = w if isinstance(w, torch.Tensor) else _t(w)
    d = _t(d)
    W1 = wavefront_at(g, w, cxy, phi)[:, None]            # [N, 1, P, P/2+1]
    W2 = wavefront_at(g, w, cxy, phi + math.pi)[:, None]
    k = kmag[None, None]
    dj = d[None, :, None, None]
    return 0.5 * (torch.exp(1j * (k * (dj - W1)).to(CT)) + torch.exp(-1j * (k * (dj - W2)).to(CT)))


def forward_spectra(H, X) -> torch.Tensor:
    """Eq. 5: Y_ij = H_ij X_i.  H [N, M, ...], X [N, ...] -> [N, M, ...]"""
    return H * X[:, None]


# --------------------------------------------------------------------------
# Eq. 6-7: deconvolution, loss
# --------------------------------------------------------------------------

def deconvolve(H, Y, eps: float) -> torch.Tensor:
    """Eq. 6: X_i = sum_j conj(H_ij) Y_ij / (sum_j |H_ij|^2 + eps) (0 where the
    denominator vanishes).  [N, P, P/2+1]"""
    A = (torch.conj(H) * Y).sum(1)
    B = (H.real ** 2 + H.imag ** 2).sum(1) + eps
    safe = torch.where(B == 0, torch.ones_like(B), B)
    return torch.where(B == 0, torch.zeros_like(A), A / safe)


def data_loss(g, H, Y, Xh, per_patch: bool = False):
    """Eq. 7 data term: sum_i sum_k c_k |k|_mm sum_j |Y_ij - H_ij X_i|^2."""
    _, _, kmag, _, ck = kgrid(g)
    wgt = ck * kmag * 1e-3
    R = Y - H * Xh[:, None]
    e = (R.real ** 2 + R.imag ** 2).sum(1)               # [N, P, P/2+1]
    lp = (e * wgt[None]).sum((1, 2))
    return lp if per_patch else lp.sum()


def tv(sos) -> torch.Tensor:
    """Anisotropic TV over the SOS nodes (m/s):
    sum |v[p+1,q] - v[p,q]| + |v[p,q+1] - v[p,q]|."""
    return (sos[1:, :] - sos[:-1, :]).abs().sum() + (sos[:, 1:] - sos[:, :-1]).abs().sum()


def mc_deconv_loss(g, w, Y, centres, d, eps: float, want_grad: bool = True):
    """Eq. 6-7 for given wavefronts: returns loss, per-patch loss, X_hat and
    (optionally) dL/dw from autograd."""
    w = _t(w).clone().requires_grad_(want_grad)
    Y = Y.to(CT) if isinstance(Y, torch.Tensor) else torch.as_tensor(Y).to(CT)
    H = transfer_functions(g, w, centres, d)
    Xh = deconvolve(H, Y, eps)
    lp = data_loss(g, H, Y, Xh, per_patch=True)
    L = lp.sum()
    grad = None
    if want_grad:
        (grad,) = torch.autograd.grad(L, w)
    return L.detach(), lp.detach(), Xh.detach(), grad


def sos_to_delays_adj(g, sos, centres, dLdw) -> torch.Tensor:
    """Vector-Jacobian product of Eq. 3: dL/dv_node = sum_{i,n} dL/dw_{i,n} dw_{i,n}/dv_node."""
    s = _t(sos).clone().requires_grad_(True)
    w = wavefront_errors(g, s, centres)
    (gs,) = torch.autograd.grad(w, s, grad_outputs=_t(dLdw))
    return gs


def objective(g, sos, Y, centres, d, eps: float, lam: float, want_grad: bool = True):
    """Eq. 7 as a function of the pixel-grid SOS: data term + lam * TV.

    Returns (L, L_data, w, dL/dsos) with the gradient from autograd."""
    s = _t(sos).clone().requires_grad_(want_grad)
    w = wavefront_errors(g, s, centres)
    Yc = Y.to(CT) if isinstance(Y, torch.Tensor) else torch.as_tensor(Y).to(CT)
    H = transfer_functions(g, w, centres, d)
    Xh = deconvolve(H, Yc, eps)
    Ld = data_loss(g, H, Yc, Xh)
    L = Ld + lam * tv(s)
    gs = None
    if want_grad:
        (gs,) = torch.autograd.grad(L, s)
    return L.detach(), Ld.detach(), w.detach(), gs


# --------------------------------------------------------------------------
# Sec. 3.3: Adam (Kingma & Ba) on the trainable nodes
# --------------------------------------------------------------------------

def adam_step(param, grad, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8, mask=None):
    """One textbook Adam update (bias-corrected); nodes with mask == 0 are left
    unchanged (their moments too).  Returns new (param, m, v)."""
    param, grad, m, v = (_t(a) for a in (param, grad, m, v))
    m2 = b1 * m + (1 - b1) * grad
    v2 = b2 * v + (1 - b2) * grad * grad
    mh = m2 / (1 - b1 ** step)
    vh = v2 / (1 - b2 ** step)
    p2 = param - lr * mh / (torch.sqrt(vh) + eps)
    if mask is not None:
        keep = _t(mask) == 0
        p2 = torch.where(keep, param, p2)
        m2 = torch.where(keep, m, m2)
        v2 = torch.where(keep, v, v2)
    return p2, m2, v2


# --------------------------------------------------------------------------
# Sec. S1.5: stitching
# --------------------------------------------------------------------------

def stitch(g, Xh, centres) -> torch.Tensor:
    """Translate every deconvolved patch irfft2(X_i) to its centre, sum, and
    divide by the summed Gaussian windows (0 where no window reaches).
    The window was applied once, when the patches were cropped."""
    xs = irfft2_ortho(Xh)
    win = window(g)
    num = torch.zeros(g.img_h, g.img_w, dtype=DT)
    den = torch.zeros(g.img_h, g.img_w, dtype=DT)
    P = g.p
    for i, (ca, cb) in enumerate(np.asarray(centres)):
        r0, c0 = int(ca) - P // 2, int(cb) - P // 2
        ra, rb = max(r0, 0), min(r0 + P, g.img_h)
        ca_, cb_ = max(c0, 0), min(c0 + P, g.img_w)
        if ra < rb and ca_ < cb_:
            num[ra:rb, ca_:cb_] += xs[i, ra - r0:rb - r0, ca_ - c0:cb_ - c0]
            den[ra:rb, ca_:cb_] += win[ra - r0:rb - r0, ca_ - c0:cb_ - c0]
    return torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), torch.zeros_like(num))


# --------------------------------------------------------------------------
# Synthetic measurement (Eq. 5 plus noise) for a recovery problem
# --------------------------------------------------------------------------

def make_measurement(g, case: dict):
    """Y = H(v_true) X + N: X from the windowed ground-truth IP patches, N from
    the windowed noise stack, both through the same patch spectra."""
    cen = case["centres"]
    w_true = wavefront_errors(g, _t(case["sos_true"]), cen)
    H = transfer_functions(g, w_true, cen, case["d"])
    X = patch_spectra(g, _t(case["ip"])[None], cen)[:, 0]
    N = patch_spectra(g, _t(case["noise"]), cen)
    return forward_spectra(H, X) + N, X, w_true


def recover(g, case: dict, Y, steps: int, lr: float, eps: float, lam: float):
    """Plain recovery loop (Sec. 3.3): Adam on the masked pixel-grid SOS.
    Returns the final SOS and the loss history."""
    sos = _t(case["sos_init"])
    mask = _t(case["mask"])
    m = torch.zeros_like(sos)
    v = torch.zeros_like(sos)
    hist = []
    for it in range(1, steps + 1):
        L, _, _, gs = objective(g, sos, Y, case["centres"], case["d"], eps, lam)
        hist.append(float(L))
        sos, m, v = adam_step(sos, gs, m, v, it, lr, mask=mask)
    return sos, hist


# --------------------------------------------------------------------------
# Neural-field SOS (Sec. 3.3 coordinate-based representation; the Fourier-
# feature MLP of the BF16 workload): features -> 4 x 128 ReLU -> tanh-bounded
# output, evaluated at the SOS nodes; nodes outside the mask stay at v_bg.
# --------------------------------------------------------------------------

def nf_unflatten(params, shapes):
    out, o = {}, 0
    for name, shape in shapes:
        n = int(np.prod(shape))
        out[name] = params[o:o + n].reshape(shape)
        o += n
    return out


def nf_features(g, freqs) -> torch.Tensor:
    """[G*G, 4F]: for every node (row-major) and frequency f_l the features
    sin(2 pi f_l x), cos(2 pi f_l x), sin(2 pi f_l y), cos(2 pi f_l y) with x, y the
    node position divided by the field of view (G sos_dx)."""
    G = g.sos_g
    c = (torch.arange(G, dtype=DT) - (G - 1) / 2.0) / G      # position / field of view
    yy, xx = torch.meshgrid(c, c, indexing="ij")
    x, y = xx.reshape(-1, 1), yy.reshape(-1, 1)
    f = _t(freqs)[None, :]
    feats = torch.stack([torch.sin(2 * math.pi * f * x), torch.cos(2 * math.pi * f * x),
                         torch.sin(2 * math.pi * f * y), torch.cos(2 * math.pi * f * y)], dim=2)
    return feats.reshape(G * G, -1)


def nf_sos(g, params, shapes, freqs, mask, v_mid: float, v_half: float) -> torch.Tensor:
    """SOS [G, G] from the neural field; params may require grad."""
    p = nf_unflatten(params, shapes)
    h = nf_features(g, freqs)
    n_hidden = sum(1 for name, _ in shapes if name.startswith("W"))
    for l in range(1, n_hidden + 1):
        h = torch.relu(h @ p[f"W{l}"].T + p[f"b{l}"])
    z = h @ p["w5"] + p["b5"]
    v = v_mid + v_half * torch.tanh(z)
    keep = _t(mask).reshape(-1) > 0
    v = torch.where(keep, v, torch.full_like(v, g.v_bg))
    return v.reshape(g.sos_g, g.sos_g)


def nf_objective(g, params, shapes, freqs, mask, v_mid, v_half, Y, centres, d, eps: float,
                 want_grad: bool = True):
    """Eq. 7 (lambda = 0, as for the neural field in Sec. 3.3) as a function of
    the neural-field parameters; gradient by autograd."""
    prm = _t(params).clone().requires_grad_(want_grad)
    sos = nf_sos(g, prm, shapes, freqs, mask, v_mid, v_half)
    w = wavefront_errors(g, sos, centres)
    Yc = Y.to(CT) if isinstance(Y, torch.Tensor) else torch.as_tensor(Y).to(CT)
    H = transfer_functions(g, w, centres, d)
    Xh = deconvolve(H, Yc, eps)
    L = data_loss(g, H, Yc, Xh)
    gp = None
    if want_grad:
        (gp,) = torch.autograd.grad(L, prm)
    return L.detach(), sos.detach(), gp


# ----------------------------------------------------------------------------
# the paper's neural field (Sec. 3.3): SIREN without hidden layers, 256 sine
# features, a linear output and two extra scalars (output scale and offset)
# ----------------------------------------------------------------------------

def siren_coords(g) -> torch.Tensor:
    """[G*G, 2] node coordinates (x = column, y = row) scaled to [-1, 1]."""
    G = g.sos_g
    c = (torch.arange(G, dtype=DT) - (G - 1) / 2.0) / ((G - 1) / 2.0)
    yy, xx = torch.meshgrid(c, c, indexing="ij")
    return torch.stack([xx.reshape(-1), yy.reshape(-1)], 1)


def siren_sos(g, params, shapes, mask, omega0: float) -> torch.Tensor:
    """SOS [G, G]: v = offset + scale (sum_f w2_f sin(omega0 (W1_f . x + b1_f)) + b2)
    on the mask, v_bg elsewhere; params may require grad."""
    p = nf_unflatten(params if isinstance(params, torch.Tensor) else _t(params), shapes)
    x = siren_coords(g)
    h = torch.sin(omega0 * (x @ p["W1"].T + p["b1"]))
    z = h @ p["w2"] + p["b2"]
    v = p["offset"] + p["scale"] * z
    keep = _t(mask).reshape(-1) > 0
    v = torch.where(keep, v, torch.full_like(v, g.v_bg))
    return v.reshape(g.sos_g, g.sos_g)


def siren_objective(g, params, shapes, mask, omega0, Y, centres, d, eps: float, want_grad: bool = True):
    """Eq. 7 (lambda = 0) as a function of the SIREN parameters; gradient by autograd."""
    prm = _t(params).clone().requires_grad_(want_grad)
    sos = siren_sos(g, prm, shapes, mask, omega0)
    w = wavefront_errors(g, sos, centres)
    Yc = Y.to(CT) if isinstance(Y, torch.Tensor) else torch.as_tensor(Y).to(CT)
    H = transfer_functions(g, w, centres, d)
    Xh = deconvolve(H, Yc, eps)
    L = data_loss(g, H, Yc, Xh)
    gp = None
    if want_grad:
        (gp,) = torch.autograd.grad(L, prm)
    return L.detach(), sos.detach(), gp
