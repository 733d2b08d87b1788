"""Seeded synthetic inputs and workload configurations.

This module is shared by the CUDA path, the benchmark and the FP64 oracle.
It holds only *inputs*: geometry numbers, delay lists, patch-centre lists and
seeded random phantoms (speed-of-sound maps, initial-pressure images, noise).
It contains none of the method's arithmetic (no delay-and-sum, no ray
integration, no transfer functions, no deconvolution, no loss).

The paper's phantoms (k-Wave simulations of a mouse-like body, a leaf phantom,
in-vivo data) are not available; these generators stand in for them with the
value ranges the paper states (Sec. S1.1: SOS 1490-1650 m/s, water background,
512-element ring, 3.2 mm patches with 75 % overlap, Sec. 3.3: M = 16 delays).
Random numbers come from NumPy's PCG64 seeded per case.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Config:
    """One workload.  SI units (metres, seconds, m/s)."""

    name: str
    img_h: int
    img_w: int
    dx: float                 # image pixel pitch [m]
    n_t: int                  # transducers on the ring
    ring_radius: float        # [m]
    ring_phase: float         # angle of transducer 0 [rad]
    v0: float                 # SOS assumed by DAS [m/s]
    v_bg: float               # fixed background (water) SOS [m/s]
    sos_g: int                # pixel-grid SOS nodes per side
    p: int                    # patch size [px], even
    centres_rows: Tuple[int, ...]   # patch-centre rows (Cartesian grid with cols)
    centres_cols: Tuple[int, ...]
    m: int                    # delay channels
    tau_us: float             # delays span [-tau_us, +tau_us] microseconds
    eps: float                # Wiener-style regulariser added to sum |H|^2
    tv_lambda: float          # TV weight
    lr: float                 # Adam learning rate [m/s per step]
    steps: int                # Adam iterations
    noise_sigma: float        # additive Gaussian noise on the delay stack
    sos_kind: str             # "blobs" | "ellipses" | "uniform"
    ip_kind: str              # "disks_lines" | "vessels"
    sos_lo: float = 1450.0
    sos_hi: float = 1600.0
    # ring channel data (the input of Eq. 1 for end-to-end runs)
    rf_fs: float = 40e6                 # sample rate [Hz]
    rf_ns: int = 4096                   # samples per transducer
    rf_t0: float = 0.0                  # time of sample 0 [s]
    rf_sigma: float = 5.6269769760e-8   # pulse width [s]: spectrum peak 4 MHz, half-amplitude band 1.9-6.5 MHz

    # ---- derived geometry (configuration readings, not method arithmetic) ----
    @property
    def fov(self) -> float:
        return self.img_w * self.dx

    @property
    def sos_dx(self) -> float:
        """SOS nodes cover the image field of view."""
        return self.fov / self.sos_g

    @property
    def mask_radius(self) -> float:
        """Circular SOS mask: the disk inscribed in the field of view."""
        return 0.5 * self.fov

    @property
    def ray_step(self) -> float:
        return 0.5 * self.sos_dx

    @property
    def window_fwhm(self) -> float:
        """Window FWHM scaled from the paper's 1.5 mm on 3.2 mm patches."""
        return (1.5 / 3.2) * self.p * self.dx

    @property
    def n_patches(self) -> int:
        return len(self.centres_rows) * len(self.centres_cols)

    @property
    def n_freq(self) -> int:
        return self.p * (self.p // 2 + 1)

    def centres(self) -> np.ndarray:
        """Patch centres as int32 [N][2] (row, col), row-major over the grid."""
        rr, cc = np.meshgrid(np.asarray(self.centres_rows), np.asarray(self.centres_cols), indexing="ij")
        return np.stack([rr.ravel(), cc.ravel()], axis=1).astype(np.int32)

    def tau(self) -> np.ndarray:
        """Delay times [s], uniform over [-tau, +tau]."""
        if self.m == 1:
            return np.zeros(1)
        return np.linspace(-self.tau_us, self.tau_us, self.m) * 1e-6

    def delays(self) -> np.ndarray:
        """Delay distances d_j [m] as float32: the stated times at the assumed SOS."""
        return (self.tau() * self.v0).astype(np.float32)

    def geometry_dict(self) -> dict:
        return dict(n_t=self.n_t, ring_radius=self.ring_radius, ring_phase=self.ring_phase,
                    v0=self.v0, v_bg=self.v_bg, img_h=self.img_h, img_w=self.img_w, dx=self.dx,
                    sos_g=self.sos_g, sos_dx=self.sos_dx, mask_radius=self.mask_radius,
                    ray_step=self.ray_step, p=self.p, window_fwhm=self.window_fwhm)

    def replace(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


def config_small() -> Config:
    """128x128 image at 0.2 mm, 256-element ring of radius 15 mm, 3x3 patches of
    32x32, 8 delays over +-0.5 us, 32x32 SOS grid with two Gaussian blobs."""
    return Config(name="pg128_ring256_p32_m8", img_h=128, img_w=128, dx=0.2e-3, n_t=256,
                  ring_radius=15e-3, ring_phase=0.0, v0=1500.0, v_bg=1500.0, sos_g=32, p=32,
                  centres_rows=(32, 64, 96), centres_cols=(32, 64, 96), m=8, tau_us=0.5,
                  eps=1e-3, tv_lambda=1e-4, lr=1.0, steps=50, noise_sigma=0.01,
                  sos_kind="blobs", ip_kind="disks_lines", sos_lo=1450.0, sos_hi=1550.0)


def config_full() -> Config:
    """512x512 image at 0.1 mm, 512-element ring of radius 40 mm, 12x12 patches of
    80x80 at stride 40 (144 patches), 32 delays, 128x128 SOS grid with 1-6
    Gaussian ellipses in 1450-1600 m/s, vessel-tree initial pressure.

    TV weight 1: the paper picks its weight as the best of an ablation over
    lambda (Sec. S3.2) under its own, unstated, normalisation of the data term;
    the same selection (SOS error after 1000 cold iterations, five seeded
    phantoms, lambda in {1e-4, 0.3, 1, 3}) on this workload's normalisation
    (sum over patches, channels and half-spectrum bins, |k| in rad/mm, TV in
    m/s) picks 1."""
    cs = tuple(36 + 40 * k for k in range(12))
    return Config(name="pg512_ring512_p80_m32", img_h=512, img_w=512, dx=0.1e-3, n_t=512,
                  ring_radius=40e-3, ring_phase=0.0, v0=1500.0, v_bg=1500.0, sos_g=128, p=80,
                  centres_rows=cs, centres_cols=cs, m=32, tau_us=0.5, eps=1e-3, tv_lambda=1.0,
                  lr=1.0, steps=1000, noise_sigma=0.01, sos_kind="ellipses", ip_kind="vessels")


def config_rf() -> Config:
    """1024x1024 image at 0.05 mm from 1024-element ring channel data, 64x64
    patches at stride 16 (61x61 = 3721 patches), 32 delays, 256x256 SOS grid."""
    cs = tuple(32 + 16 * k for k in range(61))
    return Config(name="rf1024_ring1024_p64_m32", img_h=1024, img_w=1024, dx=0.05e-3, n_t=1024,
                  ring_radius=40e-3, ring_phase=0.0, v0=1500.0, v_bg=1500.0, sos_g=256, p=64,
                  centres_rows=cs, centres_cols=cs, m=32, tau_us=0.5, eps=1e-3, tv_lambda=0.0,
                  lr=1.0, steps=100, noise_sigma=0.01, sos_kind="ellipses", ip_kind="vessels")


def config_tiny(p: int = 16, m: int = 4, n_t: int = 64, grid: int = 2) -> Config:
    """A few patches of P x P on a 64x64 image: for brute-force and FD checks."""
    img = 64
    step = img // (grid + 1)
    cs = tuple(step * (k + 1) for k in range(grid))
    return Config(name=f"tiny_p{p}_m{m}", img_h=img, img_w=img, dx=0.2e-3, n_t=n_t,
                  ring_radius=9e-3, ring_phase=0.1, v0=1500.0, v_bg=1500.0, sos_g=16, p=p,
                  centres_rows=cs, centres_cols=cs, m=m, tau_us=0.5, eps=1e-3, tv_lambda=1e-4,
                  lr=1.0, steps=5, noise_sigma=0.01, sos_kind="blobs", ip_kind="disks_lines",
                  sos_lo=1450.0, sos_hi=1550.0)


# --------------------------------------------------------------------------
# seeded phantoms
# --------------------------------------------------------------------------

def _node_xy(cfg: Config) -> Tuple[np.ndarray, np.ndarray]:
    """SOS node coordinates [m] (x along columns, y along rows), node centres."""
    g = cfg.sos_g
    c = (np.arange(g) - (g - 1) / 2.0) * cfg.sos_dx
    yy, xx = np.meshgrid(c, c, indexing="ij")
    return xx, yy


def _pixel_xy(cfg: Config) -> Tuple[np.ndarray, np.ndarray]:
    cx = (np.arange(cfg.img_w) - (cfg.img_w - 1) / 2.0) * cfg.dx
    cy = (np.arange(cfg.img_h) - (cfg.img_h - 1) / 2.0) * cfg.dx
    yy, xx = np.meshgrid(cy, cx, indexing="ij")
    return xx, yy


def sos_mask(cfg: Config) -> np.ndarray:
    """Nodes whose centre lies inside the circular mask (trainable nodes)."""
    xx, yy = _node_xy(cfg)
    return (xx * xx + yy * yy) <= cfg.mask_radius ** 2


def ellipse_params(cfg: Config, rng: np.random.Generator) -> np.ndarray:
    """Seeded parameters of an "ellipses" SOS phantom: [n][6] rows of
    (cx, cy, sa, sb, theta, amp) in metres, radians and m/s, 1 <= n <= 6."""
    rm = cfg.mask_radius
    n = int(rng.integers(1, 7))
    out = np.zeros((n, 6))
    for e in range(n):
        r = 0.6 * rm * math.sqrt(rng.uniform())
        a = rng.uniform(0, 2 * math.pi)
        cx, cy = r * math.cos(a), r * math.sin(a)
        sa, sb = rng.uniform(0.06, 0.25) * rm, rng.uniform(0.06, 0.25) * rm
        th = rng.uniform(0, math.pi)
        amp = rng.uniform(cfg.sos_lo - cfg.v_bg, cfg.sos_hi - cfg.v_bg)
        out[e] = (cx, cy, sa, sb, th, amp)
    return out


def sos_phantom(cfg: Config, rng: np.random.Generator) -> np.ndarray:
    """Ground-truth SOS on the node grid [G][G] (float64, m/s)."""
    xx, yy = _node_xy(cfg)
    rm = cfg.mask_radius
    v = np.full(xx.shape, cfg.v_bg)
    if cfg.sos_kind == "blobs":
        for _ in range(2):
            r = 0.55 * rm * math.sqrt(rng.uniform())
            a = rng.uniform(0, 2 * math.pi)
            cx, cy = r * math.cos(a), r * math.sin(a)
            sig = rng.uniform(2e-3, 4e-3)
            amp = 50.0 * (1 if rng.uniform() < 0.5 else -1)
            v = v + amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig))
    elif cfg.sos_kind == "ellipses":
        for cx, cy, sa, sb, th, amp in ellipse_params(cfg, rng):
            ux = (xx - cx) * math.cos(th) + (yy - cy) * math.sin(th)
            uy = -(xx - cx) * math.sin(th) + (yy - cy) * math.cos(th)
            v = v + amp * np.exp(-0.5 * ((ux / sa) ** 2 + (uy / sb) ** 2))
        v = np.clip(v, cfg.sos_lo, cfg.sos_hi)
    elif cfg.sos_kind == "uniform":
        pass
    else:
        raise ValueError(cfg.sos_kind)
    v[~sos_mask(cfg)] = cfg.v_bg
    return v


def _segment_dist(xx, yy, p0, p1):
    d = np.asarray(p1) - np.asarray(p0)
    L2 = float(d @ d) + 1e-30
    t = np.clip(((xx - p0[0]) * d[0] + (yy - p0[1]) * d[1]) / L2, 0.0, 1.0)
    return np.hypot(xx - (p0[0] + t * d[0]), yy - (p0[1] + t * d[1]))


def ip_phantom(cfg: Config, rng: np.random.Generator) -> np.ndarray:
    """Ground-truth initial-pressure image [H][W] in [0, 1] (float64)."""
    xx, yy = _pixel_xy(cfg)
    img = np.zeros(xx.shape)
    rmax = 0.8 * cfg.mask_radius
    if cfg.ip_kind == "disks_lines":
        for _ in range(int(rng.integers(4, 8))):
            r = rmax * math.sqrt(rng.uniform())
            a = rng.uniform(0, 2 * math.pi)
            rad = rng.uniform(0.3e-3, 1.5e-3)
            amp = rng.uniform(0.3, 1.0)
            d = np.hypot(xx - r * math.cos(a), yy - r * math.sin(a))
            img = np.maximum(img, amp * (d <= rad))
        for _ in range(int(rng.integers(3, 6))):
            p0 = rng.uniform(-rmax, rmax, 2)
            p1 = rng.uniform(-rmax, rmax, 2)
            w = rng.uniform(0.1e-3, 0.25e-3)
            amp = rng.uniform(0.3, 1.0)
            img = np.maximum(img, amp * (_segment_dist(xx, yy, p0, p1) <= w))
    elif cfg.ip_kind == "vessels":
        # random branching polylines (vessel tree), widths 0.1-0.5 mm
        stack = []
        for _ in range(int(rng.integers(2, 4))):
            a = rng.uniform(0, 2 * math.pi)
            stack.append((np.array([0.9 * rmax * math.cos(a), 0.9 * rmax * math.sin(a)]),
                          a + math.pi + rng.uniform(-0.5, 0.5), rng.uniform(0.3e-3, 0.5e-3), 0))
        segs = []
        while stack and len(segs) < 160:
            p0, ang, wid, depth = stack.pop()
            length = rng.uniform(0.08, 0.2) * rmax
            p1 = p0 + length * np.array([math.cos(ang), math.sin(ang)])
            if np.hypot(*p1) > rmax:
                continue
            segs.append((p0, p1, wid, rng.uniform(0.5, 1.0)))
            nxt = ang + rng.normal(0.0, 0.25)
            stack.append((p1, nxt, wid, depth + 1))
            if depth < 6 and rng.uniform() < 0.45:
                stack.append((p1, ang + rng.choice([-1, 1]) * rng.uniform(0.4, 1.1),
                              max(0.1e-3, wid * rng.uniform(0.6, 0.85)), depth + 1))
        for p0, p1, wid, amp in segs:
            dist = _segment_dist(xx, yy, p0, p1)
            img = np.maximum(img, amp * np.clip(1.0 - dist / (0.5 * wid), 0.0, 1.0) ** 0.5)
    else:
        raise ValueError(cfg.ip_kind)
    return img


def ellipse_phantoms_batch(cfg: Config, params: List[np.ndarray], device, dtype=None):
    """The "ellipses" phantoms of sos_phantom for a list of parameter sets
    (from ellipse_params, in the same order of random draws) evaluated at once
    with torch on `device`: [S][G][G] (float32 unless `dtype`)."""
    import torch
    dt = torch.float64 if dtype is None else dtype
    S = len(params)
    xx, yy = (torch.as_tensor(a, dtype=dt, device=device) for a in _node_xy(cfg))
    nmax = max(1, max(len(p) for p in params))
    P = np.zeros((S, nmax, 6))
    P[:, :, 2:4] = 1.0                                  # padding: zero amplitude
    for k, p in enumerate(params):
        P[k, :len(p)] = p
    P = torch.as_tensor(P, dtype=dt, device=device)
    cx, cy, sa, sb, th, amp = (P[:, :, q, None, None] for q in range(6))
    dx, dy = xx[None, None] - cx, yy[None, None] - cy
    ux = dx * torch.cos(th) + dy * torch.sin(th)
    uy = -dx * torch.sin(th) + dy * torch.cos(th)
    v = cfg.v_bg + (amp * torch.exp(-0.5 * ((ux / sa) ** 2 + (uy / sb) ** 2))).sum(1)
    v = v.clamp(cfg.sos_lo, cfg.sos_hi)
    mask = torch.as_tensor(sos_mask(cfg), device=device)
    v = torch.where(mask[None], v, torch.full_like(v, cfg.v_bg))
    return v.to(torch.float32 if dtype is None else dtype)


def make_case(cfg: Config, seed: int) -> dict:
    """All seeded inputs of one recovery problem, as float32 / int32 arrays.

    sos_true  [G][G]   ground-truth SOS (nodes outside the mask at v_bg)
    sos_init  [G][G]   uniform v_bg start
    mask      [G][G]   uint8 trainable-node mask
    ip        [H][W]   ground-truth initial pressure
    noise     [M][H][W] N(0, sigma^2) per pixel of every delay channel
    d         [M]      delay distances [m]
    centres   [N][2]   patch centres (row, col)
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sos_true = sos_phantom(cfg, rng)
    ip = ip_phantom(cfg, rng)
    noise = rng.standard_normal((cfg.m, cfg.img_h, cfg.img_w)) * cfg.noise_sigma
    return dict(
        sos_true=sos_true.astype(np.float32),
        sos_init=np.full((cfg.sos_g, cfg.sos_g), cfg.v_bg, np.float32),
        mask=sos_mask(cfg).astype(np.uint8),
        ip=ip.astype(np.float32),
        noise=noise.astype(np.float32),
        d=cfg.delays(),
        centres=cfg.centres(),
    )


def random_wavefronts(n: int, n_t: int, rng: np.random.Generator, scale: float = 3e-4) -> np.ndarray:
    """Smooth random per-transducer wavefront errors [N][N_t] (metres): a few
    random low-order Fourier harmonics in the ring angle plus a constant."""
    a = 2 * np.pi * np.arange(n_t) / n_t
    w = np.zeros((n, n_t))
    for h in range(0, 6):
        c = rng.normal(0, scale / (1 + h), (n, 1))
        s = rng.normal(0, scale / (1 + h), (n, 1))
        w += c * np.cos(h * a) + s * np.sin(h * a)
    return w.astype(np.float32)


def random_spectra(shape: Tuple[int, ...], rng: np.random.Generator) -> np.ndarray:
    """Complex64 array with standard-normal real and imaginary parts."""
    z = rng.standard_normal(shape + (2,)).astype(np.float32)
    return z


def random_rf(n_t: int, n_s: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal((n_t, n_s)).astype(np.float32)


# --------------------------------------------------------------------------
# neural-field SOS parametrisation: sizes and seeded initial parameters
# --------------------------------------------------------------------------

NF_FREQS = 16          # log-spaced frequencies, 1 .. 64 cycles per field of view
NF_FEATURES = 4 * NF_FREQS
NF_HIDDEN = 128
NF_LAYERS = 4          # hidden layers
NF_V_MID, NF_V_HALF = 1525.0, 125.0      # v = 1525 + 125 tanh(z) spans 1400 .. 1650 m/s


def nf_frequencies() -> np.ndarray:
    """Fourier-feature frequencies f_l (cycles per field of view)."""
    return np.logspace(0.0, np.log10(64.0), NF_FREQS)


def nf_shapes():
    """(name, shape) of the neural-field parameters in their flat order."""
    sh = [("W1", (NF_HIDDEN, NF_FEATURES)), ("b1", (NF_HIDDEN,))]
    for l in range(2, NF_LAYERS + 1):
        sh += [(f"W{l}", (NF_HIDDEN, NF_HIDDEN)), (f"b{l}", (NF_HIDDEN,))]
    sh += [("w5", (NF_HIDDEN,)), ("b5", (1,))]
    return sh


def nf_param_count() -> int:
    return int(sum(np.prod(s) for _, s in nf_shapes()))


# Adam learning rate of the Fourier-feature MLP field.  Measured on the benchmark
# workload (1000 iterations from a uniform 1500 m/s field): at 5e-3 the tanh
# output of every node saturates on phantom 0 (the loss stops at its starting
# value); at 1e-3 no node saturates on phantoms 0 and 1, and phantom 1 reaches
# the data loss of the true SOS (8585 against 8533) at 1.2 m/s RMS error.
NF_LR = 1e-3


def nf_init(seed: int, v_start: float = 1500.0) -> np.ndarray:
    """Seeded flat float32 parameter vector: U(-1/sqrt(fan_in), 1/sqrt(fan_in))
    for the hidden layers, a small output layer and an output bias that makes
    the initial field about v_start."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shape in nf_shapes():
        if name == "b5":
            parts.append(np.array([np.arctanh((v_start - NF_V_MID) / NF_V_HALF)]))
            continue
        fan_in = shape[1] if len(shape) == 2 else NF_HIDDEN
        bound = 1.0 / np.sqrt(fan_in)
        if name == "w5":
            bound *= 0.05
        parts.append(rng.uniform(-bound, bound, size=shape).ravel())
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# warm-start CNN: sizes, seeded initial parameters, training-set phantoms
# --------------------------------------------------------------------------

CNN_POOL = 4           # the M x 512 x 512 delay stack is averaged over 4 x 4 pixels
CNN_RES = 128          # input side after pooling
CNN_OUT = 32           # output SOS side (upsampled x4 to the 128 x 128 node grid)
# (c_in, c_out, 2 x 2 average pooling after the layer); c_in of the first is M
CNN_CONVS = ((None, 32, True), (32, 64, True), (64, 64, False), (64, 64, False), (64, 64, False))
CNN_V_MID, CNN_V_HALF = 1525.0, 125.0    # v = 1525 + 125 tanh(z) spans 1400 .. 1650 m/s
CNN_V_SCALE = 100.0                      # training loss: mean ((v - v_true) / 100 m/s)^2


def cnn_shapes(m: int = 32):
    """(name, shape) of the CNN parameters in their flat order: five 3x3
    convolutions W_l [c_out][c_in][3][3], b_l [c_out], then the 1x1 head
    w6 [64], b6 [1]."""
    sh = []
    for l, (cin, cout, _) in enumerate(CNN_CONVS, start=1):
        cin = m if cin is None else cin
        sh += [(f"W{l}", (cout, cin, 3, 3)), (f"b{l}", (cout,))]
    sh += [("w6", (CNN_CONVS[-1][1],)), ("b6", (1,))]
    return sh


def cnn_param_count(m: int = 32) -> int:
    return int(sum(np.prod(s) for _, s in cnn_shapes(m)))


def cnn_init(seed: int, m: int = 32, v_start: float = 1500.0) -> np.ndarray:
    """Seeded flat float32 parameters: U(-sqrt(6/fan_in), sqrt(6/fan_in)) for the
    convolutions, zero biases, a small head and a head bias that makes the
    initial output about v_start."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shape in cnn_shapes(m):
        if name == "b6":
            parts.append(np.array([np.arctanh((v_start - CNN_V_MID) / CNN_V_HALF)]))
        elif name.startswith("b"):
            parts.append(np.zeros(shape))
        elif name == "w6":
            parts.append(rng.uniform(-0.01, 0.01, size=shape))
        else:
            bound = math.sqrt(6.0 / (shape[1] * 9))
            parts.append(rng.uniform(-bound, bound, size=shape).ravel())
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def config_cnn() -> Config:
    """The full-size problem with training phantoms of 1-6 ellipses spanning
    1400-1650 m/s (the warm-start network's training distribution)."""
    return config_full().replace(name="cnn512_ring512_p80_m32", sos_lo=1400.0, sos_hi=1650.0)


def config_held_out() -> Config:
    """The held-out problem of the warm-start benchmark: the full-size problem
    with its SOS phantom drawn from the network's training range (1-6 ellipses,
    1400-1650 m/s)."""
    return config_full().replace(name="pg512_ring512_p80_m32_sos1400_1650", sos_lo=1400.0, sos_hi=1650.0)


# --------------------------------------------------------------------------
# the paper's neural field: SIREN without hidden layers, 256 sine features
# --------------------------------------------------------------------------

SIREN_FEATURES = 256
SIREN_OMEGA0 = 30.0    # sine frequency factor of the SIREN first layer
SIREN_LR = 5e-3        # Adam learning rate for the neural field (Sec. 3.3)


def siren_shapes():
    """(name, shape) of the SIREN parameters in their flat order: W1 [256][2],
    b1 [256], w2 [256], b2 [1], then the output scale and offset (1027 in all)."""
    f = SIREN_FEATURES
    return [("W1", (f, 2)), ("b1", (f,)), ("w2", (f,)), ("b2", (1,)), ("scale", (1,)), ("offset", (1,))]


def siren_param_count() -> int:
    return int(sum(np.prod(s) for _, s in siren_shapes()))


def siren_init(seed: int, v_start: float = 1500.0, scale: float = 50.0) -> np.ndarray:
    """Seeded flat float32 parameters with the SIREN initialisation: first
    layer U(-1/2, 1/2) (fan-in 2), biases U(-1/sqrt 2, 1/sqrt 2), output layer
    U(-sqrt(6/256)/omega0, +sqrt(6/256)/omega0), b2 = 0; output scale `scale` m/s
    and offset v_start."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = SIREN_FEATURES
    W1 = rng.uniform(-0.5, 0.5, (f, 2))
    b1 = rng.uniform(-1 / np.sqrt(2.0), 1 / np.sqrt(2.0), f)
    bw = np.sqrt(6.0 / f) / SIREN_OMEGA0
    w2 = rng.uniform(-bw, bw, f)
    return np.concatenate([W1.ravel(), b1, w2, [0.0], [scale], [v_start]]).astype(np.float32)
