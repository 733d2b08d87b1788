"""Pins of the oracle's neural-field SOS (the Fourier-feature MLP of the BF16
workload): features against their closed form, the output range, the
initialisation, and the gradient of the objective against central finite
differences on 64 random parameters."""
import math

import numpy as np
import torch

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs


def _nf_args(cfg):
    g = O.geom(cfg)
    return g, inputs.nf_shapes(), inputs.nf_frequencies(), inputs.sos_mask(cfg), inputs.NF_V_MID, inputs.NF_V_HALF


def test_features_closed_form():
    cfg = inputs.config_tiny()
    g = O.geom(cfg)
    f = inputs.nf_frequencies()
    feats = O.nf_features(g, f).numpy()
    G = cfg.sos_g
    p, q = 3, 11                                  # node row p (y), column q (x)
    x, y = (q - (G - 1) / 2) / G, (p - (G - 1) / 2) / G
    row = feats[p * G + q]
    for l in (0, 7, 15):
        assert abs(row[4 * l + 0] - math.sin(2 * math.pi * f[l] * x)) < 1e-14
        assert abs(row[4 * l + 1] - math.cos(2 * math.pi * f[l] * x)) < 1e-14
        assert abs(row[4 * l + 2] - math.sin(2 * math.pi * f[l] * y)) < 1e-14
        assert abs(row[4 * l + 3] - math.cos(2 * math.pi * f[l] * y)) < 1e-14
    assert abs(f[0] - 1.0) < 1e-15 and abs(f[-1] - 64.0) < 1e-12
    assert np.allclose(np.diff(np.log(f)), np.log(64.0) / 15)


def test_init_field_and_range():
    cfg = inputs.config_small()
    g, sh, f, mask, vm, vh = _nf_args(cfg)
    v = O.nf_sos(g, O._t(inputs.nf_init(0)), sh, f, mask, vm, vh).numpy()
    assert np.abs(v[mask > 0] - 1500.0).max() < 5.0
    assert np.all(v[mask == 0] == cfg.v_bg)
    big = O._t(inputs.nf_init(1)) * 40.0          # saturate: the output stays inside 1400-1650 m/s
    vb = O.nf_sos(g, big, sh, f, mask, vm, vh).numpy()
    assert vb.min() >= 1400.0 and vb.max() <= 1650.0


def test_nf_gradient_matches_finite_differences_on_64_parameters():
    cfg = inputs.config_tiny(p=16, m=4)
    g, sh, f, mask, vm, vh = _nf_args(cfg)
    case = inputs.make_case(cfg, 5)
    Y, _, _ = O.make_measurement(g, case)
    prm = inputs.nf_init(3).astype(np.float64)
    L0, _, gp = O.nf_objective(g, prm, sh, f, mask, vm, vh, Y, case["centres"], case["d"], cfg.eps)
    rng = np.random.default_rng(4)
    idx = rng.choice(prm.size, 64, replace=False)
    errs = []
    for k in idx:
        h = 1e-4 * max(1.0, abs(prm[k]))
        pp = prm.copy(); pp[k] += h
        pm = prm.copy(); pm[k] -= h
        fd = (float(O.nf_objective(g, pp, sh, f, mask, vm, vh, Y, case["centres"], case["d"], cfg.eps, False)[0])
              - float(O.nf_objective(g, pm, sh, f, mask, vm, vh, Y, case["centres"], case["d"], cfg.eps, False)[0])) / (2 * h)
        errs.append(abs(fd - float(gp[k])))
    assert max(errs) <= 1e-4 * float(gp.abs().max())


# ------------------------------------------------------------------ the paper's SIREN field

def _siren_args(cfg):
    return O.geom(cfg), inputs.siren_shapes(), inputs.sos_mask(cfg), inputs.SIREN_OMEGA0


def test_siren_size_and_closed_forms():
    assert inputs.siren_param_count() == 1027            # the count the paper states
    cfg = inputs.config_small()
    g, sh, mask, om = _siren_args(cfg)
    p = inputs.siren_init(0).astype(np.float64)
    # no output weights: v = offset + scale b2 everywhere on the mask
    q = p.copy()
    q[512 + 256:512 + 512] = 0.0
    q[-3], q[-2], q[-1] = 0.25, 8.0, 1510.0
    v = O.siren_sos(g, q, sh, mask, om).numpy()
    assert np.allclose(v[mask], 1512.0) and np.all(v[~mask] == cfg.v_bg)
    # one feature: v = offset + scale w2 sin(omega0 (a x + c y + b)) at the node coordinates
    q[:] = 0.0
    q[0], q[1], q[512], q[768] = 0.3, -0.7, 0.2, 2.0
    q[-2], q[-1] = 5.0, 1500.0
    xy = O.siren_coords(g).numpy()
    ref = 1500.0 + 5.0 * 2.0 * np.sin(om * (0.3 * xy[:, 0] - 0.7 * xy[:, 1] + 0.2))
    got = O.siren_sos(g, q, sh, np.ones_like(mask), om).numpy().ravel()
    assert np.allclose(got, ref, atol=1e-10)
    assert xy[:, 0].min() == -1.0 and xy[:, 0].max() == 1.0


def test_siren_initial_field_near_1500():
    cfg = inputs.config_small()
    g, sh, mask, om = _siren_args(cfg)
    v = O.siren_sos(g, inputs.siren_init(3).astype(np.float64), sh, mask, om).numpy()
    assert abs(v[mask].mean() - 1500.0) < 5.0 and v[mask].std() < 20.0


def test_siren_gradient_matches_central_differences():
    cfg = inputs.config_tiny(p=16, m=4)
    g, sh, mask, om = _siren_args(cfg)
    case = inputs.make_case(cfg, 2)
    Y, _, _ = O.make_measurement(g, case)
    p = inputs.siren_init(4).astype(np.float64)
    p[512 + 256:512 + 512] *= 20.0                        # a field that varies
    L, _, gp = O.siren_objective(g, p, sh, mask, om, Y, case["centres"], case["d"], 1e-3)
    rng = np.random.default_rng(5)
    for k in list(rng.choice(1024, 10, replace=False)) + [1024, 1025, 1026]:
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (float(O.siren_objective(g, pp, sh, mask, om, Y, case["centres"], case["d"], 1e-3, False)[0]) -
              float(O.siren_objective(g, pm, sh, mask, om, Y, case["centres"], case["d"], 1e-3, False)[0])) / (2 * h)
        gk = float(gp[k].item())
        assert abs(fd - gk) <= 2e-5 * max(abs(fd), abs(gk)) + 1e-9 * float(gp.abs().max()), (k, fd, gk)
