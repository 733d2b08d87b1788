"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/pact.h declares, and rejects invalid arguments on the host (these
calls return before any CUDA work, so no GPU is needed)."""
import ctypes
import os
import re

import pytest

from paper_2409_10876_gb300 import build as B
from paper_2409_10876_gb300 import inputs, pact

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pact_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pact.load(build_if_missing=False)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    assert set(_declared()) <= set(pact._SIGS)


def test_version(lib):
    assert b"sm_103a" in lib.pact_version()


def _geom(cfg):
    return pact.Geometry(*[cfg.geometry_dict()[k] for k, _ in pact.Geometry._fields_])


def test_null_geometry_rejected(lib):
    st = lib.pact_sos_to_delays(None, None, None, None, None)
    assert st == 1
    assert b"geometry" in lib.pact_last_error_message()


def test_bad_patch_size_rejected(lib):
    cfg = inputs.config_tiny()
    g = _geom(cfg)
    pt = pact._PatchesC(4, 15, 1234, 1e-3)          # odd P
    st = lib.pact_psf_synth(ctypes.byref(g), ctypes.byref(pt), 1, None, 4, 1, None)
    assert st == 2
    assert b"patch size" in lib.pact_last_error_message()


def test_too_many_channels_rejected(lib):
    cfg = inputs.config_tiny()
    g = _geom(cfg)
    pt = pact._PatchesC(4, 16, 1234, 1e-3)
    d = (ctypes.c_float * 65)()
    st = lib.pact_mc_deconv_loss(ctypes.byref(g), ctypes.byref(pt), 1, 1, d, 65, 1e-3, 1, None, None, None,
                                 None, 0, None)
    assert st == 2


def test_small_workspace_rejected(lib):
    cfg = inputs.config_tiny()
    g = _geom(cfg)
    pt = pact._PatchesC(4, 16, 1234, 1e-3)
    d = (ctypes.c_float * 4)(0, 1e-4, 2e-4, 3e-4)
    st = lib.pact_mc_deconv_loss(ctypes.byref(g), ctypes.byref(pt), 256, 256, d, 4, 1e-3, 256, None, None, None,
                                 256, 16, None)
    assert st == 1
    assert b"workspace" in lib.pact_last_error_message()


def test_negative_eps_and_bad_adam_rejected(lib):
    cfg = inputs.config_tiny()
    g = _geom(cfg)
    pt = pact._PatchesC(4, 16, 1234, 1e-3)
    d = (ctypes.c_float * 4)(0, 1e-4, 2e-4, 3e-4)
    assert lib.pact_mc_deconv_loss(ctypes.byref(g), ctypes.byref(pt), 256, 256, d, 4, -1.0, 256, None, None,
                                   None, 256, 1 << 30, None) == 1
    assert lib.pact_adam_step(10, 256, 256, 256, 256, 0, None, 0.1, 0.9, 0.999, 1e-8, None, None) == 1
    assert lib.pact_adam_step(10, 256, 256, 256, 256, 1, None, 0.1, 1.5, 0.999, 1e-8, None, None) == 1


def test_workspace_sizes_positive(lib):
    cfg = inputs.config_full()
    g = _geom(cfg)
    pt = pact._PatchesC(cfg.n_patches, cfg.p, 1234, cfg.window_fwhm)
    assert lib.pact_mc_deconv_loss_workspace_size(ctypes.byref(g), ctypes.byref(pt), 32) > cfg.n_patches * 4
    assert lib.pact_sos_to_delays_adj_workspace_size(ctypes.byref(g), ctypes.byref(pt)) >= cfg.sos_g ** 2 * 4
    assert lib.pact_stitch_workspace_size(ctypes.byref(g), ctypes.byref(pt)) >= 2 * 512 * 512 * 4


def test_rf_synth_rejects_bad_parameters(lib):
    cfg = inputs.config_tiny()
    g = _geom(cfg)
    ws_ok = lib.pact_rf_synth_workspace_size(ctypes.byref(g), 1)
    assert ws_ok >= cfg.n_t * 4
    assert lib.pact_rf_synth_workspace_size(ctypes.byref(g), 0) == 0
    fake = 4096                                      # never dereferenced: the calls fail on the host
    for rp, ws, code, msg in [
        (pact.RfParams(0.0, 0.0, 100, 4e-8, 0.0, 0.0), fake, 1, b"fs"),
        (pact.RfParams(40e6, 0.0, 100, -1.0, 0.0, 0.0), fake, 1, b"sigma"),
        (pact.RfParams(40e6, 0.0, 100, 4e-8, 0.0, -1.0), fake, 1, b"ring"),
        (pact.RfParams(40e6, 0.0, 1 << 20, 4e-8, 0.0, 0.0), fake, 2, b"n_s"),
        (pact.RfParams(40e6, 0.0, 100, 1e-3, 0.0, 0.0), fake, 2, b"sigma"),
        (pact.RfParams(40e6, 0.0, 100, 4e-8, 0.0, 0.0), fake + 8, 1, b"aligned"),
        (pact.RfParams(40e6, 0.0, 100, 4e-8, 0.0, 0.0), None, 1, b"workspace"),
    ]:
        st = lib.pact_rf_synth(ctypes.byref(g), fake, fake, ctypes.byref(rp), fake, ws, ws_ok, None)
        assert st == code, (rp.fs, rp.n_s, st)
        assert msg in lib.pact_last_error_message()
    rp = pact.RfParams(40e6, 0.0, 100, 4e-8, 0.0, 0.0)
    assert lib.pact_rf_synth(ctypes.byref(g), fake, fake, ctypes.byref(rp), fake, fake, 16, None) == 1


def test_fused_iteration_ends_reject_bad_arguments(lib):
    cfg = inputs.config_tiny()
    g = _geom(cfg)
    pt = pact._PatchesC(4, 16, 1234, 1e-3)
    need = lib.pact_sos_to_delays_tv_workspace_size(ctypes.byref(g), ctypes.byref(pt))
    assert need >= (cfg.sos_g ** 2) * 4 and need % 256 == 0
    # TV workspace: NULL, misaligned, too small, non-finite lambda
    assert lib.pact_sos_to_delays_tv(ctypes.byref(g), ctypes.byref(pt), 256, 256, 256, 16, 1.0, None, need, None) == 1
    assert lib.pact_sos_to_delays_tv(ctypes.byref(g), ctypes.byref(pt), 256, 256, 256, 16, 1.0, 272, need, None) == 1
    assert lib.pact_sos_to_delays_tv(ctypes.byref(g), ctypes.byref(pt), 256, 256, 256, 16, 1.0, 256, 16, None) == 1
    assert b"too small" in lib.pact_last_error_message()
    assert lib.pact_sos_to_delays_tv(ctypes.byref(g), ctypes.byref(pt), 256, 256, 256, 16, float("nan"), 256, need,
                                     None) == 1
    # adjoint + Adam: NULL moments, step 0 without a counter, betas out of range, NULL workspace
    args = lambda **kw: dict(dict(sos=256, dLdw=256, tv=None, loss=None, grad=None, m=256, v=256, step=1, cnt=None,
                                  lr=0.1, b1=0.9, b2=0.999, eps=1e-8, mask=None, ws=256, wsb=1 << 30), **kw)
    def call(a):
        return lib.pact_sos_to_delays_adj_adam(ctypes.byref(g), ctypes.byref(pt), a["sos"], a["dLdw"], a["tv"],
                                               a["loss"], a["grad"], a["m"], a["v"], a["step"], a["cnt"], a["lr"],
                                               a["b1"], a["b2"], a["eps"], a["mask"], a["ws"], a["wsb"], None)
    assert call(args(m=None)) == 1
    assert call(args(step=0)) == 1
    assert call(args(b1=1.5)) == 1
    assert call(args(ws=None)) == 1
    assert call(args(ws=272)) == 1
    assert call(args(tv=272)) == 1
