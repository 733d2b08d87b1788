"""pact_mc_deconv_loss_noalloc, the entry point for callers that cannot
allocate device memory (a plug-in whose host application owns all device
buffers, a real-time loop that must not allocate): it must give the same
outputs as pact_mc_deconv_loss with a caller workspace, on consecutive calls
that share its built-in scratch array, and must refuse problems whose scratch
need exceeds that array.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_10876_gb300 import inputs, pact

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.detach().cpu().numpy().astype(np.complex128)
    b = b.detach().cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _inputs(cfg, seed):
    rng = np.random.default_rng(seed)
    shp = (cfg.n_patches, cfg.m, cfg.p, cfg.p // 2 + 1)
    z = rng.standard_normal(shp + (2,)).astype(np.float32)
    Y = torch.as_tensor(np.ascontiguousarray(z[..., 0] + 1j * z[..., 1]).astype(np.complex64), device="cuda")
    w = torch.as_tensor(inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng), device="cuda")
    return w, Y


@pytest.mark.parametrize("cfg", [inputs.config_full(), inputs.config_small()], ids=["full", "small"])
def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(cfg):
    pb = pact.Problem(cfg, "cuda")
    need = pact.mc_deconv_loss_workspace_size(pb, cfg.m)
    assert need <= (16 << 20)
    d = cfg.delays()
    for call, seed in enumerate((1, 2)):          # two calls in a row on the shared scratch array
        w, Y = _inputs(cfg, seed)
        eps = cfg.eps if call == 0 else 1e-8      # second call also takes the FP64 path
        ref = pact.mc_deconv_loss(pb, w, Y, d, eps, want_grad=True, want_xhat=True, want_loss_pp=True)
        out = pact.mc_deconv_loss_noalloc(pb, w, Y, d, eps, want_grad=True, want_xhat=True, want_loss_pp=True)
        torch.cuda.synchronize()
        assert abs(float(out["loss"].item()) - float(ref["loss"].item())) <= 1e-4 * abs(float(ref["loss"].item()))
        assert _rel(out["loss_pp"], ref["loss_pp"]) <= 1e-4
        assert _rel(out["Xhat"], ref["Xhat"]) <= 1e-4
        assert _rel(out["dL_dw"], ref["dL_dw"]) <= 2e-3


def test_noalloc_rejects_problems_larger_than_its_scratch():
    cfg = inputs.config_rf()                      # 3721 patches x 1024 transducers: > 16 MiB of scratch
    pb = pact.Problem(cfg, "cuda")
    assert pact.mc_deconv_loss_workspace_size(pb, cfg.m) > (16 << 20)
    lib = pact.load()
    d = (ctypes.c_float * cfg.m)(*cfg.delays())
    # real device buffers, not made-up addresses (the size check returns before any launch)
    w, Y, loss = (torch.zeros(16, device="cuda") for _ in range(3))
    st = lib.pact_mc_deconv_loss_noalloc(pb.gp(), pb.pp(), w.data_ptr(), Y.data_ptr(), d, cfg.m, 1e-3,
                                         loss.data_ptr(), None, None, None, None)
    assert st == 2
    assert b"scratch" in lib.pact_last_error_message()
