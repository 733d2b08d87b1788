"""Failure detection of the fused pass on the GPU, without faulting it.

Every device-side wait of the fused deconvolution pass is bounded by the
library's wait limit.  The test hook pact_mc_deconv_inject_stall sets a flag
in the prebuilt tables that makes the consumer warps withhold the release of
their first pipeline stage: the producer's wait for that release runs into
the limit, the consumers' wait for the next stage does too, the outputs turn
NaN and a timeout is recorded in the status word; the kernel returns, the
context stays usable and the next call is normal.

The second test runs the pass while a side stream keeps the SMs busy: no CTA
of the pass waits for another CTA that may not be resident, so the result does
not depend on how many of its CTAs the GPU can hold at once.
"""
import numpy as np
import pytest
import torch

from paper_2409_10876_gb300 import inputs, pact

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _problem(cfg, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((cfg.n_patches, cfg.m, cfg.p, cfg.p // 2 + 1, 2), dtype=np.float32)
    Y = torch.as_tensor(np.ascontiguousarray(z.view(np.complex64)[..., 0]), device=DEV)
    w = torch.as_tensor(inputs.random_wavefronts(cfg.n_patches, cfg.n_t, rng), device=DEV)
    return pact.Problem(cfg, DEV), Y, w


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_bounded_wait_expires_reports_timeout_and_recovers():
    cfg = inputs.config_small()
    pb, Y, w = _problem(cfg, 3)
    d = cfg.delays()
    tables = pact.McdTables(pb, d)
    ref = pact.mc_deconv_loss(pb, w, Y, d, cfg.eps, tables=tables)
    torch.cuda.synchronize()
    ref_loss, ref_g = float(ref["loss"].item()), ref["dL_dw"].cpu().numpy()
    assert np.isfinite(ref_loss)
    pact.mc_deconv_status(pb, cfg.m, tables=tables)              # nothing to report

    assert pact.wait_limit_ns() == 200_000_000
    pact.set_wait_limit_ns(2_000_000)                               # 2 ms
    try:
        assert pact.wait_limit_ns() == 2_000_000
        pact.mc_deconv_inject_stall(pb, tables)
        bad = pact.mc_deconv_loss(pb, w, Y, d, cfg.eps, tables=tables)
        torch.cuda.synchronize()
        with pytest.raises(pact.PactError, match="status 4"):
            pact.mc_deconv_status(pb, cfg.m, tables=tables)
        assert not np.isfinite(float(bad["loss"].item()))
        assert np.isnan(bad["dL_dw"].cpu().numpy()).any()
    finally:
        pact.set_wait_limit_ns(0)
    assert pact.wait_limit_ns() == 200_000_000

    # the status word was cleared by the read, the stall flag by the launch
    pact.mc_deconv_status(pb, cfg.m, tables=tables)
    again = pact.mc_deconv_loss(pb, w, Y, d, cfg.eps, tables=tables)
    torch.cuda.synchronize()
    pact.mc_deconv_status(pb, cfg.m, tables=tables)
    assert abs(float(again["loss"].item()) - ref_loss) <= 1e-6 * abs(ref_loss)
    assert _rel(again["dL_dw"].cpu().numpy(), ref_g) <= 1e-5


def test_wait_limit_rejects_out_of_range():
    with pytest.raises(pact.PactError):
        pact.set_wait_limit_ns(10)
    with pytest.raises(pact.PactError):
        pact.set_wait_limit_ns(10**12)
    assert pact.wait_limit_ns() == 200_000_000


def test_fused_pass_beside_a_busy_stream():
    cfg = inputs.config_full()
    pb, Y, w = _problem(cfg, 4)
    d = cfg.delays()
    tables = pact.McdTables(pb, d)
    ref = pact.mc_deconv_loss(pb, w, Y, d, cfg.eps, tables=tables)
    torch.cuda.synchronize()
    ref_loss, ref_g = float(ref["loss"].item()), ref["dL_dw"].cpu().numpy()
    a = torch.randn(4096, 4096, device=DEV, dtype=torch.bfloat16)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    for _ in range(3):
        with torch.cuda.stream(side):              # long GEMMs that take SMs while the pass is launched
            for _ in range(8):
                a = torch.tanh(a @ a * 1e-3)
        out = pact.mc_deconv_loss(pb, w, Y, d, cfg.eps, tables=tables)
        torch.cuda.synchronize()
        pact.mc_deconv_status(pb, cfg.m, tables=tables)
        assert abs(float(out["loss"].item()) - ref_loss) <= 1e-6 * abs(ref_loss)
        assert _rel(out["dL_dw"].cpu().numpy(), ref_g) <= 1e-5
