"""The patch-sharded recovery on the library's kernels (one GPU): the partial
data terms and gradients of the shards add up to the whole problem's (Eq. 7
is a sum over patches), and a single-rank ShardedRecovery steps exactly like
PGRecovery.  (The exchange between ranks is covered over gloo in
tests/test_sharded.py.)"""
import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs, pact
from paper_2409_10876_gb300.recovery import PGRecovery
from paper_2409_10876_gb300.sharded import LibpactShard, ShardedRecovery, shard_range

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem():
    cfg = inputs.config_small()
    case = inputs.make_case(cfg, 6)
    Y = O.make_measurement(O.geom(cfg), case)[0].numpy().astype(np.complex64)
    return cfg, case, torch.as_tensor(Y, device=DEV)


@pytest.mark.parametrize("world", [2, 4])
def test_shards_add_up_to_the_whole(world):
    cfg, case, Y = _problem()
    sos = torch.as_tensor(case["sos_true"], device=DEV) + 3.0 * torch.as_tensor(case["mask"], device=DEV)
    pb = pact.Problem(cfg, DEV)
    w = pact.sos_to_delays(pb, sos)
    out = pact.mc_deconv_loss(pb, w, Y, case["d"], cfg.eps)
    g_full = pact.sos_to_delays_adj(pb, sos, out["dL_dw"])
    L_full = float(out["loss"].item())
    L, g = 0.0, torch.zeros_like(g_full)
    for r in range(world):
        lo, hi = shard_range(cfg.n_patches, world, r)
        sh = LibpactShard(cfg, Y[lo:hi].contiguous(), lo, hi, case["d"], cfg.eps, 0.0, 0.0, case["mask"], DEV)
        lr_, gr = sh.local(sos)
        L += float(lr_.item())
        g += gr
    torch.cuda.synchronize()
    assert abs(L - L_full) <= 1e-5 * abs(L_full)
    assert _rel(g.cpu().numpy(), g_full.cpu().numpy()) <= 1e-5


def test_single_rank_sharded_recovery_steps_like_pg_recovery():
    cfg, case, Y = _problem()
    args = (case["d"], cfg.eps, cfg.tv_lambda, cfg.lr)
    ref = PGRecovery(pact.Problem(cfg, DEV), Y, *args, torch.as_tensor(case["sos_init"]), torch.as_tensor(case["mask"]))
    ref_hist = []
    for _ in range(12):
        ref.step()
        ref_hist.append(ref.loss())
    sos = torch.as_tensor(case["sos_init"], device=DEV).clone()
    rec = ShardedRecovery(LibpactShard(cfg, Y, 0, cfg.n_patches, *args, case["mask"], DEV), sos)
    hist = [float(rec.step().item()) for _ in range(12)]
    np.testing.assert_allclose(hist, ref_hist, rtol=1e-5)
    assert _rel(sos.cpu().numpy(), ref.sos.cpu().numpy()) <= 1e-5
