"""The patch-sharded recovery iteration (one problem's patches split over
ranks, one all-reduce of the SOS gradient and loss per iteration, replicated
TV and Adam) with world_size 2 over gloo on CPU ranks, each rank's data term
computed by the FP64 oracle: the sharded run equals the single-rank run of the
same problem step by step (Eq. 7 is a sum over patches, Sec. 3.3)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs
from paper_2409_10876_gb300.sharded import ShardedRecovery, shard_range

STEPS = 4


class OracleShard:
    """The data term of this rank's patches, TV and Adam from the FP64 oracle."""

    def __init__(self, cfg, case, Y, lo, hi):
        self.cfg, self.case, self.g = cfg, case, O.geom(cfg)
        self.cen = cfg.centres()[lo:hi]
        self.Y = Y[lo:hi]
        self.m = torch.zeros(cfg.sos_g, cfg.sos_g, dtype=torch.float64)
        self.v = torch.zeros_like(self.m)
        self.t = 0

    def local(self, sos):
        if len(self.cen) == 0:
            return torch.zeros(1, dtype=torch.float64), torch.zeros_like(sos)
        _, Ld, _, g = O.objective(self.g, sos, self.Y, self.cen, self.case["d"], self.cfg.eps, 0.0)
        return Ld.reshape(1), g

    def regularise(self, sos, loss, grad):
        s = sos.detach().clone().requires_grad_(True)
        tv = O.tv(s)
        (gt,) = torch.autograd.grad(tv, s)
        loss += self.cfg.tv_lambda * tv.detach()
        grad += self.cfg.tv_lambda * gt

    def adam(self, sos, grad):
        self.t += 1
        p, self.m, self.v = O.adam_step(sos, grad, self.m, self.v, self.t, self.cfg.lr, mask=self.case["mask"])
        sos.copy_(p)


def _problem():
    cfg = inputs.config_tiny(p=16, m=4, grid=3).replace(tv_lambda=0.5)      # 9 patches: ragged shards for 2 ranks
    case = inputs.make_case(cfg, 9)
    Y, _, _ = O.make_measurement(O.geom(cfg), case)
    return cfg, case, Y


def _run(world, rank):
    cfg, case, Y = _problem()
    lo, hi = shard_range(cfg.n_patches, world, rank)
    sos = torch.as_tensor(case["sos_init"], dtype=torch.float64).clone()
    rec = ShardedRecovery(OracleShard(cfg, case, Y, lo, hi), sos)
    hist = [float(rec.step()) for _ in range(STEPS)]
    return hist, sos.numpy()


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.set_num_threads(2)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = _run(world, rank)
    finally:
        dist.destroy_process_group()


def test_shard_range_partitions_the_patches():
    for n in (1, 9, 144, 3721):
        for world in (1, 2, 3, 8):
            rs = [shard_range(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def test_two_ranks_equal_one_rank():
    ref_hist, ref_sos = _run(1, 0)
    assert np.all(np.isfinite(ref_hist)) and len(set(ref_hist)) == STEPS
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        hist, sos = res[r]
        np.testing.assert_allclose(hist, ref_hist, rtol=1e-12)
        np.testing.assert_allclose(sos, ref_sos, rtol=1e-12, atol=1e-9)
    assert np.array_equal(res[0][1], res[1][1])              # the replicas are identical
