"""One recovery problem split over ranks by patches (Sec. 3.3, Eq. 7).

The data term of Eq. 7 is a sum over patches, and every patch depends on the
one shared SOS.  So the patches (and their spectra Y) are partitioned across
ranks and the SOS parameters are replicated.  Per iteration every rank runs the
forward model and its adjoint for its own patches, giving a partial loss and
a partial gradient.  One all-reduce (sum) of the packed [gradient, loss]
follows.  Then every rank adds the TV term and takes the same Adam step, so the
replicas stay identical without a broadcast.

The host logic here does not depend on where the per-rank arithmetic runs.
`LibpactShard` runs it with the library's kernels on this rank's GPU; any
object with the same three methods can stand in for it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pact


def shard_range(n: int, world: int, rank: int):
    """Patches [lo, hi) of `rank`: contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    return n * rank // world, n * (rank + 1) // world


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def allreduce_sum(buf: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of `buf` over the ranks (no-op without a process group).
    A CUDA tensor under a CPU-only backend (gloo) goes through host memory."""
    dist = _dist()
    if dist is None or dist.get_world_size(group) == 1:
        return buf
    if buf.is_cuda and dist.get_backend(group) == "gloo":
        host = buf.cpu()
        dist.all_reduce(host, group=group)
        buf.copy_(host)
    else:
        dist.all_reduce(buf, group=group)
    return buf


class ShardedRecovery:
    """Adam on replicated parameters with the data term summed over ranks.

    `backend` provides, for this rank's patches:
      local(params) -> (loss [1], grad shaped like params)   data term (Eq. 7)
      regularise(params, loss [1], grad)                      adds lambda TV in place
      adam(params, grad)                                      one Adam step in place
    """

    def __init__(self, backend, params: torch.Tensor, group=None):
        self.backend, self.params, self.group = backend, params, group
        n = params.numel()
        self.packed = torch.zeros(n + 1, dtype=params.dtype, device=params.device)
        self.last_loss = None

    def step(self) -> torch.Tensor:
        loss, grad = self.backend.local(self.params)
        n = self.params.numel()
        self.packed[:n].copy_(grad.reshape(-1))
        self.packed[n:].copy_(loss.reshape(-1))
        allreduce_sum(self.packed, self.group)
        grad = self.packed[:n].view_as(self.params)
        loss = self.packed[n:]
        self.backend.regularise(self.params, loss, grad)
        self.backend.adam(self.params, grad)
        self.last_loss = loss
        return loss


class LibpactShard:
    """This rank's patches of a pixel-grid recovery on the library's kernels:
    sos_to_delays -> fused mc_deconv_loss + adjoint -> sos_to_delays_adj for the
    local patches; TV and Adam on the replicated SOS."""

    def __init__(self, cfg, Y_local: torch.Tensor, lo: int, hi: int, d, eps: float, lam: float, lr: float,
                 mask=None, device="cuda"):
        self.pb = pact.Problem(cfg, device, centres=cfg.centres()[lo:hi])
        self.Y = Y_local
        self.d = np.asarray(d, np.float32)
        self.eps, self.lam, self.lr = float(eps), float(lam), float(lr)
        dev = torch.device(device)
        self.mask = None if mask is None else torch.as_tensor(np.asarray(mask, np.uint8), device=dev)
        self.w = torch.empty((self.pb.n, self.pb.n_t), dtype=torch.float32, device=dev)
        self.out = {"loss": torch.zeros(1, dtype=torch.float32, device=dev),
                    "dL_dw": torch.zeros((self.pb.n, self.pb.n_t), dtype=torch.float32, device=dev)}
        self.grad = torch.empty((self.pb.g, self.pb.g), dtype=torch.float32, device=dev)
        self.tables = pact.McdTables(self.pb, self.d, dev)
        self.ws_mcd = pact._ws(self.tables.scratch_bytes, dev)
        self.ws_adj = pact._ws(pact.sos_to_delays_adj_workspace_size(self.pb), dev)
        self.m = torch.zeros((self.pb.g, self.pb.g), dtype=torch.float32, device=dev)
        self.v = torch.zeros_like(self.m)
        self.counter = torch.zeros(2, dtype=torch.int32, device=dev)

    def local(self, sos):
        pb = self.pb
        pact.sos_to_delays(pb, sos, self.w, clear=self.out["dL_dw"])
        pact.mc_deconv_loss(pb, self.w, self.Y, self.d, self.eps, want_grad=True, out=self.out, ws=self.ws_mcd,
                            tables=self.tables, accumulate=True)
        pact.sos_to_delays_adj(pb, sos, self.out["dL_dw"], self.grad, accumulate=False, ws=self.ws_adj)
        return self.out["loss"], self.grad

    def regularise(self, sos, loss, grad):
        if self.lam != 0.0:
            pact.tv(self.pb, sos, self.lam, value=loss, grad=grad, accumulate=True)

    def adam(self, sos, grad):
        pact.adam_step(sos, grad.contiguous(), self.m, self.v, 1, self.lr, mask=self.mask, step_counter=self.counter)
