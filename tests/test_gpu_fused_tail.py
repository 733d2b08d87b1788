"""The four-kernel recovery iteration (rays with the TV terms of Eq. 7, fused
pass, ray adjoint, one kernel for the partial-grid sum + TV subgradient +
Adam) against the same iteration from the separate entry points
(pact_sos_to_delays_clear, the fused pass, pact_sos_to_delays_adj, pact_tv,
pact_adam_step), step by step from the same state (Sec. 3.3)."""
import numpy as np
import pytest
import torch

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs, pact

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _setup(cfg, seed):
    case = inputs.make_case(cfg, seed)
    Y = torch.as_tensor(O.make_measurement(O.geom(cfg), case)[0].numpy().astype(np.complex64), device=DEV)
    pb = pact.Problem(cfg, DEV)
    mask = torch.as_tensor(case["mask"].astype(np.uint8), device=DEV)
    return pb, case, Y, mask


class _State:
    def __init__(self, pb, case):
        self.sos = torch.as_tensor(case["sos_init"], device=DEV).clone()
        self.m = torch.zeros_like(self.sos)
        self.v = torch.zeros_like(self.sos)
        self.counter = torch.zeros(2, dtype=torch.int32, device=DEV)
        self.grad = torch.zeros_like(self.sos)
        self.w = torch.empty((pb.n, pb.n_t), dtype=torch.float32, device=DEV)
        self.out = {"loss": torch.zeros(1, dtype=torch.float32, device=DEV),
                    "dL_dw": torch.zeros((pb.n, pb.n_t), dtype=torch.float32, device=DEV)}


@pytest.mark.parametrize("name,lam", [("small", 0.5), ("small", 0.0), ("full", 1.0)])
def test_fused_iteration_equals_separate_calls(name, lam):
    """Each step from the same state (the separate path starts from the fused
    path's state): the two differ only by summation order (and the fused pass's
    float atomics), which Adam's sign-like first steps would amplify along two
    separate trajectories."""
    cfg = inputs.config_small() if name == "small" else inputs.config_full()
    pb, case, Y, mask = _setup(cfg, 21)
    d, eps, lr = case["d"], cfg.eps, 2.0
    tables = pact.McdTables(pb, np.asarray(d, np.float32), DEV)
    ws_mcd = pact._ws(tables.scratch_bytes, DEV)
    ws_adj = pact._ws(pact.sos_to_delays_adj_workspace_size(pb), DEV)
    ws_tv = pact._ws(pact.sos_to_delays_tv_workspace_size(pb), DEV) if lam else None
    A, B = _State(pb, case), _State(pb, case)
    for it in range(4):
        for name_ in ("sos", "m", "v", "counter"):
            getattr(B, name_).copy_(getattr(A, name_))
        sos0 = A.sos.clone()
        # fused: four kernels
        if ws_tv is not None:
            pact.sos_to_delays_tv(pb, A.sos, A.w, A.out["dL_dw"], lam, ws_tv)
        else:
            pact.sos_to_delays(pb, A.sos, A.w, clear=A.out["dL_dw"])
        pact.mc_deconv_loss(pb, A.w, Y, d, eps, want_grad=True, out=A.out, ws=ws_mcd, tables=tables, accumulate=True)
        pact.sos_to_delays_adj_adam(pb, A.sos, A.out["dL_dw"], A.m, A.v, lr, mask=mask, step_counter=A.counter,
                                    tv_ws=ws_tv, loss=A.out["loss"], grad=A.grad, ws=ws_adj)
        # separate entry points, same starting state
        pact.sos_to_delays(pb, B.sos, B.w, clear=B.out["dL_dw"])
        pact.mc_deconv_loss(pb, B.w, Y, d, eps, want_grad=True, out=B.out, ws=ws_mcd, tables=tables, accumulate=True)
        pact.sos_to_delays_adj(pb, B.sos, B.out["dL_dw"], B.grad, accumulate=False, ws=ws_adj)
        if lam:
            pact.tv(pb, B.sos, lam, value=B.out["loss"], grad=B.grad, accumulate=True)
        pact.adam_step(B.sos, B.grad, B.m, B.v, 1, lr, mask=mask, step_counter=B.counter)
        torch.cuda.synchronize()
        la, lb = float(A.out["loss"].item()), float(B.out["loss"].item())
        assert abs(la - lb) <= 1e-6 * abs(lb), (it, la, lb)
        assert _rel(A.w.cpu(), B.w.cpu()) == 0.0, it
        gB = B.grad.cpu().numpy()
        assert _rel(A.grad.cpu(), gB) <= 1e-5, it
        assert _rel(A.m.cpu(), B.m.cpu()) <= 1e-5 and _rel(A.v.cpu(), B.v.cpu()) <= 1e-5, it
        # the Adam update where the gradient is clear of rounding noise
        dA, dB = (A.sos - sos0).cpu().numpy(), (B.sos - sos0).cpu().numpy()
        firm = np.abs(gB) > 1e-3 * np.abs(gB).max()
        assert firm.sum() > 0.2 * case["mask"].sum(), it
        np.testing.assert_allclose(dA[firm], dB[firm], rtol=1e-4, atol=1e-4 * lr)
        assert A.counter.cpu().tolist() == B.counter.cpu().tolist() == [it + 1, 0]
    # masked nodes never move
    off = ~case["mask"].astype(bool)
    assert np.array_equal(A.sos.cpu().numpy()[off], case["sos_init"][off])


def test_tv_terms_match_the_oracle():
    cfg = inputs.config_small()
    pb, case, Y, mask = _setup(cfg, 22)
    sos = torch.as_tensor(case["sos_true"], device=DEV) + 0.25 * torch.randn(cfg.sos_g, cfg.sos_g, device=DEV)
    lam = 0.75
    ws_tv = pact._ws(pact.sos_to_delays_tv_workspace_size(pb), DEV)
    w = torch.empty((pb.n, pb.n_t), dtype=torch.float32, device=DEV)
    clear = torch.ones((pb.n, pb.n_t), dtype=torch.float32, device=DEV)
    pact.sos_to_delays_tv(pb, sos, w, clear, lam, ws_tv)
    torch.cuda.synchronize()
    g = ws_tv.view(torch.float32)[: cfg.sos_g ** 2].cpu().numpy().reshape(cfg.sos_g, cfg.sos_g)
    s = torch.tensor(sos.cpu().numpy().astype(np.float64), requires_grad=True)
    tv = O.tv(s)
    (gt,) = torch.autograd.grad(tv, s)
    assert _rel(g, lam * gt.numpy()) <= 1e-6
    assert float(clear.abs().max()) == 0.0
    assert _rel(w.cpu(), pact.sos_to_delays(pb, sos).cpu()) == 0.0


def test_fused_tail_rejects_bad_arguments():
    cfg = inputs.config_small()
    pb, case, Y, mask = _setup(cfg, 23)
    sos = torch.as_tensor(case["sos_init"], device=DEV).clone()
    w = torch.empty((pb.n, pb.n_t), dtype=torch.float32, device=DEV)
    clear = torch.zeros((pb.n, pb.n_t), dtype=torch.float32, device=DEV)
    small = pact._ws(256, DEV)
    with pytest.raises(pact.PactError):
        pact.sos_to_delays_tv(pb, sos, w, clear, 1.0, small)
    ws_tv = pact._ws(pact.sos_to_delays_tv_workspace_size(pb), DEV)
    with pytest.raises(pact.PactError):
        pact.sos_to_delays_tv(pb, sos, w, clear, float("nan"), ws_tv)
    m, v = torch.zeros_like(sos), torch.zeros_like(sos)
    with pytest.raises(pact.PactError):
        pact.sos_to_delays_adj_adam(pb, sos, clear, m, v, 1.0, beta1=1.5, ws=pact._ws(pact.sos_to_delays_adj_workspace_size(pb), DEV))
    with pytest.raises(pact.PactError):
        pact.sos_to_delays_adj_adam(pb, sos, clear, m, v, 1.0, ws=small)
