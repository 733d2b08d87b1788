"""Host logic of warmstart.recover_warm (which branch runs, when the warm one
pauses or is dropped) on recoveries replaced by fixed loss trajectories: no
GPU.  The GPU test of the whole warm start is tests/test_gpu_warmstart.py."""
import types

import torch

from paper_2409_10876_gb300 import warmstart


class _Fake:
    def __init__(self, traj):
        self.traj, self.k, self.sos = traj, 0, torch.zeros(2)

    def capture(self):
        pass

    def iterate(self):
        self.k += 1

    def loss(self):
        return self.traj(self.k)


def _run(monkeypatch, warm, cold, iters=4000, target=None):
    trajs = [warm, cold]
    made = []

    def fake_pg(pb, Y, d, eps, lam, lr, v0, mask):
        made.append(_Fake(trajs[len(made)]))
        return made[-1]

    monkeypatch.setattr(warmstart, "PGRecovery", fake_pg)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    pb = types.SimpleNamespace(cfg=types.SimpleNamespace(v_bg=1500.0))
    Y = types.SimpleNamespace(device="cpu")
    return warmstart.recover_warm(pb, Y, None, 0.0, 0.0, 0.0, torch.zeros(2), None, iters, target=target), made


def test_good_warm_start_reaches_the_target_with_a_small_cold_share(monkeypatch):
    r, made = _run(monkeypatch, lambda k: 1.0 + 0.5 / (1 + k), lambda k: 1.0 + 5.0 / (1 + 0.01 * k), target=1.02)
    assert r["reached_s"] is not None and r["branch"] == "warm" and r["fallback"] is None
    assert r["iters"]["C"] * 4 <= r["iters"]["W"]


def test_stuck_warm_start_pauses_and_the_cold_branch_takes_over(monkeypatch):
    r, _ = _run(monkeypatch, lambda k: 1.3 + 2.0 / (1 + k), lambda k: 1.0 + 5.0 / (1 + 0.05 * k), target=1.05)
    assert r["reached_s"] is not None and r["branch"] == "cold"
    assert "below the warm branch" in r["fallback"]
    assert r["iters"]["W"] < 400 < r["iters"]["C"]


def test_warm_start_worse_than_uniform_is_dropped_at_once(monkeypatch):
    r, _ = _run(monkeypatch, lambda k: 9.0, lambda k: 1.0 + 5.0 / (1 + k), iters=200)
    assert r["branch"] == "cold" and "not below the loss at the uniform start" in r["fallback"]
    assert r["iters"]["W"] == 5


def test_non_finite_warm_loss_falls_back(monkeypatch):
    r, _ = _run(monkeypatch, lambda k: float("nan") if k > 7 else 0.5, lambda k: 1.0 + 5.0 / (1 + k), iters=300)
    assert r["branch"] == "cold" and "non-finite" in r["fallback"]


def test_both_settle_and_the_better_branch_wins(monkeypatch):
    r, _ = _run(monkeypatch, lambda k: 1.0 + 1.0 / (1 + k), lambda k: 1.2 + 1.0 / (1 + k), iters=100000)
    assert r["branch"] == "warm" and r["iters"]["W"] + r["iters"]["C"] < 100000
