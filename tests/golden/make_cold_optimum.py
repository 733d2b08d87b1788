"""Writes tests/golden/cold_optimum_<workload>_seed<seed>.json (and the end-point
SOS as a float32 .npy beside it): the FP64 oracle's plain pixel-grid recovery
(Sec. 3.3: Adam on the masked SOS nodes, Eq. 7 with the TV term) run from the
uniform start for the configuration's number of iterations on the held-out
problem of the warm-start benchmark.  The best loss of that run is the cold
optimum L*_cold that "within 1 % of the FP64 cold optimum" refers to.

Calls only oracle/ and the seeded input generators.  About 2 s per iteration on
8 host threads at full size (the run takes 30-40 minutes).  From the
repository root:

    python tests/golden/make_cold_optimum.py [--seed 1000] [--steps 1000] [--threads N]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import torch                                  # noqa: E402

from oracle import pact_oracle as O          # noqa: E402
from paper_2409_10876_gb300 import inputs    # noqa: E402


def config_hash(cfg, seed: int, steps: int) -> str:
    """Hash of every configuration field, the seed and the iteration count."""
    return hashlib.sha1(repr((cfg, int(seed), int(steps))).encode()).hexdigest()[:16]


def golden_path(cfg, seed: int, ext: str = "json") -> str:
    return os.path.join(HERE, f"cold_optimum_{cfg.name}_seed{seed}.{ext}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    if args.threads:
        torch.set_num_threads(args.threads)
    cfg = inputs.config_held_out()
    steps = cfg.steps if args.steps is None else args.steps
    g = O.geom(cfg)
    case = inputs.make_case(cfg, args.seed)
    Y, _, _ = O.make_measurement(g, case)
    t0 = time.time()
    sos, hist = O.recover(g, case, Y, steps, cfg.lr, cfg.eps, cfg.tv_lambda)
    el = time.time() - t0
    sos = sos.numpy()
    L_true, Ld_true, _, _ = O.objective(g, case["sos_true"], Y, case["centres"], case["d"], cfg.eps, cfg.tv_lambda,
                                        want_grad=False)
    L_end, Ld_end, _, _ = O.objective(g, sos, Y, case["centres"], case["d"], cfg.eps, cfg.tv_lambda, want_grad=False)
    mask = case["mask"].astype(bool)
    truth = case["sos_true"].astype(np.float64)
    rms = lambda s: float(np.sqrt(np.mean((s[mask] - truth[mask]) ** 2)))
    k_best = int(np.argmin(hist))
    out = {
        "what": "FP64 oracle cold recovery (Adam on the masked pixel-grid SOS from uniform v_bg; Eq. 3-7 + TV), "
                "loss at the SOS each iteration starts from",
        "workload": cfg.name, "seed": args.seed, "steps": steps, "config_hash": config_hash(cfg, args.seed, steps),
        "lr": cfg.lr, "eps": cfg.eps, "tv_lambda": cfg.tv_lambda,
        "L_star_cold": float(hist[k_best]), "iteration_of_L_star": k_best + 1,
        "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
        "loss_after_last_update": float(L_end), "data_loss_after_last_update": float(Ld_end),
        "loss_at_truth": float(L_true), "data_loss_at_truth": float(Ld_true),
        "sos_rms_mps": {"uniform": rms(case["sos_init"].astype(np.float64)), "end": rms(sos)},
        "history_every_10": [float(h) for h in hist[::10]],
        "host": {"threads": torch.get_num_threads(), "seconds": el},
    }
    with open(golden_path(cfg, args.seed), "w") as f:
        json.dump(out, f, indent=1)
    np.save(golden_path(cfg, args.seed, "npy"), sos.astype(np.float32))
    print(json.dumps({k: v for k, v in out.items() if k != "history_every_10"}))


if __name__ == "__main__":
    main()
