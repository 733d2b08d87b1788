"""Writes tests/golden/tiny_case.json: FP64 oracle outputs on a tiny seeded
case (a regression guard for the oracle itself).  Calls only oracle/ and the
seeded input generators; run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pact_oracle as O          # noqa: E402
from paper_2409_10876_gb300 import inputs    # noqa: E402


def main():
    cfg = inputs.config_tiny(p=16, m=4)
    g = O.geom(cfg)
    case = inputs.make_case(cfg, 21)
    Y, X, w_true = O.make_measurement(g, case)
    L, Ld, w, gs = O.objective(g, case["sos_init"], Y, case["centres"], case["d"], cfg.eps, cfg.tv_lambda)
    Lt, Ldt, _, _ = O.objective(g, case["sos_true"], Y, case["centres"], case["d"], cfg.eps, cfg.tv_lambda, False)
    out = {
        "what": "oracle outputs, config_tiny(p=16, m=4), make_case seed 21 (Eq. 3-7)",
        "loss_init": float(L),
        "loss_true": float(Lt),
        "w_true_sample": [float(w_true[i, n]) for i, n in [(0, 0), (1, 17), (2, 40), (3, 63)]],
        "grad_init_l2": float(np.linalg.norm(gs.numpy())),
        "grad_init_sample": [float(gs[p, q]) for p, q in [(8, 8), (5, 10), (11, 6)]],
        "Y_abs_sum": float(Y.abs().sum()),
    }
    with open(os.path.join(HERE, "tiny_case.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
