"""The oracle still reproduces the values stored by tests/golden/make_golden.py."""
import json
import os

import numpy as np

from oracle import pact_oracle as O
from paper_2409_10876_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tiny_case_regression():
    ref = json.load(open(os.path.join(HERE, "golden", "tiny_case.json")))
    cfg = inputs.config_tiny(p=16, m=4)
    g = O.geom(cfg)
    case = inputs.make_case(cfg, 21)
    Y, X, w_true = O.make_measurement(g, case)
    L, Ld, w, gs = O.objective(g, case["sos_init"], Y, case["centres"], case["d"], cfg.eps, cfg.tv_lambda)
    assert abs(float(L) - ref["loss_init"]) < 1e-10 * abs(ref["loss_init"])
    ws = [float(w_true[i, n]) for i, n in [(0, 0), (1, 17), (2, 40), (3, 63)]]
    assert np.allclose(ws, ref["w_true_sample"], rtol=1e-10, atol=1e-18)
    assert abs(float(np.linalg.norm(gs.numpy())) - ref["grad_init_l2"]) < 1e-9 * ref["grad_init_l2"]
