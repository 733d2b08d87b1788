"""Checkpoint files (host side): round trip, and rejection of truncated,
altered or foreign files -- faults injected on the host, no GPU."""
import os

import numpy as np
import pytest

from paper_2409_10876_gb300 import checkpoint, inputs


def _arrays():
    rng = np.random.default_rng(0)
    return {"sos": rng.standard_normal((16, 16)).astype(np.float32),
            "adam_m": rng.standard_normal((16, 16)).astype(np.float32),
            "adam_v": rng.random((16, 16)).astype(np.float32),
            "counter": np.array([7, 0], np.int32)}


def test_round_trip(tmp_path):
    p = str(tmp_path / "ck.npz")
    h = checkpoint.config_hash(inputs.config_small(), lr=1.0)
    checkpoint.save(p, _arrays(), {"iteration": 7, "seed": 3, "config_hash": h})
    arrays, meta = checkpoint.load(p, h)
    for k, v in _arrays().items():
        assert np.array_equal(arrays[k], v) and arrays[k].dtype == v.dtype
    assert meta["iteration"] == 7 and meta["seed"] == 3
    assert not [f for f in os.listdir(tmp_path) if ".tmp." in f]      # written under a temporary name, renamed


def test_config_hash_distinguishes_settings():
    cfg = inputs.config_small()
    assert checkpoint.config_hash(cfg, lr=1.0) != checkpoint.config_hash(cfg, lr=0.5)
    assert checkpoint.config_hash(cfg) != checkpoint.config_hash(cfg.replace(tv_lambda=1.0))
    assert checkpoint.config_hash(cfg, lr=1.0) == checkpoint.config_hash(cfg, lr=1.0)


def test_rejects_foreign_truncated_and_altered_files(tmp_path):
    p = str(tmp_path / "ck.npz")
    checkpoint.save(p, _arrays(), {"iteration": 1, "config_hash": "abc"})
    with pytest.raises(checkpoint.CheckpointError, match="configuration"):
        checkpoint.load(p, "other")
    raw = open(p, "rb").read()
    t = str(tmp_path / "trunc.npz")
    open(t, "wb").write(raw[: len(raw) // 2])
    with pytest.raises(checkpoint.CheckpointError):
        checkpoint.load(t)
    # flip one byte of an array: the archive still reads, the checksum does not match
    a = _arrays()
    q = str(tmp_path / "alt.npz")
    checkpoint.save(q, a, {"iteration": 1})
    arrays, meta = checkpoint.load(q)
    a["sos"][3, 3] += 1.0
    np.savez(q, __meta__=np.frombuffer(__import__("json").dumps(meta).encode(), np.uint8), **a)
    with pytest.raises(checkpoint.CheckpointError, match="checksum"):
        checkpoint.load(q)
    with pytest.raises(checkpoint.CheckpointError):
        checkpoint.load(str(tmp_path / "missing.npz"))
