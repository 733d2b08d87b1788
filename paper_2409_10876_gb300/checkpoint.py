"""Checkpoint and resume of a recovery run (no counterpart in the paper).

A checkpoint holds what a recovery needs to continue exactly where it stopped:
the SOS parameters (pixel grid or neural-field weights), the Adam moments and
step counter, the iteration count, the seed and a hash of the configuration
it was made for.  Files are NumPy .npz archives written to a temporary name
and renamed into place (a crash never leaves a half-written checkpoint under
the final name), with a SHA-256 of the arrays in the metadata so that a
truncated or altered file is rejected instead of resuming from garbage.
"""
from __future__ import annotations

import hashlib
import io
import json
import os
import zipfile

import numpy as np

FORMAT = 1


class CheckpointError(RuntimeError):
    pass


def config_hash(cfg, **extra) -> str:
    """Hash of every field of a workload configuration plus the keyword
    arguments (learning rate, TV weight, ...)."""
    return hashlib.sha1(repr((cfg, sorted(extra.items()))).encode()).hexdigest()[:16]


def _digest(arrays: dict) -> str:
    h = hashlib.sha256()
    for k in sorted(arrays):
        a = np.ascontiguousarray(arrays[k])
        h.update(k.encode())
        h.update(str(a.dtype).encode())
        h.update(repr(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


def save(path: str, arrays: dict, meta: dict) -> None:
    """Writes `arrays` (name -> ndarray) and `meta` (JSON-serialisable) to
    `path` atomically."""
    arrays = {k: np.asarray(v) for k, v in arrays.items()}
    if "__meta__" in arrays:
        raise CheckpointError("'__meta__' is reserved")
    m = dict(meta, format=FORMAT, sha256=_digest(arrays))
    buf = io.BytesIO()
    np.savez(buf, __meta__=np.frombuffer(json.dumps(m).encode(), np.uint8), **arrays)
    tmp = f"{path}.tmp.{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(buf.getvalue())
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path: str, expect_hash: str = None):
    """Reads a checkpoint; returns (arrays, meta).  Raises CheckpointError for
    a missing, truncated or altered file, an unknown format, or a
    configuration hash other than `expect_hash` (when given)."""
    try:
        with np.load(path, allow_pickle=False) as z:
            arrays = {k: z[k] for k in z.files}
    except (OSError, ValueError, EOFError, zipfile.BadZipFile, KeyError) as e:
        raise CheckpointError(f"cannot read checkpoint {path}: {e}") from e
    if "__meta__" not in arrays:
        raise CheckpointError(f"{path}: no metadata")
    try:
        meta = json.loads(arrays.pop("__meta__").tobytes().decode())
    except ValueError as e:
        raise CheckpointError(f"{path}: bad metadata: {e}") from e
    if meta.get("format") != FORMAT:
        raise CheckpointError(f"{path}: format {meta.get('format')} (expected {FORMAT})")
    if meta.get("sha256") != _digest(arrays):
        raise CheckpointError(f"{path}: contents do not match their checksum")
    if expect_hash is not None and meta.get("config_hash") != expect_hash:
        raise CheckpointError(f"{path}: made for configuration {meta.get('config_hash')}, not {expect_hash}")
    return arrays, meta
