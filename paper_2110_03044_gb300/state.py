"""Checkpoint and resume of a rollout: the state of the method is the cell
field theta and the number of steps taken (the velocity, the mesh and the
step size are inputs the caller keeps), so a checkpoint is those two plus a
description to check against on resume.

``save_state`` writes theta (copied to the host) with the step counter and
the caller's metadata into one ``.npz`` file, written to a temporary name
and renamed into place so that a crash mid-write leaves the previous file.
``load_state`` reads it back, checks the metadata the caller expects, and
returns theta on the requested device with the step counter.  A decomposed
run saves each rank's owned cells under a per-rank name (``rank_path``).
"""
from __future__ import annotations

import json
import os

import numpy as np


def rank_path(path: str, rank: int) -> str:
    """The file of rank ``rank`` of a decomposed run's checkpoint ``path``."""
    root, ext = os.path.splitext(path)
    return "%s.rank%d%s" % (root, rank, ext or ".npz")


def save_state(path: str, theta, step: int, **meta) -> None:
    """Write theta (any torch tensor or array, flattened), the step counter
    and ``meta`` (JSON-serialisable values) to ``path`` atomically."""
    try:
        import torch
        if isinstance(theta, torch.Tensor):
            theta = theta.detach().cpu().numpy()
    except ImportError:
        pass
    arr = np.ascontiguousarray(np.asarray(theta).reshape(-1))
    if int(step) < 0:
        raise ValueError("step must be >= 0")
    info = dict(meta, step=int(step), dtype=str(arr.dtype), n=int(arr.shape[0]))
    tmp = path + ".tmp"
    with open(tmp, "wb") as fh:
        np.savez(fh, theta=arr, info=np.frombuffer(json.dumps(info, sort_keys=True).encode(),
                                                  dtype=np.uint8))
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)


def load_state(path: str, device=None, **expect):
    """(theta, step, meta) from ``path``; theta is a torch tensor on
    ``device`` (the host by default).  Every keyword in ``expect`` must equal
    the saved metadata (a checkpoint of another mesh, dtype or limiter is
    refused with ValueError)."""
    import torch
    with np.load(path) as z:
        arr = z["theta"]
        info = json.loads(bytes(z["info"]).decode())
    for k, v in expect.items():
        if info.get(k) != v:
            raise ValueError("checkpoint %s has %s=%r, expected %r" % (path, k, info.get(k), v))
    if arr.shape[0] != info["n"] or str(arr.dtype) != info["dtype"]:
        raise ValueError("checkpoint %s is damaged" % path)
    t = torch.from_numpy(arr.copy())
    if device is not None:
        t = t.to(device)
    return t, int(info["step"]), info
