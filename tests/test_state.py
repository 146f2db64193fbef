"""Checkpoint and resume of a rollout (paper_2110_03044_gb300.state): a
rollout split by a save and a load gives the bits of the unsplit one (the
oracle as the stepper, on the host), metadata is checked on resume, and a
damaged or foreign checkpoint is refused."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_2110_03044_gb300.state import load_state, rank_path, save_state


def test_split_rollout_resumes_bit_for_bit(tmp_path):
    mesh = W.structured_mesh(8, 6, 5, 0.1, 0.2, 0.3)
    rng = np.random.default_rng(2)
    th = rng.uniform(-1, 1, mesh.n_cells)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 3)
    dt = 0.02
    whole = oracle.step(mesh, "superbee", 3, dt, 6, u, th)
    half = oracle.step(mesh, "superbee", 3, dt, 3, u, th)
    p = str(tmp_path / "ck.npz")
    save_state(p, torch.from_numpy(half), 3, limiter="superbee", dims=[8, 6, 5], rk_order=3)
    t, step, meta = load_state(p, limiter="superbee", dims=[8, 6, 5])
    assert step == 3 and meta["rk_order"] == 3 and t.dtype == torch.float64
    rest = oracle.step(mesh, "superbee", 3, dt, 6 - step, u, t.numpy())
    assert np.array_equal(rest, whole)


def test_checkpoint_is_refused_when_it_does_not_match(tmp_path):
    p = str(tmp_path / "ck.npz")
    save_state(p, np.arange(10, dtype=np.float32), 7, limiter="smart")
    t, step, _ = load_state(p)
    assert step == 7 and t.dtype == torch.float32 and t.shape == (10,)
    with pytest.raises(ValueError):
        load_state(p, limiter="superbee")
    with pytest.raises(ValueError):
        save_state(p, np.zeros(3), -1)
    # an interrupted write leaves the previous checkpoint in place
    assert not os.path.exists(p + ".tmp")
    assert rank_path(p, 2).endswith("ck.rank2.npz")
    # a file whose array does not match its record is damaged
    import json
    bad = str(tmp_path / "bad.npz")
    info = json.dumps({"step": 1, "dtype": "float64", "n": 5}).encode()
    np.savez(bad, theta=np.zeros(4), info=np.frombuffer(info, dtype=np.uint8))
    with pytest.raises(ValueError):
        load_state(bad)
