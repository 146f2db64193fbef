"""The batched form: many periodic boxes of uneven sizes advanced by one
persistent launch per stage (graph-replayed).  In FP64 every box must match
the single-mesh path bit for bit (same tile code, same inputs); in FP32 the
single-mesh path runs another tile, so within the tolerance; and every box
matches the oracle within the per-step tolerance."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
SHAPES = [(33, 17, 9), (40, 40, 12), (8, 8, 8), (64, 9, 20), (31, 1, 1), (21, 14, 1), (5, 12, 6)]


def _boxes(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i, sh in enumerate(SHAPES):
        h = tuple(0.5 / d for d in sh)
        mesh = W.structured_mesh(*sh, *h)
        th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
        u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 10 + i)
        dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
        out.append((mesh, th, u, dt))
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rk,nsteps", [(3, 2), (1, 3), (1, 4)])
@pytest.mark.parametrize("lim", ["vanleer", "superbee", "smart"])
def test_batch_matches_single_mesh_path(fl, lim, rk, nsteps, dtype):
    boxes = _boxes()
    meshes = [fl.Mesh.structured(*b[0].dims, *b[0].h) for b in boxes]
    batch = fl.fl_batch_create([m.handle for m in meshes])
    th = [torch.tensor(b[1], dtype=dtype, device="cuda") for b in boxes]
    us = [torch.tensor(b[2], dtype=dtype, device="cuda") for b in boxes]
    dts = [b[3] for b in boxes]
    ref = [t.clone() for t in th]
    for m, t, u, dt in zip(meshes, ref, us, dts):
        fl.step_rk(m, lim, t, u, dt, nsteps, rk_order=rk)
    nb = fl.fl_batch_workspace_size(batch, dtype, rk)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_batch_step_rk(batch, lim, dtype, rk, dts, nsteps, th, us, ws, nb)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(th, ref)):
        if (boxes[i][0].dims[1] == 1 and boxes[i][0].dims[2] == 1) or dtype == torch.float32:
            # 1D boxes run the resident line kernel on the single-mesh path,
            # and FP32 single meshes the register tile (the batch keeps the
            # shared-memory tile): the same method, other rounding orders
            assert float((a - b).abs().max() / b.abs().max()) <= TOL[dtype] * nsteps
        else:
            assert torch.equal(a, b), i
    # and per step against the oracle (first box set, one step)
    th1 = [torch.tensor(b[1], dtype=dtype, device="cuda") for b in boxes]
    fl.fl_batch_step_rk(batch, lim, dtype, rk, dts, 1, th1, us, ws, nb)
    for (mesh, t0, u, dt), g in zip(boxes, th1):
        t0c = t0.astype(np.float32).astype(np.float64) if dtype == torch.float32 else t0
        uc = u.astype(np.float32).astype(np.float64) if dtype == torch.float32 else u
        r = oracle.step(mesh, lim, rk, dt, 1, uc, t0c)
        got = g.cpu().double().numpy()
        assert np.max(np.abs(got - r)) / np.max(np.abs(r)) <= TOL[dtype]
    fl.fl_batch_destroy(batch)
    for m in meshes:
        m.close()


def test_batched_config_equals_single_mesh_path(fl):
    """64 boxes with seeded sizes in [32, 128]^3 (about 34M cells): one batched
    FP64 step equals 64 single-mesh steps bit for bit (the same tile code on
    the same inputs).  Every cell of every box is checked against the oracle
    in test_gpu_full_size.py."""
    dims = W.batched_box_dims()
    boxes = [W.random_box(d, 1000 + i) for i, d in enumerate(dims)]
    meshes = [fl.Mesh.structured(*d, *b[0].h) for d, b in zip(dims, boxes)]
    batch = fl.fl_batch_create([m.handle for m in meshes])
    th = [torch.tensor(b[1], device="cuda") for b in boxes]
    us = [torch.tensor(b[2], device="cuda") for b in boxes]
    dts = [b[3] for b in boxes]
    ref = [t.clone() for t in th]
    for m, t, u, dt in zip(meshes, ref, us, dts):
        fl.step_rk(m, "vanleer", t, u, dt, 1, rk_order=3)
    nb = fl.fl_batch_workspace_size(batch, torch.float64, 3)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_batch_step_rk(batch, "vanleer", torch.float64, 3, dts, 1, th, us, ws, nb)
    torch.cuda.synchronize()
    for a, b in zip(th, ref):
        assert torch.equal(a, b)
    fl.fl_batch_destroy(batch)
    for m in meshes:
        m.close()


# every work decomposition the autotuner may pick, fixed with
# fl_batch_set_tiling: (kind, cells per thread, warps, z chunk)
TILINGS32 = [(0, 1, 8, 16), (1, 1, 8, 16), (1, 2, 4, 32), (1, 4, 8, 64), (1, 4, 4, 3),
             (1, 2, 1, 7), (2, 4, 4, 16), (2, 4, 1, 7), (2, 4, 8, 3), (2, 4, 2, 64)]


@pytest.mark.parametrize("tiling", TILINGS32)
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_batch_fp32_every_tiling_matches_oracle(fl, lim, rk, tiling):
    # the flat-run tiles and the rectangles give the bits of the single-mesh
    # FP32 kernels (the same face flux and cell-sum order), so every box is
    # checked against the oracle per step and against the single-mesh path.
    # The boxes put rows of 5 .. 64 cells, a row start at every position of
    # a four-cell group, partial last groups and one-row planes through the
    # tiles; kind 2 runs on padded copies with periodic ghost cells (Euler
    # with one step ends in the RK buffer, copied back from there), nx < 8
    # keeping the one-cell tile
    boxes = _boxes(seed=2)
    dtype = torch.float32
    meshes = [fl.Mesh.structured(*b[0].dims, *b[0].h) for b in boxes]
    batch = fl.fl_batch_create([m.handle for m in meshes])
    fl.fl_batch_set_tiling(batch, lim, dtype, rk, *tiling)
    assert fl.fl_batch_tiling(batch, lim, dtype, rk) == tiling
    th0 = [b[1].astype(np.float32).astype(np.float64) for b in boxes]
    us = [b[2].astype(np.float32).astype(np.float64) for b in boxes]
    th = [torch.tensor(t, dtype=dtype, device="cuda") for t in th0]
    ud = [torch.tensor(u, dtype=dtype, device="cuda") for u in us]
    dts = [b[3] for b in boxes]
    nb = fl.fl_batch_workspace_size(batch, dtype, rk)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_batch_step_rk(batch, lim, dtype, rk, dts, 1, th, ud, ws, nb)
    for (mesh, _, _, dt), t0, u, g in zip(boxes, th0, us, th):
        ref = oracle.step(mesh, lim, rk, dt, 1, u, t0)
        got = g.cpu().double().numpy()
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= TOL[dtype]
    # and two more steps against the single-mesh path (the same FP32 bits)
    ref = [t.clone() for t in th]
    for m, t, u, dt in zip(meshes, ref, ud, dts):
        fl.step_rk(m, lim, t, u, dt, 2, rk_order=rk)
    fl.fl_batch_step_rk(batch, lim, dtype, rk, dts, 2, th, ud, ws, nb)
    for i, (a, b) in enumerate(zip(th, ref)):
        if tiling[0] == 0 or (boxes[i][0].dims[1] == 1 and boxes[i][0].dims[2] == 1):
            # 1D lines run the resident line kernel on the single-mesh path,
            # and the rectangles the shared-memory tile
            assert float((a - b).abs().max() / b.abs().max()) <= 2 * TOL[dtype]
        else:
            assert torch.equal(a, b), (i, boxes[i][0].dims)
    fl.fl_batch_destroy(batch)
    for m in meshes:
        m.close()


def test_batch_tiling_query_and_validation(fl):
    boxes = _boxes(seed=3)[:3]
    meshes = [fl.Mesh.structured(*b[0].dims, *b[0].h) for b in boxes]
    batch = fl.fl_batch_create([m.handle for m in meshes])
    with pytest.raises(fl.FLError):  # nothing chosen yet
        fl.fl_batch_tiling(batch, "superbee", torch.float32, 3)
    th = [torch.tensor(b[1], dtype=torch.float32, device="cuda") for b in boxes]
    us = [torch.tensor(b[2], dtype=torch.float32, device="cuda") for b in boxes]
    nb = fl.fl_batch_workspace_size(batch, torch.float32, 3)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_batch_step_rk(batch, "superbee", torch.float32, 3, [b[3] for b in boxes], 1, th, us,
                        ws, nb)
    kind, cx, w, zc = fl.fl_batch_tiling(batch, "superbee", torch.float32, 3)
    assert kind in (0, 1, 2) and cx in (1, 2, 4) and 1 <= w <= 8 and 1 <= zc <= 255
    assert kind != 2 or cx == 4
    for bad in [(2, 1, 8, 16), (1, 3, 8, 16), (1, 2, 9, 16), (0, 2, 8, 16), (1, 2, 4, 0),
                (2, 4, 9, 16), (2, 4, 0, 16), (3, 4, 4, 16)]:
        with pytest.raises(fl.FLError):
            fl.fl_batch_set_tiling(batch, "superbee", torch.float32, 3, *bad)
    with pytest.raises(fl.FLError):  # flat runs are FP32 only
        fl.fl_batch_set_tiling(batch, "superbee", torch.float64, 3, 1, 2, 4, 16)
    with pytest.raises(fl.FLError):
        fl.fl_batch_set_tiling(batch, "superbee", torch.float64, 3, 2, 4, 4, 16)
    fl.fl_batch_destroy(batch)
    for m in meshes:
        m.close()
