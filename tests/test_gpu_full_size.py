"""Every cell of the full-size configurations against the oracle.

One SSP-RK3 step of each configuration, in the launch configuration the
benchmark times, compared cell by cell with the FP64 oracle run on the whole
mesh (one oracle step of 256^3 takes about half a second on the host's
cores): 1e-12 relative in FP64, 1e-5 in FP32 (the oracle then starts from the
FP32-rounded inputs).

* 256^3 Taylor-Green, every limiter: FP64 (the stage tile), FP32 (the TMA
  kernel); 250^3 in FP32 (250 is not a multiple of 4: the register tile);
* the same mesh as face-based (unstructured) storage: seeded cell and face
  permutations, half of the faces reoriented, SMART, FP64;
* all 64 boxes of the batched configuration, van Leer, FP64 and FP32.

The mass of each result is summed exactly on the host (math.fsum) and must
equal the initial mass to 1e-12 (FP64) or 1e-5 (FP32)."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
LIMS = ["minmod", "vanleer", "superbee", "smart"]


def _cast(x, dtype):
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _mass(x, vol):
    return math.fsum((np.asarray(x, np.float64) * vol).tolist())


@pytest.fixture(scope="module")
def tg256():
    wl = W.config_taylor_green(n=256, seed=1, nsteps=1)
    return wl, oracle.OracleMesh(wl.mesh)


@pytest.fixture(scope="module")
def tg250():
    wl = W.config_taylor_green(n=250, seed=1, nsteps=1)
    return wl, oracle.OracleMesh(wl.mesh)


def _structured_case(fl, wl, om, lim, dtype, n):
    th0, u = _cast(wl.theta0, dtype), _cast(wl.u, dtype)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    g = torch.tensor(th0, dtype=dtype, device="cuda")
    ws, nb = fl.workspace_for(m, dtype, 3)
    fl.fl_step_rk(m.handle, lim, dtype, 3, wl.dt, 1, g, torch.tensor(u, dtype=dtype,
                                                                     device="cuda"), ws, nb)
    got = g.cpu().double().numpy()
    m.close()
    ref = oracle.step(om, lim, 3, wl.dt, 1, u, th0)
    assert _rel(got, ref) <= TOL[dtype]
    vol = wl.mesh.volumes
    m0 = _mass(th0, vol)
    assert abs(_mass(got, vol) - m0) <= (1e-12 if dtype == torch.float64 else 1e-5) * abs(m0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
def test_taylor_green_256_every_cell(fl, tg256, lim, dtype):
    wl, om = tg256
    _structured_case(fl, wl, om, lim, dtype, 256)


@pytest.mark.parametrize("lim", LIMS)
def test_taylor_green_250_register_tile_every_cell(fl, tg250, lim):
    wl, om = tg250
    _structured_case(fl, wl, om, lim, torch.float32, 250)


def test_unstructured_storage_256_every_cell(fl, tg256):
    wl, _ = tg256
    pm, cp, fp, flip = W.permuted_mesh(wl.mesh, seed=2)
    up = W.permute_face_field(wl.u, fp, flip)
    thp = W.permute_cell_field(wl.theta0, cp)
    m = fl.Mesh.from_faces(pm.n_cells, pm.face_cells, pm.normals, pm.areas, pm.volumes,
                           renumber=True)
    f64 = torch.float64
    g = m.to_internal(torch.tensor(thp, device="cuda"), "cell")
    ui = m.to_internal(torch.tensor(up, device="cuda"), "face")
    nb = fl.fl_workspace_size(m.handle, f64, 3)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_step_rk(m.handle, "smart", f64, 3, wl.dt, 1, g, ui, ws, nb)
    got = m.to_user(g, "cell").cpu().numpy()
    m.close()
    del g, ui, ws
    ref = oracle.step(pm, "smart", 3, wl.dt, 1, up, thp)
    assert _rel(got, ref) <= 1e-12
    m0 = _mass(thp, pm.volumes)
    assert abs(_mass(got, pm.volumes) - m0) <= 1e-12 * abs(m0)


@pytest.fixture(scope="module")
def boxes64():
    dims = W.batched_box_dims()
    return dims, [W.random_box(d, 1000 + i) for i, d in enumerate(dims)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_64_boxes_every_cell(fl, boxes64, dtype):
    dims, boxes = boxes64
    meshes = [fl.Mesh.structured(*d, *b[0].h) for d, b in zip(dims, boxes)]
    batch = fl.fl_batch_create([m.handle for m in meshes])
    th0 = [_cast(b[1], dtype) for b in boxes]
    us = [_cast(b[2], dtype) for b in boxes]
    th = [torch.tensor(t, dtype=dtype, device="cuda") for t in th0]
    ud = [torch.tensor(u, dtype=dtype, device="cuda") for u in us]
    dts = [b[3] for b in boxes]
    nb = fl.fl_batch_workspace_size(batch, dtype, 3)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_batch_step_rk(batch, "vanleer", dtype, 3, dts, 1, th, ud, ws, nb)
    got = [t.cpu().double().numpy() for t in th]
    fl.fl_batch_destroy(batch)
    for m in meshes:
        m.close()
    for (mesh, _, _, dt), t0, u, g in zip(boxes, th0, us, got):
        ref = oracle.step(mesh, "vanleer", 3, dt, 1, u, t0)
        assert _rel(g, ref) <= TOL[dtype]
        m0 = _mass(t0, mesh.volumes)
        assert abs(_mass(g, mesh.volumes) - m0) <= \
            (1e-12 if dtype == torch.float64 else 1e-5) * max(abs(m0), _mass(np.abs(t0),
                                                                             mesh.volumes))
