"""Degenerate meshes of the method: meshes without faces.

A 1 x 1 x 1 structured box and a face-based mesh of isolated cells have no
faces, so R(theta) = 0 (eq. (M): an empty sum), every step leaves theta
unchanged up to the rounding of the RK blend, and no velocity element exists
to read (u_f is an empty buffer, passed as a null pointer)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", ["superbee", "vanleer", "smart"])
def test_single_cell_box(fl, lim, dtype, rk):
    mesh = W.structured_mesh(1, 1, 1, 0.1, 0.2, 0.3)
    assert mesh.n_faces == 0
    m = fl.Mesh.structured(1, 1, 1, *mesh.h)
    th = np.array([0.7])
    u = torch.empty(0, dtype=dtype, device="cuda")
    ref = oracle.step(mesh, lim, rk, 0.05, 4, np.zeros(0), th)
    g = torch.tensor(th, dtype=dtype, device="cuda")
    fl.step_rk(m, lim, g, u, 0.05, 4, rk_order=rk)
    assert _rel(g.cpu().double().numpy(), ref) <= TOL[dtype]
    R, thf = fl.conv_limited_apply(m, lim, g, u, want_theta_f=True)
    assert R.cpu().tolist() == [0.0] and thf.numel() == 0
    m.close()


@pytest.mark.parametrize("renumber", [True, False])
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_face_based_mesh_without_faces(fl, dtype, rk, renumber):
    n = 5
    mesh = W.Mesh(n, np.zeros((0, 2), np.int32), np.zeros((0, 3)), np.zeros(0),
                  np.linspace(0.5, 1.5, n))
    m = fl.Mesh.from_faces(n, mesh.face_cells, mesh.normals, mesh.areas, mesh.volumes,
                           renumber=renumber)
    cp, fp, flip = m.permutation()
    assert len(fp) == 0 and sorted(cp.tolist()) == list(range(n))
    th = np.linspace(-1.0, 2.0, n)
    ref = oracle.step(mesh, "superbee", rk, 0.05, 3, np.zeros(0), th)
    x = np.empty_like(th)
    x[cp] = th
    g = torch.tensor(x, dtype=dtype, device="cuda")
    u = torch.empty(0, dtype=dtype, device="cuda")
    fl.step_rk(m, "superbee", g, u, 0.05, 3, rk_order=rk)
    assert _rel(g.cpu().double().numpy()[cp], ref) <= TOL[dtype]
    R = fl.conv_limited_apply(m, "superbee", g, u)
    assert R.cpu().tolist() == [0.0] * n
    m.close()
