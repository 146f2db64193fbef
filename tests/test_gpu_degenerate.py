"""Degenerate cases of the method: meshes without faces, and zero or negative
time steps.

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


# dt = 0 and dt < 0: the step is theta + dt R(theta) with the upwind side
# still taken from u_f (the FP64 path pre-scales w = dt (A/V) u_f only when
# dt > 0, since a negative factor would flip every upwind test)
@pytest.mark.parametrize("dt_scale", [0.0, -1.0])
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("case", ["f64 tile", "f32 tma", "f32 register tile", "f64 face-based"])
def test_zero_and_negative_time_step(fl, case, rk, dt_scale):
    dtype = torch.float64 if case.startswith("f64") else torch.float32
    shape = (128, 8, 5) if case == "f32 tma" else (37, 21, 13)
    h = (0.7 / shape[0], 0.9 / shape[1], 1.1 / shape[2])
    mesh = W.structured_mesh(*shape, *h)
    rng = np.random.default_rng(17)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 18)
    if dtype == torch.float32:
        th = th.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    dt = dt_scale * 0.1 * min(h) / np.max(np.abs(u))
    ref = oracle.step(mesh, "superbee", rk, dt, 1, u, th)
    if case == "f64 face-based":
        pm, cp, fp, flip = W.permuted_mesh(mesh, seed=3)
        m = fl.Mesh.from_faces(pm.n_cells, pm.face_cells, pm.normals, pm.areas, pm.volumes,
                               renumber=True)
        icp, ifp, _ = m.permutation()
        # user order of the permuted mesh, then the library's internal order
        th_u = np.empty_like(th)
        th_u[cp] = th
        u_u = np.empty_like(u)
        u_u[fp] = np.where(flip, -u, u)
        x = np.empty_like(th_u)
        x[icp] = th_u
        uu = np.empty_like(u_u)
        uu[ifp] = u_u
        g = torch.tensor(x, dtype=dtype, device="cuda")
        fl.step_rk(m, "superbee", g, torch.tensor(uu, dtype=dtype, device="cuda"), dt, 1,
                   rk_order=rk)
        got = g.cpu().double().numpy()[icp][cp]
    else:
        m = fl.Mesh.structured(*shape, *h)
        g = torch.tensor(th, dtype=dtype, device="cuda")
        fl.step_rk(m, "superbee", g, torch.tensor(u, dtype=dtype, device="cuda"), dt, 1,
                   rk_order=rk)
        got = g.cpu().double().numpy()
    assert _rel(got, ref) <= TOL[dtype]
    m.close()
