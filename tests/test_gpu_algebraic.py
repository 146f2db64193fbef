"""The algebraic formulation on the GPU (Algorithm 1 as 4 SpMV + 4 pointwise
kernels, Algorithm 5's update as U, M and an axpy) against the oracle, and
its matrices against the paper's storage count (Section 3: 2 |F| non-zeros
for E and Pi, 2k |F| for S and T on a k-regular mesh)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _alg(fl, mesh):
    return fl.Algebraic(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas, mesh.volumes)


def _inputs(mesh, seed):
    rng = np.random.default_rng(seed)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, seed + 1)
    return th, u


@pytest.mark.parametrize("shape,k", [((6, 5, 4), 6), ((7, 4, 1), 4), ((9, 1, 1), 2)])
def test_storage_matches_the_paper_count(fl, shape, k):
    mesh = W.structured_mesh(*shape, 0.1, 0.2, 0.3)
    a = _alg(fl, mesh)
    nnz, width, nbytes = a.info()
    F, C = mesh.n_faces, mesh.n_cells
    assert nnz[0] == 2 * F and width[0] == 2            # E
    assert nnz[3] == 2 * F and width[3] == 2            # Pi
    assert nnz[1] == 2 * k * F and width[1] == 2 * k    # T
    assert nnz[2] == 2 * k * F and width[2] == 2 * k    # -S
    assert nnz[4] == k * C and width[4] == k            # M
    assert nbytes == 12 * (2 * F + 2 * F + 2 * (2 * k * F) + k * C)
    a.close()


@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("case", ["structured", "permuted", "line", "plane"])
def test_face_values_match_oracle(fl, case, lim):
    if case == "structured":
        mesh = W.structured_mesh(13, 9, 6, 0.07, 0.11, 0.13)
    elif case == "permuted":
        mesh = W.permuted_mesh(W.structured_mesh(8, 7, 5, 0.1, 0.12, 0.15), seed=3)[0]
    elif case == "line":
        mesh = W.structured_mesh(33, 1, 1, 0.03, 1.0, 1.0)
    else:
        mesh = W.structured_mesh(11, 10, 1, 0.09, 0.1, 1.0)
    th, u = _inputs(mesh, 4)
    a = _alg(fl, mesh)
    got = a.face_values(lim, torch.tensor(th, device="cuda"), torch.tensor(u, device="cuda"))
    ref = oracle.face_values(mesh, lim, th, u)["theta_f"]
    assert _rel(got.cpu().numpy(), ref) <= 1e-12
    a.close()


def test_flat_field_and_zero_velocity_keep_the_upwind_value(fl):
    # d_u == 0 and u_f = 0 / -0 everywhere: theta_f = theta_C exactly
    mesh = W.structured_mesh(8, 6, 5, 0.1, 0.1, 0.1)
    th = np.full(mesh.n_cells, 0.375)
    u = np.zeros(mesh.n_faces)
    u[::2] = -0.0
    a = _alg(fl, mesh)
    got = a.face_values("superbee", torch.tensor(th, device="cuda"), torch.tensor(u, device="cuda"))
    assert np.all(got.cpu().numpy() == 0.375)
    a.close()


@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_euler_steps_match_oracle_and_fused_path(fl, lim):
    shape = (20, 12, 9)
    mesh = W.structured_mesh(*shape, 0.05, 0.08, 0.1)
    th, u = _inputs(mesh, 7)
    dt = 0.3 * 0.05 / np.max(np.abs(u)) / 3
    a = _alg(fl, mesh)
    ud = torch.tensor(u, device="cuda")
    cur = th
    for _ in range(3):  # per step from the oracle's state
        ref = oracle.step(mesh, lim, 1, dt, 1, u, cur)
        g = torch.tensor(cur, device="cuda")
        a.step_euler(lim, g, ud, dt, 1)
        assert _rel(g.cpu().numpy(), ref) <= 1e-12
        cur = ref
    # several steps in one call, and the fused path on the same mesh
    ga = torch.tensor(th, device="cuda")
    a.step_euler(lim, ga, ud, dt, 5)
    ref5 = oracle.step(mesh, lim, 1, dt, 5, u, th)
    assert _rel(ga.cpu().numpy(), ref5) <= 1e-11
    m = fl.Mesh.structured(*shape, 0.05, 0.08, 0.1)
    gf = torch.tensor(th, device="cuda")
    fl.step_rk(m, lim, gf, ud, dt, 5, rk_order=1)
    assert _rel(ga.cpu().numpy(), gf.cpu().numpy()) <= 1e-11
    m.close()
    a.close()


def test_rejects_bad_meshes(fl):
    mesh = W.structured_mesh(4, 4, 4, 0.1, 0.1, 0.1)
    fc = mesh.face_cells.copy()
    fc[3, 1] = fc[3, 0]
    with pytest.raises(fl.FLError):
        fl.fl_alg_create(mesh.n_cells, fc, mesh.normals, mesh.areas, mesh.volumes)
    vol = mesh.volumes.copy()
    vol[5] = 0.0
    with pytest.raises(fl.FLError):
        fl.fl_alg_create(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas, vol)
    fc = mesh.face_cells.copy()
    fc[0, 0] = mesh.n_cells
    with pytest.raises(fl.FLError):
        fl.fl_alg_create(mesh.n_cells, fc, mesh.normals, mesh.areas, mesh.volumes)
