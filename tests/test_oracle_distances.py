"""Pins of the oracle's distance weights on non-uniform meshes (Algorithm 3:
each upstream term divided by its face distance d_j and the ratio taken
against (theta_D - theta_C) / d_f; Algorithm 2's (d_i / d_U) in 1D).

What fixes them, apart from the oracle itself:
  * a linear profile on a stretched line has the same gradient on every
    face, so the weighted r is 1 and every limiter (Psi(1) = 1) gives the
    central face value; unweighted r is d_U / d_f there;
  * Algorithm 2 evaluated directly on a stretched periodic line;
  * uniform distances reproduce the unweighted oracle bit for bit (a power of
    two as the distance makes the weights exact), and scaling every
    distance by the same factor changes nothing;
  * a stretched 3D box with flow along x equals the stretched 1D line on
    every x line (Sweby's collapse, Section 3.1);
  * conservation, and the tangent-linear model and adjoint of the weighted
    operator against central differences and the dot-product identity."""
import numpy as np
import pytest

import oracle
import workloads as W

LIMS = ["minmod", "vanleer", "superbee", "smart"]


def _line(n=32, ratio=3.0, seed=1):
    w = W.stretched_widths(n, 1.0, ratio, seed)
    return W.stretched_mesh(w), w


def _box(seed=3):
    wx = W.stretched_widths(9, 1.0, 2.5, seed)
    wy = W.stretched_widths(7, 0.8, 2.0, seed + 1)
    wz = W.stretched_widths(5, 0.6, 3.0, seed + 2)
    return W.stretched_mesh(wx, wy, wz), (wx, wy, wz)


@pytest.mark.parametrize("direction", [1.0, -1.0])
@pytest.mark.parametrize("lim", LIMS)
def test_linear_profile_gives_central_face_values(lim, direction):
    mesh, w = _line()
    n = len(w)
    xc = np.cumsum(w) - 0.5 * w
    th = 2.0 + 0.7 * xc
    u = np.full(mesh.n_faces, 0.3 * direction)
    fv = oracle.face_values(mesh, lim, th, u)
    # faces 1 .. n-3 and their upstream faces avoid the periodic seam
    f = np.arange(1, n - 2)
    r = fv["dU"][f] / fv["du"][f]
    assert np.max(np.abs(r - 1.0)) <= 1e-13
    mean = 0.5 * (th[f] + th[f + 1])
    assert np.max(np.abs(fv["theta_f"][f] - mean)) <= 1e-14 * np.max(np.abs(th))
    # the same mesh without its distances is not central: the weights matter
    mesh.distances = None
    fv0 = oracle.face_values(mesh, lim, th, u)
    assert np.max(np.abs(fv0["dU"][f] / fv0["du"][f] - 1.0)) > 0.05


def _algorithm2(d, th, u, lim):
    """Algorithm 2 on a periodic line: face i between cells i and i+1."""
    n = len(th)
    out = np.empty(n)
    for i in range(n):
        if u[i] > 0:
            C, U, D = i, (i - 1) % n, (i + 1) % n
            dU = d[(i - 1) % n]
        else:
            C, U, D = (i + 1) % n, (i + 2) % n, i
            dU = d[(i + 1) % n]
        if th[D] == th[C]:
            out[i] = th[C]
            continue
        r = (d[i] / dU) * (th[C] - th[U]) / (th[D] - th[C])
        psi = oracle.psi(lim, np.array([r]))[0]
        out[i] = 0.5 * (th[C] + th[D]) + 0.5 * (psi - 1.0) * (th[D] - th[C])
    return out


@pytest.mark.parametrize("lim", LIMS + ["upwind", "central"])
def test_algorithm2_on_a_stretched_line(lim):
    mesh, w = _line(n=40, ratio=4.0, seed=5)
    rng = np.random.default_rng(6)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    th[5:9] = 0.25  # flat run: d_u == 0 faces
    u = W.mixed_sign_velocity(mesh.n_faces, 7)
    ref = _algorithm2(mesh.distances, th, u, lim)
    got = oracle.face_values(mesh, lim, th, u)["theta_f"]
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(th))


@pytest.mark.parametrize("name", ["box", "tet"])
def test_uniform_and_scaled_distances(name):
    if name == "box":
        mesh = W.structured_mesh(6, 5, 4, 0.5, 0.5, 0.5)
    else:
        mesh = W.tet_mesh(3)
    rng = np.random.default_rng(8)
    th = rng.uniform(-1, 1, mesh.n_cells)
    u = W.mixed_sign_velocity(mesh.n_faces, 9)
    ref_fv = oracle.face_values(mesh, "superbee", th, u)
    ref_step = oracle.step(mesh, "vanleer", 3, 0.01, 2, u, th)
    # a power of two as the common distance: the weights are exact
    mesh.distances = np.full(mesh.n_faces, 0.5)
    fv = oracle.face_values(mesh, "superbee", th, u)
    np.testing.assert_array_equal(fv["theta_f"], ref_fv["theta_f"])
    np.testing.assert_array_equal(fv["dU"], ref_fv["dU"])
    np.testing.assert_array_equal(oracle.step(mesh, "vanleer", 3, 0.01, 2, u, th), ref_step)
    # any common scale: only ratios enter
    d = rng.uniform(0.5, 2.0, mesh.n_faces)
    mesh.distances = d
    a = oracle.step(mesh, "smart", 3, 0.01, 2, u, th)
    mesh.distances = 4.0 * d
    np.testing.assert_array_equal(oracle.step(mesh, "smart", 3, 0.01, 2, u, th), a)
    mesh.distances = 3.0 * d
    assert np.max(np.abs(oracle.step(mesh, "smart", 3, 0.01, 2, u, th) - a)) <= 1e-14


@pytest.mark.parametrize("lim", LIMS)
def test_stretched_box_collapses_to_lines(lim):
    mesh, (wx, wy, wz) = _box()
    nx, ny, nz = len(wx), len(wy), len(wz)
    C = mesh.n_cells
    rng = np.random.default_rng(10)
    th = rng.uniform(0, 1, C)
    ux = rng.uniform(0.2, 1.0, C) * np.where(rng.random(C) < 0.5, 1.0, -1.0)
    u = np.concatenate([ux, np.zeros(C), np.zeros(C)])
    dt = 0.2 * np.min(wx)
    got = oracle.step(mesh, lim, 3, dt, 2, u, th)
    line = W.stretched_mesh(wx)
    for k in range(nz):
        for j in range(ny):
            sl = slice(nx * (j + ny * k), nx * (j + ny * k) + nx)
            ref = oracle.step(line, lim, 3, dt, 2, ux[sl], th[sl])
            assert np.max(np.abs(got[sl] - ref)) <= 1e-14


@pytest.mark.parametrize("lim", LIMS)
def test_conservation_on_a_stretched_box(lim):
    mesh, _ = _box(seed=11)
    rng = np.random.default_rng(12)
    th = rng.uniform(0, 1, mesh.n_cells)
    u = 0.5 * W.mixed_sign_velocity(mesh.n_faces, 13)
    dt = 0.05 * np.min(mesh.volumes / mesh.volumes.max()) * 0.1
    m0 = np.sum(mesh.volumes * th)
    th1 = oracle.step(mesh, lim, 3, dt, 40, u, th)
    assert abs(np.sum(mesh.volumes * th1) - m0) <= 1e-13 * abs(m0)


@pytest.mark.parametrize("lim", ["superbee", "smart", "vanleer"])
def test_weighted_tlm_and_adjoint(lim):
    mesh, _ = _box(seed=14)
    om = oracle.OracleMesh(mesh)
    rng = np.random.default_rng(15)
    th = rng.uniform(0, 1, mesh.n_cells)
    u = W.mixed_sign_velocity(mesh.n_faces, 16)
    dt = 0.002
    v = rng.normal(size=mesh.n_cells)
    _, dth = oracle.step_tlm(om, lim, 3, dt, 2, u, th, v)
    eps = 1e-6
    fd = (oracle.step(om, lim, 3, dt, 2, u, th + eps * v)
          - oracle.step(om, lim, 3, dt, 2, u, th - eps * v)) / (2 * eps)
    tol = 1e-6 if lim == "vanleer" else 1e-7
    assert np.linalg.norm(fd - dth) / np.linalg.norm(dth) < tol
    # <J v, w> = <v, J^T w> for the operator R
    w = rng.normal(size=mesh.n_cells)
    _, d = oracle.step_tlm(om, lim, 1, 1.0, 1, u, th, v)
    Jv = d - v
    JTw = oracle.rhs_adjoint(om, lim, th, u, w)
    assert abs(np.dot(Jv, w) - np.dot(v, JTw)) <= 1e-13 * np.linalg.norm(Jv) * np.linalg.norm(w)
