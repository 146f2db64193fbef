"""Pins of the oracle on non-hexahedral meshes (tetrahedra and triangular
prisms), where the upstream difference is the n_f . n_j-weighted sum over
all other faces of the upwind cell (eq. Delta_Upwind with the sign
correction): the stencil oracle against the dense matrix algebra of the
paper (E, S, T, Pi, M assembled from their definitions), free-stream
preservation, and conservation."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import brute

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]
MESHES = {"tet": lambda: W.tet_mesh(3), "prism": lambda: W.prism_mesh(3)}


@pytest.mark.parametrize("name", ["tet", "prism"])
@pytest.mark.parametrize("n", [3, 4])
def test_generated_meshes_are_closed_and_fill_the_box(name, n):
    m = W.tet_mesh(n) if name == "tet" else W.prism_mesh(n)
    k = 4 if name == "tet" else 5
    assert np.all(np.bincount(m.face_cells.ravel(), minlength=m.n_cells) == k)
    s = np.zeros((m.n_cells, 3))
    np.add.at(s, m.face_cells[:, 0], m.normals * m.areas[:, None])
    np.add.at(s, m.face_cells[:, 1], -m.normals * m.areas[:, None])
    assert np.abs(s).max() <= 1e-15          # sum of outward vector areas = 0
    assert m.volumes.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.allclose(np.linalg.norm(m.normals, axis=1), 1.0, atol=1e-15)
    assert np.all(m.face_cells[:, 0] != m.face_cells[:, 1])


@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("name", ["tet", "prism"])
def test_stencil_oracle_equals_matrix_algebra(name, lim):
    m = MESHES[name]()
    rng = np.random.default_rng(5)
    th = rng.uniform(-1, 1, m.n_cells) + (rng.random(m.n_cells) < 0.3)
    u = W.mixed_sign_velocity(m.n_faces, 6)
    ops = brute.operators(m)
    thf, du, dU = brute.face_values(ops, lim, th, u)
    o = oracle.face_values(m, lim, th, u)
    C, D, _ = brute.selection(ops, u)
    assert np.array_equal(o["C"], C) and np.array_equal(o["D"], D)
    assert np.max(np.abs(o["du"] - du)) <= 1e-15 * 4
    assert np.max(np.abs(o["dU"] - dU)) <= 1e-14
    assert np.max(np.abs(o["theta_f"] - thf)) <= 1e-14
    R = oracle.rhs(m, lim, th, u)
    assert np.max(np.abs(R - brute.rhs(ops, lim, th, u))) <= 1e-12 * np.max(np.abs(R))


@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("name", ["tet", "prism"])
def test_free_stream_is_preserved(name, rk):
    # a constant field in a uniform flow U . n_f: d_u = 0 on every face, the
    # face value is the constant, and the closed cells make the net flux 0
    m = MESHES[name]()
    U = np.array([0.3, -0.7, 0.45])
    u = m.normals @ U
    th = np.full(m.n_cells, 1.25)
    out = oracle.step(m, "superbee", rk, 0.01, 3, u, th)
    assert np.max(np.abs(out - 1.25)) <= 1e-14


@pytest.mark.parametrize("name", ["tet", "prism"])
def test_conservation(name):
    m = MESHES[name]()
    rng = np.random.default_rng(8)
    th = rng.uniform(0, 1, m.n_cells)
    u = 0.2 * W.mixed_sign_velocity(m.n_faces, 9)
    out = oracle.step(m, "smart", 3, 0.002, 5, u, th)
    m0 = float(np.sum(th * m.volumes))
    assert abs(float(np.sum(out * m.volumes)) - m0) <= 1e-14 * 10
