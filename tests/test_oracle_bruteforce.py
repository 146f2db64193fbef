"""The stencil oracle against the paper's matrix algebra, assembled densely
(brute force) on tiny meshes, and the topology constructors against the
matrices printed for the paper's 2D example."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import brute

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]


def test_printed_face_adjacency(golden):
    # eq. (ADJM) is reproduced exactly from the printed incidence eq. (Tfc)
    E = golden("paper_E_CF_2d.txt")
    _, _, _, A, _ = brute.topology(E)
    assert np.array_equal(A, golden("paper_A_FF_2d.txt"))
    assert np.all(A >= 0)
    assert np.array_equal(A, A.T)


def test_printed_directed_adjacency_up_to_orientation(golden):
    # eq. (DADJM) equals offdiag(E B^T) up to one global sign: the printed
    # example takes face orientation opposite to the text's convention
    E = golden("paper_E_CF_2d.txt")
    _, _, _, A, DA = brute.topology(E)
    printed = golden("paper_DA_FF_2d.txt")
    assert np.array_equal(printed, -DA)
    assert np.array_equal(np.abs(printed), A)


def _mesh_1d(n=8):
    return W.structured_mesh(n, 1, 1, 1.0 / n, 1.0, 1.0)


def _mesh_3d(n=4):
    h = 2 * np.pi / n
    return W.structured_mesh(n, n, n, h, h, h)


def _mesh_3d_aniso():
    return W.structured_mesh(5, 4, 6, 0.3, 0.7, 1.1)


MESHES = {"1d8": _mesh_1d, "3d4": _mesh_3d, "3d546": _mesh_3d_aniso}


@pytest.mark.parametrize("mname", sorted(MESHES))
@pytest.mark.parametrize("lim", LIMS)
def test_stencil_equals_matrix_algebra(mname, lim):
    mesh = MESHES[mname]()
    ops = brute.operators(mesh)
    rng = np.random.default_rng(123)
    th = rng.normal(size=mesh.n_cells)
    u = W.mixed_sign_velocity(mesh.n_faces, 7)
    fv = oracle.face_values(mesh, lim, th, u)
    thf, du, dU = brute.face_values(ops, lim, th, u)
    C, D, U = brute.selection(ops, u)
    # selection is exact
    assert np.array_equal(fv["C"], C)
    assert np.array_equal(fv["D"], D)
    assert np.array_equal(fv["U"], U)
    assert np.array_equal(fv["s"], np.where(u > 0, 1, -1))
    scale = np.max(np.abs(th))
    np.testing.assert_allclose(fv["du"], du, rtol=0, atol=1e-15 * scale)
    np.testing.assert_allclose(fv["dU"], dU, rtol=0, atol=2e-15 * scale)
    np.testing.assert_allclose(fv["theta_f"], thf, rtol=0, atol=1e-14 * scale)
    R = oracle.rhs(mesh, lim, th, u)
    Rb = ops["M"] @ (u * thf)
    np.testing.assert_allclose(R, Rb, rtol=0, atol=1e-13 * np.max(np.abs(Rb)))


@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_steps_equal_matrix_algebra(rk, lim):
    mesh = _mesh_3d()
    ops = brute.operators(mesh)
    rng = np.random.default_rng(5)
    th = rng.uniform(0, 1, mesh.n_cells)
    u = W.mixed_sign_velocity(mesh.n_faces, 3)
    dt = 0.1 * mesh.h[0] / np.max(np.abs(u))
    a = oracle.step(mesh, lim, rk, dt, 5, u, th)
    b = brute.step(ops, lim, rk, dt, 5, u, th)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_upstream_sign_correction_needed():
    # Without the left factor Q the printed d_U = N (I x A^U) N^T E theta
    # flips sign for faces whose flow runs against the normal: the corrected
    # form is required for Sweby's ratio on both flow directions.
    mesh = _mesh_1d()
    ops = brute.operators(mesh)
    th = np.random.default_rng(0).normal(size=8)
    u = np.array([1, -1, 1, -1, 1, -1, 1, -1], dtype=float)
    Q = brute.sign_matrix(u)
    AU = 0.5 * (ops["A"] - Q @ ops["DA"])
    printed = ops["N"] @ np.kron(np.eye(ops["d"]), AU) @ ops["N"].T @ ops["E"] @ th
    fv = oracle.face_values(mesh, "superbee", th, u)
    sweby = th[fv["C"]] - th[fv["U"]]
    assert np.allclose(fv["dU"], sweby, atol=1e-15)
    assert np.allclose(printed[u > 0], sweby[u > 0], atol=1e-15)
    assert np.allclose(printed[u < 0], -sweby[u < 0], atol=1e-15)
