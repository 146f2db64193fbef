"""Geometry of the stretched (non-uniform) tensor-product meshes that stand
in for non-uniform inputs: closed cells, volumes that fill the box, face
distances equal to the distance between the cell centres, and the uniform
case reducing to the uniform box."""
import numpy as np

import workloads as W


def test_stretched_box_geometry():
    wx = W.stretched_widths(9, 2.0, 3.0, 1)
    wy = W.stretched_widths(7, 1.5, 2.0, 2)
    wz = W.stretched_widths(5, 1.0, 2.5, 3)
    assert abs(wx.sum() - 2.0) <= 1e-14 and wx.max() / wx.min() <= 3.0 + 1e-12
    m = W.stretched_mesh(wx, wy, wz)
    C = m.n_cells
    # volumes fill the box
    assert abs(m.volumes.sum() - 2.0 * 1.5 * 1.0) <= 1e-12
    # every cell is closed: the signed area vectors of its faces sum to zero
    s = np.zeros((C, 3))
    vec = m.normals * m.areas[:, None]
    np.add.at(s, m.face_cells[:, 0], vec)
    np.add.at(s, m.face_cells[:, 1], -vec)
    assert np.max(np.abs(s)) <= 1e-14
    # distances: centre to centre along the face normal (periodic)
    cx = np.cumsum(wx) - 0.5 * wx
    cy = np.cumsum(wy) - 0.5 * wy
    cz = np.cumsum(wz) - 0.5 * wz
    idx = np.arange(C)
    centre = np.stack([cx[idx % 9], cy[(idx // 9) % 7], cz[idx // 63]], axis=1)
    L = np.array([2.0, 1.5, 1.0])
    delta = centre[m.face_cells[:, 1]] - centre[m.face_cells[:, 0]]
    delta = (delta + 0.5 * L) % L - 0.5 * L  # periodic image
    along = np.einsum("ij,ij->i", delta, m.normals)
    np.testing.assert_allclose(along, m.distances, rtol=0, atol=1e-14)


def test_uniform_widths_give_the_uniform_box():
    m = W.stretched_mesh(np.full(6, 0.25), np.full(5, 0.25), np.full(4, 0.25))
    u = W.structured_mesh(6, 5, 4, 0.25, 0.25, 0.25)
    np.testing.assert_array_equal(m.face_cells, u.face_cells)
    np.testing.assert_array_equal(m.normals, u.normals)
    np.testing.assert_allclose(m.areas, u.areas, rtol=1e-15)
    np.testing.assert_allclose(m.volumes, u.volumes, rtol=1e-15)
    np.testing.assert_array_equal(m.distances, np.full(m.n_faces, 0.25))
