"""Host-side validation of fl_mesh_create (no GPU needed: every rejection
happens before any device call)."""
import numpy as np
import pytest

import workloads as W


def _box():
    return W.structured_mesh(4, 4, 4, 0.25, 0.25, 0.25)


def _create(fl, m, fc=None, nrm=None, ar=None, vol=None, n_cells=None):
    return fl.fl_mesh_create(m.n_cells if n_cells is None else n_cells,
                             m.face_cells if fc is None else fc,
                             m.normals if nrm is None else nrm,
                             m.areas if ar is None else ar,
                             m.volumes if vol is None else vol, fl.FL_RENUMBER)


@pytest.mark.parametrize("bad", ["n_cells", -1])
def test_rejects_out_of_range_cells(fl, bad):
    # an index outside [0, n_cells) in the connectivity is FL_EINDEX
    m = _box()
    fc = m.face_cells.copy()
    fc[5, 1] = m.n_cells if bad == "n_cells" else bad
    with pytest.raises(fl.FLError) as e:
        _create(fl, m, fc=fc)
    assert e.value.status == fl.FL_EINDEX
    assert "out of range" in str(e.value)


def test_algebraic_chain_rejects_out_of_range_cells(fl):
    m = _box()
    fc = m.face_cells.copy()
    fc[7, 0] = m.n_cells + 3
    with pytest.raises(fl.FLError) as e:
        fl.fl_alg_create(m.n_cells, fc, m.normals, m.areas, m.volumes)
    assert e.value.status == fl.FL_EINDEX


def test_rejects_degenerate_face(fl):
    m = _box()
    fc = m.face_cells.copy()
    fc[3, 1] = fc[3, 0]
    with pytest.raises(fl.FLError) as e:
        _create(fl, m, fc=fc)
    assert e.value.status == fl.FL_EINVAL


def test_rejects_non_unit_normal_and_bad_geometry(fl):
    m = _box()
    nrm = m.normals.copy()
    nrm[0] *= 1.5
    with pytest.raises(fl.FLError):
        _create(fl, m, nrm=nrm)
    ar = m.areas.copy()
    ar[2] = 0.0
    with pytest.raises(fl.FLError):
        _create(fl, m, ar=ar)
    vol = m.volumes.copy()
    vol[1] = -1.0
    with pytest.raises(fl.FLError):
        _create(fl, m, vol=vol)


def test_rejects_duplicated_face(fl):
    m = _box()
    fc = np.concatenate([m.face_cells, m.face_cells[:1]])
    nrm = np.concatenate([m.normals, m.normals[:1]])
    ar = np.concatenate([m.areas, m.areas[:1]])
    with pytest.raises(fl.FLError) as e:
        _create(fl, m, fc=fc, nrm=nrm, ar=ar)
    assert e.value.status in (fl.FL_EINVAL, fl.FL_EUNSUPPORTED)


def test_general_polyhedra_pass_host_validation(fl):
    # tetrahedra have no opposite faces: the mesh takes the general
    # weighted upstream stencil, and every host-side check passes (on a
    # machine without a GPU creation stops only at the device step)
    import workloads as W
    m = W.tet_mesh(3)
    with pytest.raises(fl.FLError) as e:
        _create(fl, m)
    assert e.value.status == fl.FL_ECUDA


def test_rejects_cells_with_too_many_faces(fl):
    # more than 8 faces on one cell: beyond the per-cell slot table
    m = _box()
    extra = 4
    fc = np.concatenate([m.face_cells, np.tile(m.face_cells[:1], (extra, 1))])
    nrm = np.concatenate([m.normals, np.tile(m.normals[:1], (extra, 1))])
    ar = np.concatenate([m.areas, np.tile(m.areas[:1], extra)])
    with pytest.raises(fl.FLError) as e:
        _create(fl, m, fc=fc, nrm=nrm, ar=ar)
    assert e.value.status in (fl.FL_EINVAL, fl.FL_EUNSUPPORTED)


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_rejects_bad_face_distance(fl, bad):
    m = W.stretched_mesh(W.stretched_widths(8, 1.0, 2.0, 1), W.stretched_widths(5, 1.0, 2.0, 2))
    d = m.distances.copy()
    d[4] = bad
    with pytest.raises(fl.FLError) as e:
        fl.fl_mesh_create_weighted(m.n_cells, m.face_cells, m.normals, m.areas, m.volumes, d,
                                   fl.FL_RENUMBER)
    assert e.value.status == fl.FL_EINVAL
    assert "distance" in str(e.value)


def test_rejects_missing_face_distances(fl):
    m = _box()
    with pytest.raises(ValueError):
        fl.fl_mesh_create_weighted(m.n_cells, m.face_cells, m.normals, m.areas, m.volumes,
                                   np.ones(m.n_faces - 1))
