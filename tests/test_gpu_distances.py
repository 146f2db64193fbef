"""Non-uniform face-based meshes (fl_mesh_create_weighted: Algorithm 3's
distance weights in the upstream difference) against the oracle with the
same distances: face values, selection, R(theta), steps, conservation and
the adjoint, on stretched hexahedral boxes (in permuted order with
reoriented faces, with and without the library's renumbering) and on
tetrahedra with seeded distances."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_unstructured import Dev

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


class DevW(Dev):
    """Dev for a mesh with face distances."""

    def __init__(self, fl, mesh, renumber=True):
        self.m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                                    mesh.volumes, renumber=renumber, distances=mesh.distances)
        self._maps()


def _mesh(name):
    if name == "box":
        wx = W.stretched_widths(13, 1.0, 3.0, 1)
        wy = W.stretched_widths(10, 0.9, 2.0, 2)
        wz = W.stretched_widths(7, 0.7, 2.5, 3)
        return W.stretched_mesh(wx, wy, wz)
    if name == "box_permuted":
        return W.permuted_mesh(_mesh("box"), seed=4)[0]
    if name == "line":
        return W.stretched_mesh(W.stretched_widths(41, 1.0, 4.0, 5))
    m = W.tet_mesh(4)
    m.distances = np.random.default_rng(6).uniform(0.1, 0.3, m.n_faces)
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _cast(x, dtype):
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


@pytest.mark.parametrize("renumber", [True, False])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("name", ["box", "box_permuted", "line", "tet"])
def test_apply_and_selection(fl, name, lim, dtype, renumber):
    m = _mesh(name)
    rng = np.random.default_rng(7)
    th = _cast(rng.uniform(-1, 1, m.n_cells) + (rng.random(m.n_cells) < 0.3), dtype)
    u = _cast(W.mixed_sign_velocity(m.n_faces, 8), dtype)
    d = DevW(fl, m, renumber)
    R = torch.empty(m.n_cells, dtype=dtype, device="cuda")
    thf = torch.empty(m.n_faces, dtype=dtype, device="cuda")
    ud = d.faces_in(u, dtype)
    fl.fl_conv_limited_apply(d.m.handle, lim, dtype, d.cells_in(th, dtype), ud, R, thf)
    ref = oracle.face_values(m, lim, th, u)
    assert _rel(d.faces_out(thf), ref["theta_f"]) <= TOL[dtype]
    R_ref = oracle.rhs(m, lim, th, u)
    scale = np.max(np.abs(u)) * np.max(np.abs(th)) * np.max(m.areas) / np.min(m.volumes)
    assert np.max(np.abs(d.cells_out(R) - R_ref)) <= 16 * TOL[dtype] * scale
    sel = torch.empty((m.n_faces, 4), dtype=torch.int32, device="cuda")
    fl.fl_face_selection(d.m.handle, dtype, ud, sel)
    s = sel.cpu().numpy()[d.fp]
    inv = np.empty_like(d.cp)
    inv[d.cp] = np.arange(len(d.cp))
    assert np.array_equal(s[:, 0], ref["s"])
    assert np.array_equal(inv[s[:, 1]], ref["C"])
    assert np.array_equal(inv[s[:, 2]], ref["D"])
    has_u = ref["U"] >= 0
    assert np.array_equal(s[~has_u, 3], ref["U"][~has_u])
    assert np.array_equal(inv[s[has_u, 3]], ref["U"][has_u])
    d.m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
@pytest.mark.parametrize("name", ["box_permuted", "tet"])
def test_step_parity_per_step(fl, name, lim, rk, dtype):
    m = _mesh(name)
    rng = np.random.default_rng(9)
    th = _cast(rng.uniform(0, 1, m.n_cells), dtype)
    u = _cast(0.3 * W.mixed_sign_velocity(m.n_faces, 10), dtype)
    dt = 0.05 * np.min(m.volumes) / np.max(m.areas) / np.max(np.abs(u))
    d = DevW(fl, m)
    ud = d.faces_in(u, dtype)
    ws = torch.empty(fl.fl_workspace_size(d.m.handle, dtype, rk), dtype=torch.uint8,
                     device="cuda")
    cur = th
    for _ in range(3):
        ref = oracle.step(m, lim, rk, dt, 1, u, cur)
        g = d.cells_in(cur, dtype)
        fl.fl_step_rk(d.m.handle, lim, dtype, rk, dt, 1, g, ud, ws, ws.numel())
        got = d.cells_out(g)
        assert _rel(got, ref) <= TOL[dtype]
        cur = ref if dtype == torch.float64 else got
    d.m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_mass_conserved(fl, dtype):
    m = _mesh("box_permuted")
    rng = np.random.default_rng(11)
    th = _cast(rng.uniform(0, 1, m.n_cells), dtype)
    u = _cast(0.3 * W.mixed_sign_velocity(m.n_faces, 12), dtype)
    dt = 0.05 * np.min(m.volumes) / np.max(m.areas) / np.max(np.abs(u))
    d = DevW(fl, m)
    g = d.cells_in(th, dtype)
    fl.step_rk(d.m, "superbee", g, d.faces_in(u, dtype), dt, 30, rk_order=3)
    got = d.cells_out(g)
    m0, m1 = np.sum(m.volumes * th), np.sum(m.volumes * got)
    assert np.all(np.isfinite(got))
    assert abs(m1 - m0) <= (1e-13 if dtype == torch.float64 else 1e-6) * abs(m0)
    d.m.close()


def test_uniform_distances_match_the_unweighted_mesh(fl):
    """Equal distances reduce the weights to 1: the weighted general stencil
    and the unweighted hexahedral path agree to rounding."""
    base = W.permuted_mesh(W.structured_mesh(12, 9, 7, 0.25, 0.25, 0.25), seed=13)[0]
    rng = np.random.default_rng(14)
    th = rng.uniform(0, 1, base.n_cells)
    u = W.mixed_sign_velocity(base.n_faces, 15)
    plain = Dev(fl, base)
    base.distances = np.full(base.n_faces, 0.25)
    weighted = DevW(fl, base)
    for d in (plain, weighted):
        g = d.cells_in(th, torch.float64)
        fl.step_rk(d.m, "smart", g, d.faces_in(u, torch.float64), 0.01, 2, rk_order=3)
        d.result = d.cells_out(g)
        d.m.close()
    assert _rel(weighted.result, plain.result) <= 1e-14


@pytest.mark.parametrize("lim", ["superbee", "vanleer", "smart"])
@pytest.mark.parametrize("name", ["box_permuted", "tet"])
def test_operator_adjoint_and_gradient(fl, name, lim):
    m = _mesh(name)
    rng = np.random.default_rng(16)
    th = rng.uniform(0, 1, m.n_cells)
    u = 0.3 * W.mixed_sign_velocity(m.n_faces, 17)
    mu = rng.normal(size=m.n_cells)
    d = DevW(fl, m)
    out = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_conv_limited_adjoint(d.m.handle, lim, torch.float64, d.cells_in(th, torch.float64),
                               d.faces_in(u, torch.float64), d.cells_in(mu, torch.float64), out)
    ref = oracle.rhs_adjoint(m, lim, th, u, mu)
    scale = np.max(np.abs(u)) * np.max(np.abs(mu)) * np.max(m.areas) / np.min(m.volumes)
    assert np.max(np.abs(d.cells_out(out) - ref)) <= 16e-12 * scale
    # checkpointed gradient of J = 0.5 ||theta_T - target||^2 over 4 steps
    dt = 0.05 * np.min(m.volumes) / np.max(m.areas) / np.max(np.abs(u))
    target = rng.uniform(0, 1, m.n_cells)
    _, g_ref = oracle.gradient(m, lim, 3, dt, 4, u, th, target)
    th_T = oracle.step(m, lim, 3, dt, 4, u, th)
    nb = fl.fl_adjoint_workspace_size(d.m.handle, torch.float64, 3, 4, 2)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    grad = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_step_rk_adjoint(d.m.handle, lim, torch.float64, 3, dt, 4, 2,
                          d.cells_in(th, torch.float64), d.faces_in(u, torch.float64),
                          d.cells_in(th_T - target, torch.float64), grad, ws, nb)
    assert _rel(d.cells_out(grad), g_ref) <= 1e-11
    d.m.close()


def test_distance_errors(fl):
    m = _mesh("line")
    bad = m.distances.copy()
    bad[3] = 0.0
    with pytest.raises(fl.FLError, match="bad distance"):
        fl.Mesh.from_faces(m.n_cells, m.face_cells, m.normals, m.areas, m.volumes,
                           distances=bad)
    bad[3] = np.nan
    with pytest.raises(fl.FLError, match="bad distance"):
        fl.Mesh.from_faces(m.n_cells, m.face_cells, m.normals, m.areas, m.volumes,
                           distances=bad)
    with pytest.raises(ValueError):
        fl.Mesh.from_faces(m.n_cells, m.face_cells, m.normals, m.areas, m.volumes,
                           distances=m.distances[:-1])
