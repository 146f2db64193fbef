"""Non-hexahedral face-based meshes (tetrahedra, triangular prisms) on the
fused unstructured kernel: the upstream difference is the weighted sum over
the other faces of the upwind cell (eq. Delta_Upwind with the sign
correction), against the oracle -- face values, selection, R(theta) and
steps -- plus free-stream preservation and the algebraic chain on the same
meshes."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_unstructured import Dev

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
MESHES = {"tet3": lambda: W.tet_mesh(3), "tet5": lambda: W.tet_mesh(5),
          "prism4": lambda: W.prism_mesh(4)}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _cast(x, dtype):
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


@pytest.mark.parametrize("renumber", [True, False])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("name", ["tet3", "tet5", "prism4"])
def test_apply_and_selection(fl, name, lim, dtype, renumber):
    m = MESHES[name]()
    rng = np.random.default_rng(2)
    th = _cast(rng.uniform(-1, 1, m.n_cells) + (rng.random(m.n_cells) < 0.3), dtype)
    u = _cast(W.mixed_sign_velocity(m.n_faces, 3), dtype)
    d = Dev(fl, m, renumber)
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
    # U exists where exactly one other face of C is not orthogonal to f
    has_u = ref["U"] >= 0
    assert np.array_equal(s[~has_u, 3], ref["U"][~has_u])
    assert np.array_equal(inv[s[has_u, 3]], ref["U"][has_u])
    d.m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
@pytest.mark.parametrize("name", ["tet5", "prism4"])
def test_step_parity_per_step(fl, name, lim, rk, dtype):
    m = MESHES[name]()
    rng = np.random.default_rng(4)
    th = _cast(rng.uniform(0, 1, m.n_cells), dtype)
    u = _cast(0.3 * W.mixed_sign_velocity(m.n_faces, 5), dtype)
    dt = 0.05 * np.min(m.volumes) / np.max(m.areas) / np.max(np.abs(u))
    d = Dev(fl, m)
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


@pytest.mark.parametrize("name", ["tet5", "prism4"])
def test_free_stream_and_conservation(fl, name):
    m = MESHES[name]()
    U = np.array([0.3, -0.7, 0.45])
    u = m.normals @ U
    d = Dev(fl, m)
    ud = d.faces_in(u, torch.float64)
    th = d.cells_in(np.full(m.n_cells, 1.25), torch.float64)
    fl.step_rk(d.m, "superbee", th, ud, 0.002, 5, rk_order=3)
    assert float((th - 1.25).abs().max()) <= 1e-14
    rng = np.random.default_rng(6)
    th0 = rng.uniform(0, 1, m.n_cells)
    g = d.cells_in(th0, torch.float64)
    fl.step_rk(d.m, "smart", g, ud, 0.002, 5, rk_order=3)
    got = d.cells_out(g)
    m0 = float(np.sum(th0 * m.volumes))
    assert abs(float(np.sum(got * m.volumes)) - m0) <= 1e-13
    d.m.close()


@pytest.mark.parametrize("lim", ["superbee", "smart"])
def test_algebraic_chain_on_tetrahedra(fl, lim):
    m = W.tet_mesh(4)
    rng = np.random.default_rng(7)
    th = rng.uniform(-1, 1, m.n_cells)
    u = W.mixed_sign_velocity(m.n_faces, 8)
    a = fl.Algebraic(m.n_cells, m.face_cells, m.normals, m.areas, m.volumes)
    got = a.face_values(lim, torch.tensor(th, device="cuda"), torch.tensor(u, device="cuda"))
    assert _rel(got.cpu().numpy(), oracle.face_values(m, lim, th, u)["theta_f"]) <= 1e-12
    a.close()
