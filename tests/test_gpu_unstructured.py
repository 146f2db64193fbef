"""Parity of the CUDA face-based (unstructured storage) path with the oracle.

Meshes are hexahedral boxes written out face by face, relabelled with seeded
random permutations and with a seeded half of the faces reoriented (c0 <-> c1,
normal and u_f negated).  The library renumbers them for locality; the tests
hold every field in the user's numbering and convert it with the library's
own calls (fl_mesh_to_internal / fl_mesh_to_user)."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _perm_case(shape, seed=2, h=None):
    h = h or (0.7 / shape[0], 0.9 / shape[1], 1.1 / shape[2])
    base = W.structured_mesh(*shape, *h)
    pm, cp, fp, flip = W.permuted_mesh(base, seed=seed)
    return base, pm, cp, fp, flip


class Dev:
    """Library mesh; fields cross to and from its internal numbering through
    the library's own conversion calls (fl_mesh_to_internal / _to_user)."""

    def __init__(self, fl, mesh, renumber=True):
        self.m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                                    mesh.volumes, renumber=renumber)
        self._maps()

    def _maps(self):
        # the published numbering, used only to translate the cell ids that
        # the selection dump reports (an index output, not a field)
        self.cp, self.fp, flip = self.m.permutation()
        assert not flip.any()

    def cells_in(self, x, dtype):
        return self.m.to_internal(torch.tensor(x, dtype=dtype, device="cuda"), "cell")

    def faces_in(self, x, dtype):
        return self.m.to_internal(torch.tensor(x, dtype=dtype, device="cuda"), "face")

    def cells_out(self, t):
        return self.m.to_user(t, "cell").cpu().double().numpy()

    def faces_out(self, t):
        return self.m.to_user(t, "face").cpu().double().numpy()


@pytest.mark.parametrize("renumber", [True, False])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("shape", [(12, 12, 12), (17, 9, 6), (9, 1, 1), (11, 7, 1)])
def test_apply_and_selection(fl, shape, lim, dtype, renumber):
    _, pm, _, _, _ = _perm_case(shape)
    rng = np.random.default_rng(1)
    th = rng.uniform(-1, 1, pm.n_cells) + (rng.random(pm.n_cells) < 0.3)
    u = W.mixed_sign_velocity(pm.n_faces, 5)
    if dtype == torch.float32:
        th = th.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    d = Dev(fl, pm, renumber)
    R = torch.empty(pm.n_cells, dtype=dtype, device="cuda")
    thf = torch.empty(pm.n_faces, dtype=dtype, device="cuda")
    ud = d.faces_in(u, dtype)
    fl.fl_conv_limited_apply(d.m.handle, lim, dtype, d.cells_in(th, dtype), ud, R, thf)
    ref = oracle.face_values(pm, lim, th, u)
    assert _rel(d.faces_out(thf), ref["theta_f"]) <= TOL[dtype]
    R_ref = oracle.rhs(pm, lim, th, u)
    scale = np.max(np.abs(u)) * np.max(np.abs(th)) * np.max(pm.areas) / np.min(pm.volumes)
    assert np.max(np.abs(d.cells_out(R) - R_ref)) <= 8 * TOL[dtype] * scale
    sel = torch.empty((pm.n_faces, 4), dtype=torch.int32, device="cuda")
    fl.fl_face_selection(d.m.handle, dtype, ud, sel)
    s = sel.cpu().numpy()[d.fp]  # rows back in user face order, cells internal
    inv = np.empty_like(d.cp)
    inv[d.cp] = np.arange(len(d.cp))
    assert np.array_equal(s[:, 0], ref["s"])
    assert np.array_equal(inv[s[:, 1]], ref["C"])
    assert np.array_equal(inv[s[:, 2]], ref["D"])
    if min(x for x in shape if x > 1) >= 3:
        assert np.array_equal(inv[s[:, 3]], ref["U"])
    d.m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_step_parity_per_step(fl, lim, rk, dtype):
    _, pm, _, _, _ = _perm_case((13, 10, 7), seed=4)
    rng = np.random.default_rng(3)
    th = rng.uniform(0, 1, pm.n_cells)
    u = 0.3 * W.mixed_sign_velocity(pm.n_faces, 8)
    dt = 0.1 * (0.7 / 13) / np.max(np.abs(u))
    if dtype == torch.float32:
        th = th.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    d = Dev(fl, pm)
    ud = d.faces_in(u, dtype)
    ws = torch.empty(fl.fl_workspace_size(d.m.handle, dtype, rk), dtype=torch.uint8,
                     device="cuda")
    cur = th
    for _ in range(3):
        ref = oracle.step(pm, lim, rk, dt, 1, u, cur)
        g = d.cells_in(cur, dtype)
        fl.fl_step_rk(d.m.handle, lim, dtype, rk, dt, 1, g, ud, ws, ws.numel())
        got = d.cells_out(g)
        assert _rel(got, ref) <= TOL[dtype]
        cur = ref if dtype == torch.float64 else got
    d.m.close()


def test_equals_structured_path(fl):
    # the same Taylor-Green case through both storage paths
    wl = W.config_taylor_green(n=20, seed=1, nsteps=4, limiter="smart")
    pm, cp, fp, flip = W.permuted_mesh(wl.mesh, seed=2)
    up = W.permute_face_field(wl.u, fp, flip)
    thp = W.permute_cell_field(wl.theta0, cp)
    d = Dev(fl, pm)
    g = d.cells_in(thp, torch.float64)
    ws = torch.empty(fl.fl_workspace_size(d.m.handle, torch.float64, 3), dtype=torch.uint8,
                     device="cuda")
    fl.fl_step_rk(d.m.handle, "smart", torch.float64, 3, wl.dt, 4, g, d.faces_in(up, torch.float64),
                  ws, ws.numel())
    un = d.cells_out(g)[cp]  # back to the structured numbering
    ms = fl.Mesh.structured(20, 20, 20, *wl.mesh.h)
    gs = torch.tensor(wl.theta0, device="cuda")
    fl.step_rk(ms, "smart", gs, torch.tensor(wl.u, device="cuda"), wl.dt, 4, rk_order=3)
    assert _rel(un, gs.cpu().numpy()) <= 1e-13
    d.m.close()
    ms.close()
