"""The adjoint on face-based meshes (hexahedra in permuted order with
reoriented faces, tetrahedra, triangular prisms): the operator transpose
against the oracle's adjoint, the dot-product identity with the oracle's
tangent-linear model, and the checkpointed gradient against the oracle's
reference gradient."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_unstructured import Dev

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]


def _mesh(name):
    if name == "hex":
        return W.permuted_mesh(W.structured_mesh(9, 7, 6, 0.1, 0.12, 0.15), seed=3)[0]
    if name == "tet":
        return W.tet_mesh(4)
    return W.prism_mesh(4)


def _cast(x, dtype):
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("name", ["hex", "tet", "prism"])
def test_operator_adjoint_matches_oracle(fl, name, lim, dtype):
    m = _mesh(name)
    rng = np.random.default_rng(1)
    th = _cast(rng.uniform(-1, 1, m.n_cells) + (rng.random(m.n_cells) < 0.3), dtype)
    u = _cast(W.mixed_sign_velocity(m.n_faces, 2), dtype)
    mu = _cast(rng.normal(size=m.n_cells), dtype)
    d = Dev(fl, m)
    out = torch.empty(m.n_cells, dtype=dtype, device="cuda")
    fl.fl_conv_limited_adjoint(d.m.handle, lim, dtype, d.cells_in(th, dtype),
                               d.faces_in(u, dtype), d.cells_in(mu, dtype), out)
    ref = oracle.rhs_adjoint(m, lim, th, u, mu)
    scale = np.max(np.abs(u)) * np.max(np.abs(mu)) * np.max(m.areas) / np.min(m.volumes)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.max(np.abs(d.cells_out(out) - ref)) <= 16 * tol * scale
    d.m.close()


@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
@pytest.mark.parametrize("name", ["hex", "tet"])
def test_dot_product_with_cpu_tangent_linear(fl, name, lim):
    m = _mesh(name)
    rng = np.random.default_rng(5)
    th0 = rng.uniform(0, 1, m.n_cells)
    u = 0.3 * W.mixed_sign_velocity(m.n_faces, 6)
    dt = 0.05 * np.min(m.volumes) / np.max(m.areas) / np.max(np.abs(u))
    d = Dev(fl, m)
    nb = fl.fl_adjoint_workspace_size(d.m.handle, torch.float64, 3, 2, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        v = rng.normal(size=m.n_cells)
        w = rng.normal(size=m.n_cells)
        _, Jv = oracle.step_tlm(m, lim, 3, dt, 2, u, th0, v)
        JTw = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
        fl.fl_step_rk_adjoint(d.m.handle, lim, torch.float64, 3, dt, 2, 1,
                              d.cells_in(th0, torch.float64), d.faces_in(u, torch.float64),
                              d.cells_in(w, torch.float64), JTw, ws, nb)
        lhs = float(np.dot(Jv, w))
        rhs = float(np.dot(v, d.cells_out(JTw)))
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jv) * np.linalg.norm(w)
    d.m.close()


@pytest.mark.parametrize("rk,every", [(3, 3), (1, 4)])
@pytest.mark.parametrize("lim", ["superbee", "vanleer", "smart"])
@pytest.mark.parametrize("name", ["hex", "tet", "prism"])
def test_checkpointed_gradient_matches_oracle(fl, name, lim, rk, every):
    m = _mesh(name)
    nsteps = 7
    rng = np.random.default_rng(7)
    th0 = rng.uniform(0, 1, m.n_cells)
    tgt = rng.uniform(0, 1, m.n_cells)
    u = 0.3 * W.mixed_sign_velocity(m.n_faces, 8)
    dt = 0.05 * np.min(m.volumes) / np.max(m.areas) / np.max(np.abs(u))
    J_ref, g_ref = oracle.gradient(m, lim, rk, dt, nsteps, u, th0, tgt)
    thT = oracle.step(m, lim, rk, dt, nsteps, u, th0)
    d = Dev(fl, m)
    nb = fl.fl_adjoint_workspace_size(d.m.handle, torch.float64, rk, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_step_rk_adjoint(d.m.handle, lim, torch.float64, rk, dt, nsteps, every,
                          d.cells_in(th0, torch.float64), d.faces_in(u, torch.float64),
                          d.cells_in(thT - tgt, torch.float64), g, ws, nb)
    gg = d.cells_out(g)
    assert np.max(np.abs(gg - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))
    d.m.close()
