"""fl_step_rk_noalloc: the explicit step for callers that cannot allocate.

Hosts such as plugin frameworks that own the device memory pool, real-time
loops that cannot pay for an allocation, or deployments whose memory is fixed
at start-up cannot hand this library a workspace.  fl_step_rk_noalloc takes
its stage buffers from a fixed scratch area inside the library instead.

These tests call it through the C ABI on every kind of mesh it serves (a 3D
structured box through the stage tile or, in FP32, the TMA kernel; a 1D line
on one CTA and on a cluster; renumbered face-based hexahedra and tetrahedra)
and check, twice in a row, that it gives the result of fl_step_rk with a
caller-provided workspace, and that one step matches the FP64 oracle; both
within the parity tolerances used everywhere (1e-12 relative in FP64, 1e-5
in FP32).  Meshes too large for the area are refused before anything runs.

The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}

# (mesh, dtype, rk, limiter)
CASES = [("box", torch.float64, 3, "superbee"),
         ("box", torch.float32, 1, "smart"),
         ("box", torch.float64, 1, "vanleer"),
         ("box_tma", torch.float32, 3, "vanleer"),
         ("line1000", torch.float64, 1, "vanleer"),
         ("line12", torch.float32, 3, "minmod"),
         ("hex_renumbered", torch.float64, 3, "smart"),
         ("tet", torch.float32, 3, "superbee")]


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


def _case(name, dtype):
    """(library mesh, user-order mesh for the oracle, theta, u, dt)."""
    import paper_2110_03044_gb300 as fl
    rng = np.random.default_rng(17)
    if name in ("box", "box_tma", "line1000", "line12"):
        shape = {"box": (37, 21, 13), "box_tma": (128, 8, 5), "line1000": (1000, 1, 1),
                 "line12": (12, 1, 1)}[name]
        mesh = W.structured_mesh(*shape, *(0.7 / s for s in shape))
        m = fl.Mesh.structured(*shape, *mesh.h)
    else:
        mesh = W.permuted_mesh(W.structured_mesh(9, 8, 7, 0.1, 0.1, 0.1), 3)[0] \
            if name == "hex_renumbered" else W.tet_mesh(4)
        m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                               mesh.volumes, renumber=True)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.2 * W.mixed_sign_velocity(mesh.n_faces, 4)
    if dtype == torch.float32:
        th = th.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    dt = 0.05 * np.min(mesh.volumes) / np.max(mesh.areas) / np.max(np.abs(u))
    return m, mesh, th, u, dt


@pytest.mark.parametrize("name,dtype,rk,lim", CASES)
def test_noalloc_matches_workspace_call_twice(fl, name, dtype, rk, lim):
    m, _, th, u, dt = _case(name, dtype)
    th0 = m.to_internal(torch.tensor(th, dtype=dtype, device="cuda"), "cell")
    ud = m.to_internal(torch.tensor(u, dtype=dtype, device="cuda"), "face")
    ref = th0.clone()
    new = th0.clone()
    for _ in range(2):  # two calls in a row, each advancing 3 steps
        fl.step_rk(m, lim, ref, ud, dt, 3, rk_order=rk)
        fl.fl_step_rk_noalloc(m.handle, lim, dtype, rk, dt, 3, new, ud)
        torch.cuda.synchronize()
        assert _rel(new, ref) <= TOL[dtype]
    m.close()


@pytest.mark.parametrize("name,dtype,rk,lim", CASES)
def test_noalloc_step_matches_oracle(fl, name, dtype, rk, lim):
    m, mesh, th, u, dt = _case(name, dtype)
    g = m.to_internal(torch.tensor(th, dtype=dtype, device="cuda"), "cell")
    ud = m.to_internal(torch.tensor(u, dtype=dtype, device="cuda"), "face")
    fl.fl_step_rk_noalloc(m.handle, lim, dtype, rk, dt, 1, g, ud)
    got = m.to_user(g, "cell").cpu().double().numpy()
    ref = oracle.step(mesh, lim, rk, dt, 1, u, th)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= TOL[dtype]
    m.close()


def test_noalloc_rejects_meshes_beyond_the_area(fl):
    # 2^21 + 2^20 FP64 cells need 48 MiB of RK3 stage buffers (> 32 MiB)
    n = 1 << 21
    m = fl.Mesh.structured(n + (n >> 1), 1, 1, 1.0, 1.0, 1.0)
    th = torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
    u = torch.zeros(m.n_faces, dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk_noalloc(m.handle, "superbee", torch.float64, 3, 0.1, 1, th, u)
    assert e.value.status == fl.FL_EINVAL
    m.close()
