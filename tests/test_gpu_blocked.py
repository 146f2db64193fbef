"""Parity of the temporally blocked step (fl_step_rk_blocked: one launch per
SSP-RK3 step or per three Euler steps, each stage's halo recomputed on chip)
with the CPU oracle, through the C ABI.

Per launch the GPU starts from the oracle's theta^n; the bar is
||theta_gpu - theta_ref||_inf / ||theta_ref||_inf <= 1e-12 in FP64 and 1e-5
in FP32.  Shapes span several 32 x 16 tiles with ragged tails, meshes
smaller than one tile's halo (the periodic wrap reaches around more than
once), 2D and 1D meshes, and z ranges split into several chunks.  At the
256^3 size the benchmark times, sampled cells are recomputed by the oracle
on local patches and the mass is checked over the whole mesh."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.patch import patch

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
SHAPES = [(37, 21, 13), (64, 48, 40), (33, 17, 25), (5, 3, 7), (40, 9, 1), (70, 1, 1),
          (1, 12, 7), (2, 2, 2)]


def _inputs(shape, dtype, seed=5):
    nx, ny, nz = shape
    h = (0.7 / nx, 0.9 / ny, 1.1 / nz)
    mesh = W.structured_mesh(nx, ny, nz, *h)
    rng = np.random.default_rng(seed)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, seed + 1)
    if dtype == torch.float32:
        th = th.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    umax = np.max(np.abs(u)) if u.size else 1.0
    dt = 0.4 * min(mesh.h) / umax / 3
    return mesh, th, u, dt


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("shape", SHAPES)
def test_rk3_step_per_launch(fl, shape, lim, dtype):
    mesh, th, u, dt = _inputs(shape, dtype)
    m = fl.Mesh.structured(*shape, *mesh.h)
    ud = _dev(u, dtype)
    cur = th
    for _ in range(2):
        ref = oracle.step(mesh, lim, 3, dt, 1, u, cur)
        g = _dev(cur, dtype)
        fl.step_rk_blocked(m, lim, g, ud, dt, 1, rk_order=3)
        got = g.cpu().double().numpy()
        assert _rel(got, ref) <= TOL[dtype], (shape, lim)
        cur = ref if dtype == torch.float64 else got
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("shape", SHAPES)
def test_three_euler_steps_per_launch(fl, shape, lim, dtype):
    mesh, th, u, dt = _inputs(shape, dtype, seed=9)
    m = fl.Mesh.structured(*shape, *mesh.h)
    ref = oracle.step(mesh, lim, 1, dt, 3, u, th)
    g = _dev(th, dtype)
    fl.step_rk_blocked(m, lim, g, _dev(u, dtype), dt, 3, rk_order=1)
    assert _rel(g.cpu().double().numpy(), ref) <= TOL[dtype], (shape, lim)
    m.close()


# Euler step counts that are not multiples of three: the rest runs stage by
# stage after the blocked launches; RK3 over several launches (ping-pong
# buffers, odd and even counts)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rk,nsteps", [(1, 1), (1, 2), (1, 4), (1, 5), (1, 7), (3, 2), (3, 3)])
@pytest.mark.parametrize("shape", [(37, 21, 13), (128, 16, 9)])
def test_step_counts(fl, shape, rk, nsteps, dtype):
    mesh, th, u, dt = _inputs(shape, dtype, seed=11)
    m = fl.Mesh.structured(*shape, *mesh.h)
    ref = oracle.step(mesh, "superbee", rk, dt, nsteps, u, th)
    g = _dev(th, dtype)
    fl.step_rk_blocked(m, "superbee", g, _dev(u, dtype), dt, nsteps, rk_order=rk)
    assert _rel(g.cpu().double().numpy(), ref) <= nsteps * TOL[dtype]
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_mass_conserved_over_rollout(fl, lim, dtype):
    shape = (64, 48, 40)
    mesh, th, u, dt = _inputs(shape, dtype, seed=13)
    m = fl.Mesh.structured(*shape, *mesh.h)
    g = _dev(th, dtype)
    ws = torch.empty(fl.fl_reduce_workspace_size(), dtype=torch.uint8, device="cuda")
    m0 = fl.fl_reduce_mass(m.handle, dtype, g, ws)
    fl.step_rk_blocked(m, lim, g, _dev(u, dtype), dt, 20, rk_order=3)
    m1 = fl.fl_reduce_mass(m.handle, dtype, g, ws)
    assert bool(torch.isfinite(g).all())
    # the cell sums telescope exactly only if every CTA computes bit-identical
    # halo values; a mismatch would leave O(dt R) per tile edge
    assert abs(m1 - m0) <= (1e-13 if dtype == torch.float64 else 1e-6) * abs(m0)
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", ["superbee", "smart"])
def test_full_size_256_sampled_and_conserved(fl, lim, dtype):
    """One blocked SSP-RK3 step of the 256^3 Taylor-Green case; 24 sampled
    cells recomputed by the oracle on 13^3 patches (radius 6 = 2 cells per
    stage), and mass conservation over the whole mesh."""
    n = 256
    wl = W.config_taylor_green(n=n, seed=1, nsteps=1, limiter=lim)
    th0, u = wl.theta0, wl.u
    if dtype == torch.float32:
        th0 = th0.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    g = _dev(th0, dtype)
    ws = torch.empty(fl.fl_reduce_workspace_size(), dtype=torch.uint8, device="cuda")
    m0 = fl.fl_reduce_mass(m.handle, dtype, g, ws)
    fl.step_rk_blocked(m, lim, g, _dev(u, dtype), wl.dt, 1, rk_order=3)
    m1 = fl.fl_reduce_mass(m.handle, dtype, g, ws)
    got = g.cpu().double().numpy()
    assert abs(m1 - m0) <= (1e-12 if dtype == torch.float64 else 1e-5) * abs(m0)
    rng = np.random.default_rng(17)
    scale = np.max(np.abs(th0))
    # tile corners (32 x 16 tiles), the periodic wrap, then random cells
    fixed = [(0, 0, 0), (255, 255, 255), (31, 15, 128), (32, 16, 127), (95, 47, 0)]
    cells = fixed + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(19)]
    for c in cells:
        pm, pc, fidx, centre = patch((n, n, n), wl.mesh.h, c, 6)
        ref = oracle.step(pm, lim, 3, wl.dt, 1, u[fidx], th0[pc])
        assert abs(got[pc[centre]] - ref[centre]) <= TOL[dtype] * scale, c
    m.close()


def test_errors(fl):
    mesh, th, u, dt = _inputs((8, 8, 8), torch.float64)
    m = fl.Mesh.structured(8, 8, 8, *mesh.h)
    g = _dev(th, torch.float64)
    ud = _dev(u, torch.float64)
    with pytest.raises(fl.FLError, match="rk_order"):
        fl.step_rk_blocked(m, "superbee", g, ud, dt, 1, rk_order=2)
    nb = fl.fl_workspace_size(m.handle, torch.float64, 3)
    small = torch.empty(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(fl.FLError, match="workspace too small"):
        fl.fl_step_rk_blocked(m.handle, "superbee", torch.float64, 3, dt, 1, g, ud, small, nb - 8)
    before = g.clone()
    fl.step_rk_blocked(m, "superbee", g, ud, dt, 0, rk_order=3)
    assert torch.equal(g, before)
    m.close()
    # a face-based mesh is refused before any launch
    um = W.structured_mesh(4, 4, 4, 0.25, 0.25, 0.25)
    fm = fl.Mesh.from_faces(um.n_cells, um.face_cells, um.normals, um.areas, um.volumes)
    th2 = _dev(np.ones(um.n_cells), torch.float64)
    u2 = _dev(np.ones(um.n_faces), torch.float64)
    with pytest.raises(fl.FLError, match="FL_EUNSUPPORTED"):
        fl.step_rk_blocked(fm, "superbee", th2, u2, 0.01, 1, rk_order=3)
    fm.close()
