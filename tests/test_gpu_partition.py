"""The graph partition on the GPU: W ranks emulated in one process on one
GPU, each a host thread with its own local mesh (fl_mesh_create_local),
running the library's cell-range stage kernels through the same step_rk /
gradient_rk loops a multi-GPU run uses.  The exchange
(ThreadGroupGraphTransport) gathers each neighbour's values with
fl_halo_pack straight into the receiving rank's halo slice, between two host
barriers; every launch goes to the one default stream, in order, so no
kernel waits on another.

* The owned cells of the partitioned rollout equal fl_step_rk_stage on the
  whole (not renumbered) face-based mesh bit for bit: local faces keep the
  whole mesh's relative order, and only the stencils of owned and first-ring
  cells are resolved, so hexahedra keep their single-term upstream stencil.
* The partitioned reverse sweep equals fl_step_rk_adjoint on the whole mesh
  to rounding, and the oracle's gradient.
* The cell-range entry points, the halo gather (with its FL_EINDEX latch) and
  the local-mesh argument checks."""
import threading

import numpy as np
import pytest
import torch

import workloads as W
from paper_2110_03044_gb300.partition import (GraphRollout, ThreadGroupGraphTransport, build_parts,
                                              partition_graph)

pytestmark = pytest.mark.gpu

MESHES = {
    "hex": lambda: W.structured_mesh(12, 10, 8, 0.7 / 12, 0.9 / 10, 1.1 / 8),
    "tet": lambda: W.tet_mesh(5),
    "prism": lambda: W.prism_mesh(5),
    "tiny": lambda: W.structured_mesh(4, 3, 2, 0.25, 0.3, 0.5),
}


def _case(name):
    mesh = MESHES[name]()
    rng = np.random.default_rng(5)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 6)
    dt = 0.1 * float(np.min(mesh.volumes)) ** (1 / 3) / float(np.max(np.abs(u)))
    return mesh, th, u, dt


def _partitioned(fl, name, world, lim, dtype, rk, nsteps, overlap=True, grad=None,
                 renumber=False):
    mesh, th, u, dt = _case(name)
    part = partition_graph(mesh.n_cells, mesh.face_cells, world)
    parts = build_parts(mesh.n_cells, mesh.face_cells, part, world)
    tr = ThreadGroupGraphTransport(world)
    ug = torch.tensor(u, dtype=dtype, device="cuda")
    rollouts = [GraphRollout(mesh, gp, ug, lim, dtype, dt, transport=tr, overlap=overlap,
                             renumber=renumber) for gp in parts]
    for ro in rollouts:
        tr.register(ro)
    out = [None] * world
    err = []

    def rank(r):
        try:
            torch.cuda.set_device(0)
            ro = rollouts[r]
            tl = ro.local_field(torch.tensor(th, dtype=dtype, device="cuda"))
            if grad is None:
                res = ro.step(tl, rk, nsteps)
            else:
                lam = ro.local_field(torch.tensor(grad, dtype=dtype, device="cuda"))
                res = ro.gradient(tl, lam, rk, nsteps, 2)
            torch.cuda.synchronize()
            out[r] = (ro.gp.owned_ids, ro.gp.owned(res).cpu())
        except BaseException as e:  # noqa: BLE001 -- reported below
            err.append(e)
            tr.bar.abort()

    ts = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for ro in rollouts:
        ro.close()
    if err:
        raise err[0]
    got = torch.empty(mesh.n_cells, dtype=dtype)
    for ids, vals in out:
        got[torch.as_tensor(ids)] = vals
    return got


def _whole_mesh(fl, mesh):
    return fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                              mesh.volumes)


@pytest.mark.parametrize("name,world,overlap", [("hex", 1, True), ("hex", 2, True),
                                                ("hex", 3, True), ("hex", 4, False),
                                                ("tet", 3, True), ("prism", 2, True),
                                                ("tiny", 7, True), ("tiny", 30, True)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1), ("smart", 3)])
def test_partitioned_rollout_equals_whole_mesh_bitwise(fl, name, world, overlap, dtype, lim, rk):
    mesh, th, u, dt = _case(name)
    nsteps = 3
    got = _partitioned(fl, name, world, lim, dtype, rk, nsteps, overlap)
    m = _whole_mesh(fl, mesh)
    uu = torch.tensor(u, dtype=dtype, device="cuda")
    w = None
    if dtype == torch.float64:
        w = torch.empty_like(uu)
        fl.fl_velocity_prescale(m.handle, dtype, dt, uu, w)
    x = torch.tensor(th, dtype=dtype, device="cuda")
    a, b = torch.empty_like(x), torch.empty_like(x)
    for _ in range(nsteps):
        if rk == 1:
            fl.fl_step_rk_stage(m.handle, lim, dtype, 1, 0, dt, None, x, a, uu, w)
            x, a = a, x
        else:
            fl.fl_step_rk_stage(m.handle, lim, dtype, 3, 0, dt, None, x, a, uu, w)
            fl.fl_step_rk_stage(m.handle, lim, dtype, 3, 1, dt, x, a, b, uu, w)
            fl.fl_step_rk_stage(m.handle, lim, dtype, 3, 2, dt, x, b, x, uu, w)
    m.close()
    assert torch.equal(got, x.cpu())


@pytest.mark.parametrize("name,world", [("hex", 3), ("tet", 2), ("prism", 4)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_renumbered_local_meshes_match_the_oracle(fl, name, world, dtype):
    # FL_RENUMBER on the local meshes: the interior and the rim in compact
    # blocks, the part's lists in the library's internal order; the cells then
    # sum their faces in another order, so the rollout equals the whole-mesh
    # oracle to rounding (1e-12 FP64, 1e-5 FP32 of max |theta|)
    import oracle
    mesh, th, u, dt = _case(name)
    got = _partitioned(fl, name, world, "smart", dtype, 3, 3, renumber=True).double().numpy()
    ref = oracle.step(mesh, "smart", 3, dt, 3, u, th)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("name,world", [("hex", 3), ("prism", 2)])
def test_renumbered_partitioned_gradient_matches_the_oracle(fl, name, world):
    # the reverse sweep on renumbered local meshes (internal order, cell
    # ranges of the interior and the rim) against the oracle's gradient
    import oracle
    mesh, th, u, dt = _case(name)
    tgt = np.random.default_rng(10).normal(size=mesh.n_cells)
    thT = oracle.step(mesh, "smart", 3, dt, 3, u, th)
    got = _partitioned(fl, name, world, "smart", torch.float64, 3, 3, grad=thT - tgt,
                       renumber=True).numpy()
    _, g_ref = oracle.gradient(mesh, "smart", 3, dt, 3, u, th, tgt)
    assert np.max(np.abs(got - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("name,world", [("hex", 3), ("tet", 2)])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1)])
def test_partitioned_gradient_matches_whole_mesh_and_oracle(fl, name, world, lim, rk):
    import oracle
    mesh, th, u, dt = _case(name)
    nsteps = 3
    tgt = np.random.default_rng(9).normal(size=mesh.n_cells)
    thT = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
    got = _partitioned(fl, name, world, lim, torch.float64, rk, nsteps, grad=thT - tgt).numpy()
    m = _whole_mesh(fl, mesh)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, rk, nsteps, 2)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty(mesh.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_step_rk_adjoint(m.handle, lim, torch.float64, rk, dt, nsteps, 2,
                          torch.tensor(th, device="cuda"), torch.tensor(u, device="cuda"),
                          torch.tensor(thT - tgt, device="cuda"), g, ws, nb)
    m.close()
    whole = g.cpu().numpy()
    assert np.max(np.abs(got - whole)) <= 1e-12 * np.max(np.abs(whole))
    _, g_ref = oracle.gradient(mesh, lim, rk, dt, nsteps, u, th, tgt)
    assert np.max(np.abs(got - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))


def _one_local(fl, name="hex", world=3, rank=1):
    from paper_2110_03044_gb300.partition import local_mesh_arrays
    mesh, th, u, dt = _case(name)
    part = partition_graph(mesh.n_cells, mesh.face_cells, world)
    gp = build_parts(mesh.n_cells, mesh.face_cells, part)[rank]
    C, n_o, n_i, fcl, nrm, ar, vol, dist = local_mesh_arrays(mesh, gp)
    m = fl.Mesh(fl.fl_mesh_create_local(C, n_o, n_i, fcl, nrm, ar, vol, dist))
    return mesh, th, u, dt, gp, m


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_stage_cells_compose_and_leave_other_cells(fl, dtype):
    mesh, th, u, dt, gp, m = _one_local(fl)
    assert fl.fl_mesh_local_info(m.handle) == (gp.n_owned, gp.n_interior)
    assert 0 < gp.n_interior < gp.n_owned < gp.n_cells
    x = gp.local_cells(torch.tensor(th, dtype=dtype, device="cuda")).contiguous()
    thn = (x * 0.5).contiguous()
    uu = gp.local_faces(torch.tensor(u, dtype=dtype, device="cuda")).contiguous()
    n_i, n_o = gp.n_interior, gp.n_owned
    for s in range(3):
        ref = torch.full_like(x, 9.5)
        fl.fl_step_rk_stage(m.handle, "superbee", dtype, 3, s, dt, thn, x, ref, uu)
        torch.cuda.synchronize()
        assert bool((ref[n_o:] == 9.5).all())  # no halo cell is written
        y = torch.full_like(x, 9.5)
        fl.fl_step_rk_stage_cells(m.handle, "superbee", dtype, 3, s, dt, 0, n_i, thn, x, y, uu)
        torch.cuda.synchronize()
        assert torch.equal(y[:n_i], ref[:n_i]) and bool((y[n_i:] == 9.5).all())
        fl.fl_step_rk_stage_cells(m.handle, "superbee", dtype, 3, s, dt, n_i, n_o, thn, x, y, uu)
        assert torch.equal(y, ref)
        mu = torch.sin(x * 3).contiguous()
        out_ref = torch.full_like(x, -2.0)
        fl.fl_step_rk_stage_adjoint(m.handle, "superbee", dtype, 3, s, dt, x, mu, thn, x,
                                    out_ref, uu)
        out = torch.full_like(x, -2.0)
        for c0, c1 in [(n_i, n_o), (0, n_i)]:
            fl.fl_step_rk_stage_adjoint_cells(m.handle, "superbee", dtype, 3, s, dt, c0, c1, x, mu,
                                              thn, x, out, uu)
        torch.cuda.synchronize()
        assert torch.equal(out, out_ref) and bool((out[n_o:] == -2.0).all())
    m.close()


def test_local_mesh_argument_errors_and_halo_pack(fl):
    mesh, th, u, dt, gp, m = _one_local(fl)
    x = gp.local_cells(torch.tensor(th, device="cuda")).contiguous()
    uu = gp.local_faces(torch.tensor(u, device="cuda")).contiguous()
    y = torch.zeros_like(x)
    for c0, c1 in [(1, gp.n_owned), (0, gp.n_cells), (gp.n_owned, gp.n_interior)]:
        with pytest.raises(fl.FLError) as e:
            fl.fl_step_rk_stage_cells(m.handle, "smart", torch.float64, 1, 0, dt, c0, c1, None, x,
                                      y, uu)
        assert e.value.status == fl.FL_EINVAL
    # the halo gather, then an index out of range: FL_EINDEX from the next call
    idx = torch.tensor([3, 0, gp.n_cells - 1, 7], dtype=torch.int32, device="cuda")
    buf = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    fl.fl_halo_pack(m.handle, torch.float64, x, idx, 4, buf)
    torch.cuda.synchronize()
    assert torch.equal(buf, x[idx.long()])
    bad = torch.tensor([1, gp.n_cells], dtype=torch.int32, device="cuda")
    buf2 = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    fl.fl_halo_pack(m.handle, torch.float64, x, bad, 2, buf2)
    torch.cuda.synchronize()
    assert float(buf2[0]) == float(x[1]) and float(buf2[1]) == -1.0
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk_stage_cells(m.handle, "smart", torch.float64, 1, 0, dt, 0, gp.n_owned, None,
                                  x, y, uu)
    assert e.value.status == fl.FL_EINDEX
    fl.fl_step_rk_stage_cells(m.handle, "smart", torch.float64, 1, 0, dt, 0, gp.n_owned, None, x,
                              y, uu)  # the latch was cleared
    m.close()
    with pytest.raises(fl.FLError) as e:  # n_interior > n_owned
        fl.fl_mesh_create_local(mesh.n_cells, 5, 6, mesh.face_cells, mesh.normals, mesh.areas,
                                mesh.volumes)
    assert e.value.status == fl.FL_EINVAL
    # a structured mesh takes planes, not cell ranges
    sm = fl.Mesh.structured(8, 8, 8, 0.1, 0.1, 0.1)
    xs = torch.zeros(512, dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk_stage_cells(sm.handle, "smart", torch.float64, 1, 0, dt, 0, 512, None, xs,
                                  torch.zeros_like(xs), torch.zeros(3 * 512, dtype=torch.float64,
                                                                    device="cuda"))
    assert e.value.status == fl.FL_EUNSUPPORTED
    sm.close()


def test_partitioned_mass_is_conserved(fl):
    # sum_c V_c theta_c over the ranks' owned cells (fl_reduce_mass on each
    # local mesh sums its owned cells) before and after a rollout
    import math
    mesh, th, u, dt = _case("tet")
    got = _partitioned(fl, "tet", 3, "superbee", torch.float64, 3, 5).numpy()
    m0 = math.fsum((th * mesh.volumes).tolist())
    assert abs(math.fsum((got * mesh.volumes).tolist()) - m0) <= 1e-13 * abs(m0)
    _, _, _, _, gp, m = _one_local(fl, "tet", 3, 0)
    x = gp.local_cells(torch.tensor(th, device="cuda")).contiguous()
    ws = torch.empty(max(fl.fl_reduce_workspace_size(), 1), dtype=torch.uint8, device="cuda")
    owned_mass = fl.fl_reduce_mass(m.handle, torch.float64, x, ws)
    want = math.fsum((th[gp.owned_ids] * mesh.volumes[gp.owned_ids]).tolist())
    assert abs(owned_mass - want) <= 1e-13 * abs(m0)
    m.close()
