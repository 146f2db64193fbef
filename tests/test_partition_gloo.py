"""The graph partition of face-based meshes and its two-ring halo exchange,
on the host: world_size 1, 2 and 3 gloo groups, with the oracle's stage and
adjoint on each rank's local face arrays as the per-rank computation (the
GPU runs the library's local meshes instead; see test_gpu_partition.py).

* The partition gives every cell one part, parts of the requested sizes;
  the first part (a breadth-first ball at every level) is connected.
* A part's halo is exactly the other parts' cells within two cells of an
  owned cell; its interior cells have no halo cell within two cells; its
  local faces are the faces of its owned and first-ring cells in ascending
  global id; send and receive lists pair up.
* A partitioned Euler / SSP-RK3 rollout (with and without overlap) gives,
  on every owned cell, the bits of the whole-mesh oracle (the local faces
  keep the whole mesh's relative order, so every cell sums its faces in the
  same order), on hexahedra, tetrahedra and prisms.
* The partitioned reverse sweep (two rings serve the adjoint as well) gives
  the whole-mesh oracle's gradient to 1e-13."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_2110_03044_gb300.decomp import gradient_rk, step_rk
from paper_2110_03044_gb300.partition import (GraphTransport, LocalGraphTransport, build_parts,
                                              cell_graph, local_mesh_arrays, partition_graph)

MESHES = {
    "hex": lambda: W.structured_mesh(9, 7, 6, 0.7 / 9, 0.9 / 7, 1.1 / 6),
    "tet": lambda: W.tet_mesh(4),
    "prism": lambda: W.prism_mesh(4),
    "tiny": lambda: W.structured_mesh(4, 3, 2, 0.25, 0.3, 0.5),
}


def _dist_from(ptr, nbr, sources, n):
    """Graph distance of every cell from the set ``sources`` (-1: unreached)."""
    d = np.full(n, -1, dtype=np.int64)
    frontier = list(sources)
    for s in frontier:
        d[s] = 0
    head = 0
    while head < len(frontier):
        c = frontier[head]
        head += 1
        for q in nbr[ptr[c]:ptr[c + 1]]:
            if d[q] < 0:
                d[q] = d[c] + 1
                frontier.append(int(q))
    return d


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partition_covers_and_balances(name, world):
    mesh = MESHES[name]()
    part = partition_graph(mesh.n_cells, mesh.face_cells, world)
    assert part.shape == (mesh.n_cells,) and part.min() >= 0 and part.max() < world
    sizes = np.bincount(part, minlength=world)
    # recursive shares: each split gives floor(n k1 / k) cells to its first side
    assert sizes.max() - sizes.min() <= world
    # the first side of every bisection is a breadth-first ball of the graph:
    # the part of rank 0 (first side all the way down) is connected
    ptr, nbr, _ = cell_graph(mesh.n_cells, mesh.face_cells)
    cells = np.flatnonzero(part == 0)
    member = part == 0
    seen = {int(cells[0])}
    stack = [int(cells[0])]
    while stack:
        c = stack.pop()
        for q in nbr[ptr[c]:ptr[c + 1]]:
            if member[q] and int(q) not in seen:
                seen.add(int(q))
                stack.append(int(q))
    assert len(seen) == cells.shape[0]


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("world", [1, 2, 3])
def test_local_parts_hold_the_two_ring_stencil(name, world):
    mesh = MESHES[name]()
    n = mesh.n_cells
    fc = np.asarray(mesh.face_cells, dtype=np.int64)
    part = partition_graph(n, fc, world)
    parts = build_parts(n, fc, part)
    ptr, nbr, _ = cell_graph(n, fc)
    owned_all = np.concatenate([p.owned_ids for p in parts])
    assert np.array_equal(np.sort(owned_all), np.arange(n))
    for gp in parts:
        own = np.zeros(n, dtype=bool)
        own[gp.owned_ids] = True
        assert np.array_equal(np.sort(gp.owned_ids), np.flatnonzero(part == gp.rank))
        d_own = _dist_from(ptr, nbr, gp.owned_ids, n)
        want_halo = np.flatnonzero((d_own >= 1) & (d_own <= 2))
        assert np.array_equal(np.sort(gp.halo_ids), want_halo)
        # halo grouped by owner part, ascending ids within a group
        owners = part[gp.halo_ids]
        assert (np.diff(owners) >= 0).all()
        for r in np.unique(owners):
            g = gp.halo_ids[owners == r]
            assert (np.diff(g) > 0).all()
        # interior: no non-owned cell within two cells
        if (~own).any():
            d_out = _dist_from(ptr, nbr, np.flatnonzero(~own), n)
            inner = gp.owned_ids[:gp.n_interior]
            rim = gp.owned_ids[gp.n_interior:]
            assert (d_out[inner] >= 3).all() and (d_out[rim] <= 2).all()
        else:
            assert gp.n_interior == gp.n_owned
        # local faces: faces of owned and first-ring cells, ascending
        ring1 = (d_own == 1)
        fmask = own[fc[:, 0]] | own[fc[:, 1]] | ring1[fc[:, 0]] | ring1[fc[:, 1]]
        assert np.array_equal(gp.face_ids, np.flatnonzero(fmask))
        assert np.array_equal(gp.cell_ids[gp.face_cells], fc[gp.face_ids])
    # send lists pair with receive lists, value by value
    for q in parts:
        for src, off, cnt in q.recv:
            sent = dict(parts[src].send)[q.rank]
            assert sent.shape == (cnt,)
            assert np.array_equal(parts[src].owned_ids[sent], q.halo_ids[off:off + cnt])


def _case(name):
    mesh = MESHES[name]()
    rng = np.random.default_rng(3)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 4)
    dt = 0.1 * float(np.min(mesh.volumes)) ** (1 / 3) / float(np.max(np.abs(u)))
    return mesh, th, u, dt


class _LocalOracle:
    """The oracle's stage and adjoint on a part's local face arrays, written
    into a local cell range only."""

    def __init__(self, mesh, gp, lim, rk, dt, u_local):
        C, n_o, n_i, fcl, nrm, ar, vol, dist = local_mesh_arrays(mesh, gp)
        lm = W.Mesh(n_cells=C, face_cells=fcl, normals=nrm, areas=ar, volumes=vol)
        self.om = oracle.OracleMesh(lm)
        self.lim, self.rk, self.dt = lim, rk, dt
        self.u = u_local.numpy()

    def stage(self, s, thn, x, y, c0, c1):
        xn = x.numpy()
        t = xn if thn is None else thn.numpy()
        full = oracle.stage(self.om, self.lim, self.rk, s, self.dt, t, xn, self.u)
        y[c0:c1] = torch.from_numpy(full[c0:c1])

    def stage_adjoint(self, s, x, mu, lam_a, lam_b, out, c0, c1):
        b = {0: 1.0, 1: 0.25, 2: 2.0 / 3.0}[s if self.rk == 3 else 0]
        m = mu.numpy()
        y = b * (m + self.dt * oracle.rhs_adjoint(self.om, self.lim, x.numpy(), self.u, m))
        if self.rk == 3 and s == 0:
            y = y + 0.75 * lam_a.numpy() + (1.0 / 3.0) * lam_b.numpy()
        out[c0:c1] = torch.from_numpy(y[c0:c1])


def _rank_run(name, rank, world, lim, rk, nsteps, transport, overlap, grad):
    mesh, th, u, dt = _case(name)
    part = partition_graph(mesh.n_cells, mesh.face_cells, world)
    gp = build_parts(mesh.n_cells, mesh.face_cells, part, world)[rank]
    lo = _LocalOracle(mesh, gp, lim, rk, dt, gp.local_faces(torch.from_numpy(u)))
    tl = gp.local_cells(torch.from_numpy(th)).clone()
    if grad:
        tgt = np.random.default_rng(7).normal(size=mesh.n_cells)
        thT = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
        lam = gp.local_cells(torch.from_numpy(thT - tgt)).clone()
        out = gradient_rk(gp, transport, lo.stage, lo.stage_adjoint, rk, nsteps, 2, tl, lam,
                          lambda: torch.full_like(tl, float("nan")), overlap=overlap)
    else:
        a = torch.full_like(tl, float("nan"))
        b = torch.full_like(tl, float("nan"))
        out = step_rk(gp, transport, lo.stage, rk, nsteps, tl, a, b, overlap=overlap)
    return gp.owned_ids.copy(), gp.owned(out).numpy().copy()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(name, rank, world, port, lim, rk, nsteps, overlap, grad, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _rank_run(name, rank, world, lim, rk, nsteps, GraphTransport(), overlap,
                                  grad))
    finally:
        dist.destroy_process_group()


def _gloo(name, world, lim, rk, nsteps, overlap=True, grad=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker,
                         args=(name, r, world, port, lim, rk, nsteps, overlap, grad, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    mesh = MESHES[name]()
    got = np.full(mesh.n_cells, np.nan)
    for _, ids, vals in out:
        got[ids] = vals
    return got


def test_one_part_runs_without_exchange():
    mesh, th, u, dt = _case("hex")
    ids, one = _rank_run("hex", 0, 1, "superbee", 3, 2, LocalGraphTransport(), True, False)
    got = np.empty(mesh.n_cells)
    got[ids] = one
    assert np.array_equal(got, oracle.step(mesh, "superbee", 3, dt, 2, u, th))


@pytest.mark.parametrize("name,world,overlap,lim,rk", [
    ("hex", 2, True, "superbee", 3), ("hex", 3, True, "smart", 3), ("hex", 2, False, "vanleer", 1),
    ("hex", 3, False, "superbee", 3), ("tet", 3, True, "smart", 3), ("tet", 2, True, "vanleer", 1),
    ("prism", 2, True, "superbee", 3), ("prism", 3, False, "smart", 3)])
def test_gloo_partitioned_rollout_equals_whole_mesh_oracle(name, world, overlap, lim, rk):
    mesh, th, u, dt = _case(name)
    got = _gloo(name, world, lim, rk, 3, overlap)
    ref = oracle.step(mesh, lim, rk, dt, 3, u, th)
    assert np.array_equal(got, ref)  # bit for bit


@pytest.mark.parametrize("name,world", [("hex", 2), ("tet", 3)])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1)])
def test_gloo_partitioned_gradient_equals_whole_mesh_oracle(name, world, lim, rk):
    mesh, th, u, dt = _case(name)
    got = _gloo(name, world, lim, rk, 3, grad=True)
    tgt = np.random.default_rng(7).normal(size=mesh.n_cells)
    _, g_ref = oracle.gradient(mesh, lim, rk, dt, 3, u, th, tgt)
    assert np.max(np.abs(got - g_ref)) <= 1e-13 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("name", ["hex", "tet"])
def test_reordered_part_follows_an_internal_order(name):
    # a renumbered local mesh permutes the interior and the rim among
    # themselves and keeps the halo: the part's lists follow that order and
    # still name the same global cells, faces and exchange values
    mesh = MESHES[name]()
    fc = np.asarray(mesh.face_cells, dtype=np.int64)
    part = partition_graph(mesh.n_cells, fc, 3)
    parts = build_parts(mesh.n_cells, fc, part)
    rng = np.random.default_rng(11)
    new = []
    for gp in parts:
        n_i, n_o, C = gp.n_interior, gp.n_owned, gp.n_cells
        cp = np.concatenate([rng.permutation(n_i), n_i + rng.permutation(n_o - n_i),
                             np.arange(n_o, C)])
        fp = rng.permutation(gp.face_ids.shape[0])
        r = gp.reordered(cp, fp)
        # the cell at internal index cp[i] is the cell at local index i
        assert np.array_equal(r.owned_ids[cp[:n_o]], gp.owned_ids)
        assert np.array_equal(r.face_ids[fp], gp.face_ids)
        assert np.array_equal(r.cell_ids[r.face_cells], fc[r.face_ids])
        assert np.array_equal(np.sort(r.owned_ids[:n_i]), np.sort(gp.owned_ids[:n_i]))
        new.append(r)
        with pytest.raises(ValueError):  # the halo must stay in place
            bad = cp.copy()
            if C > n_o + 1:
                bad[[n_o, n_o + 1]] = bad[[n_o + 1, n_o]]
                gp.reordered(bad, fp)
            else:
                raise ValueError
    for q in new:
        for src, off, cnt in q.recv:
            sent = dict(new[src].send)[q.rank]
            assert np.array_equal(new[src].owned_ids[sent], q.halo_ids[off:off + cnt])


def test_more_ranks_than_cells_gives_empty_parts():
    # 24 cells over 30 ranks: six ranks own nothing and hold no halo; every
    # other part is one cell, all rim (no interior), its halo two rings deep
    mesh = MESHES["tiny"]()
    fc = np.asarray(mesh.face_cells, dtype=np.int64)
    part = partition_graph(mesh.n_cells, fc, 30)
    parts = build_parts(mesh.n_cells, fc, part, 30)
    assert len(parts) == 30
    sizes = [p.n_owned for p in parts]
    assert sorted(sizes) == [0] * 6 + [1] * 24
    for gp in parts:
        if gp.n_owned == 0:
            assert gp.n_cells == 0 and gp.face_ids.shape == (0,) and not gp.send and not gp.recv
            assert gp.split() == (None, [(0, 0)], (0, 0))
        else:
            assert gp.n_interior == 0 and gp.split()[0] is None
    # trailing empty ranks are kept when the world is given
    assert len(build_parts(mesh.n_cells, fc, np.zeros(mesh.n_cells, np.int32), 3)) == 3


@pytest.mark.parametrize("world", [7, 30])
def test_gloo_tiny_parts_equal_whole_mesh_oracle(world):
    # parts of a few cells (no interior) and empty parts: the exchange-first
    # path, and ranks that only pass messages on
    mesh, th, u, dt = _case("tiny")
    got = _gloo("tiny", world, "superbee", 3, 2)
    assert np.array_equal(got, oracle.step(mesh, "superbee", 3, dt, 2, u, th))
