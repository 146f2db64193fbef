"""The z-slab domain decomposition and its per-stage halo exchange, on the
host: world_size 1, 2 and 3 gloo groups, with the oracle's stage as the
per-rank computation (the GPU runs the library's stage kernel instead; see
test_gpu_decomp.py).

* The slabs cover the planes once, each owning at least the halo depth.
* A stage runs every owned plane once and no ghost plane: with overlap, the
  planes two or more planes from both cuts between starting the exchange and
  waiting for it, the planes next to the cuts after.
* A decomposed SSP-RK3 / Euler rollout, with and without overlap, gives on
  every owned plane the bits of the one-rank decomposed run (the exchange
  delivers exactly the planes each stage reads; scratch planes no stage
  writes hold NaN) and the whole-mesh oracle to rounding (the cell sums of
  the wrapped plane 0 run in another face order there).
* Mass is conserved across the cuts to round-off.
* The decomposed reverse sweep (checkpoints, recomputed segments, the
  adjoint's halo exchanged before every adjoint stage, three ghost planes)
  gives the one-rank sweep's gradient bit for bit and the oracle's reference
  gradient to 1e-12."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_2110_03044_gb300.decomp import HALO, LocalTransport, Slab, TorchTransport, step_rk


@pytest.mark.parametrize("nz,world", [(24, 1), (24, 2), (25, 3), (9, 4), (4, 2)])
def test_slabs_cover_every_plane_once(nz, world):
    dims = (5, 3, nz)
    owned = []
    for r in range(world):
        s = Slab(dims, r, world)
        assert s.nz_local >= HALO
        assert s.local_dims == (5, 3, s.nz_local + 2 * HALO)
        assert s.down == (r - 1) % world and s.up == (r + 1) % world
        gp = s.global_planes()
        assert gp[HALO:HALO + s.nz_local] == list(range(s.lo, s.hi))
        assert gp[:HALO] == [(s.lo - HALO + k) % nz for k in range(HALO)]
        owned += list(range(s.lo, s.hi))
    assert owned == list(range(nz))


def test_slab_refuses_too_thin_slabs():
    with pytest.raises(ValueError):
        Slab((4, 4, 5), 0, 3)  # 5 planes over 3 ranks: a slab of 1 < halo
    with pytest.raises(ValueError):
        Slab((4, 4, 1), 0, 1)


def test_local_fields_cut_from_global():
    dims = (4, 3, 10)
    s = Slab(dims, 1, 2)
    g = torch.arange(4 * 3 * 10, dtype=torch.float64)
    loc = s.local_cells(g)
    P = 12
    assert torch.equal(s.owned(loc), g[5 * P:10 * P])
    assert torch.equal(loc[:P], g[3 * P:4 * P])          # ghost plane 3
    assert torch.equal(loc[-P:], g[1 * P:2 * P])         # ghost plane 11 -> 1
    u = torch.arange(3 * 120, dtype=torch.float64)
    lu = s.local_faces(u, 3)
    assert lu.numel() == 3 * loc.numel()
    assert torch.equal(lu[loc.numel():loc.numel() + P], u[120 + 3 * P:120 + 4 * P])


class _Recorder:
    """A transport that only records the order of its calls."""

    def __init__(self):
        self.log = []

    def exchange(self, slab, x):
        self.log.append("exchange")

    def start(self, slab, x):
        self.log.append("start")
        log = self.log

        class Pending:
            def wait(self):
                log.append("wait")

        return Pending()


@pytest.mark.parametrize("nz,world,overlap", [(16, 2, True), (16, 2, False), (8, 2, True),
                                              (9, 2, True), (5, 1, True), (4, 1, True)])
def test_exchange_and_run_covers_owned_planes_once(nz, world, overlap):
    from paper_2110_03044_gb300.decomp import REACH, exchange_and_run
    slab = Slab((3, 2, nz), 0, world)
    tr = _Recorder()
    exchange_and_run(slab, tr, None, lambda z0, z1: tr.log.append((z0, z1)), overlap)
    h, n = slab.halo, slab.nz_local
    ranges = [e for e in tr.log if isinstance(e, tuple)]
    planes = sorted(k for z0, z1 in ranges for k in range(z0, z1))
    assert planes == list(range(h, h + n))  # every owned plane once, no ghost plane
    if overlap and n > 2 * REACH:
        assert tr.log == ["start", (h + REACH, h + n - REACH), "wait", (h, h + REACH),
                          (h + n - REACH, h + n)]
    else:
        assert tr.log == ["exchange", (h, h + n)]


def _case():
    dims = (9, 7, 12)
    h = (0.7 / 9, 0.9 / 7, 1.1 / 12)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(3)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 4)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    return dims, h, mesh, th, u, dt


def _oracle_stage(slab, h, lim, rk, dt, u_local):
    """The oracle's stage on the local mesh, written into local planes
    [z0, z1) of y only (the other planes of y keep their values)."""
    lm = oracle.OracleMesh(W.structured_mesh(*slab.local_dims, *h))
    uu = u_local.numpy()
    P = slab.plane

    def stage(s, thn, x, y, z0, z1):
        xn = x.numpy()
        t = xn if thn is None else thn.numpy()
        full = oracle.stage(lm, lim, rk, s, dt, t, xn, uu)
        y[z0 * P:z1 * P] = torch.from_numpy(full[z0 * P:z1 * P])

    return stage


def _run_rank(rank, world, lim, rk, nsteps, transport, overlap=True):
    dims, h, mesh, th, u, dt = _case()
    slab = Slab(dims, rank, world)
    tl = slab.local_cells(torch.from_numpy(th)).clone()
    ul = slab.local_faces(torch.from_numpy(u), 3)
    # scratch full of NaN: a plane the stages never write must never be read
    a = torch.full_like(tl, float("nan"))
    b = torch.full_like(tl, float("nan"))
    step_rk(slab, transport, _oracle_stage(slab, h, lim, rk, dt, ul), rk, nsteps, tl, a, b,
            overlap=overlap)
    return slab.lo, slab.hi, slab.owned(tl).numpy().copy()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, lim, rk, nsteps, overlap, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _run_rank(rank, world, lim, rk, nsteps, TorchTransport(), overlap))
    finally:
        dist.destroy_process_group()


def _gloo_run(world, lim, rk, nsteps, overlap=True):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, lim, rk, nsteps, overlap, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return sorted(out)


@pytest.mark.parametrize("world,overlap", [(2, True), (3, True), (2, False)])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1), ("smart", 3)])
def test_gloo_decomposed_rollout_equals_one_rank(world, overlap, lim, rk):
    dims, h, mesh, th, u, dt = _case()
    nsteps = 3
    P = dims[0] * dims[1]
    # the one-rank decomposed run (its halo comes from itself)
    lo, hi, one = _run_rank(0, 1, lim, rk, nsteps, LocalTransport(), overlap=False)
    assert (lo, hi) == (0, dims[2])
    got = np.empty(mesh.n_cells)
    for _, lo, hi, part in _gloo_run(world, lim, rk, nsteps, overlap):
        got[lo * P:hi * P] = part
    assert np.array_equal(got, one)  # bit for bit
    ref = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    m0 = math.fsum((th * mesh.volumes).tolist())
    assert abs(math.fsum((got * mesh.volumes).tolist()) - m0) <= 1e-13 * abs(m0)


# ------------------------------------------------ the decomposed reverse sweep
def _oracle_stage_adjoint(slab, h, lim, rk, dt, u_local):
    lm = oracle.OracleMesh(W.structured_mesh(*slab.local_dims, *h))
    uu = u_local.numpy()
    b = {0: 1.0, 1: 0.25, 2: 2.0 / 3.0}
    P = slab.plane

    def stage_adjoint(s, x, mu, lam_a, lam_b, out, z0, z1):
        m = mu.numpy()
        y = b[s if rk == 3 else 0] * (m + dt * oracle.rhs_adjoint(lm, lim, x.numpy(), uu, m))
        if rk == 3 and s == 0:
            y = y + 0.75 * lam_a.numpy() + (1.0 / 3.0) * lam_b.numpy()
        out[z0 * P:z1 * P] = torch.from_numpy(y[z0 * P:z1 * P])

    return stage_adjoint


def _grad_rank(rank, world, lim, rk, nsteps, every, transport, overlap=True):
    from paper_2110_03044_gb300.decomp import HALO_ADJOINT, gradient_rk
    dims, h, mesh, th, u, dt = _case()
    tgt = np.random.default_rng(7).normal(size=mesh.n_cells)
    thT = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
    slab = Slab(dims, rank, world, halo=HALO_ADJOINT)
    tl = slab.local_cells(torch.from_numpy(th)).clone()
    lam = slab.local_cells(torch.from_numpy(thT - tgt)).clone()
    ul = slab.local_faces(torch.from_numpy(u), 3)
    g = gradient_rk(slab, transport, _oracle_stage(slab, h, lim, rk, dt, ul),
                    _oracle_stage_adjoint(slab, h, lim, rk, dt, ul), rk, nsteps, every, tl, lam,
                    lambda: torch.full_like(tl, float("nan")), overlap=overlap)
    return slab.lo, slab.hi, slab.owned(g).numpy().copy()


def _grad_worker(rank, world, port, lim, rk, nsteps, every, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _grad_rank(rank, world, lim, rk, nsteps, every, TorchTransport()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1)])
def test_gloo_decomposed_gradient_equals_one_rank(world, lim, rk):
    dims, h, mesh, th, u, dt = _case()
    nsteps, every = 3, 2
    P = dims[0] * dims[1]
    _, _, one = _grad_rank(0, 1, lim, rk, nsteps, every, LocalTransport(), overlap=False)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, world, port, lim, rk, nsteps, every, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = np.empty(mesh.n_cells)
    for _, lo, hi, part in out:
        got[lo * P:hi * P] = part
    assert np.array_equal(got, one)  # bit for bit
    tgt = np.random.default_rng(7).normal(size=mesh.n_cells)
    _, g_ref = oracle.gradient(mesh, lim, rk, dt, nsteps, u, th, tgt)
    assert np.max(np.abs(got - g_ref)) <= 1e-12 * np.max(np.abs(g_ref))


# ------------------------------------------------------------------ pencils
@pytest.mark.parametrize("grid", [(1, 1), (2, 2), (3, 1), (1, 3), (2, 3)])
def test_pencils_tile_the_box_and_pair_their_messages(grid):
    from paper_2110_03044_gb300.decomp import Pencil, PencilTransport
    dims = (5, 9, 12)
    py, pz = grid
    pcs = [Pencil(dims, r, grid) for r in range(py * pz)]
    owner = np.full(dims[0] * dims[1] * dims[2], -1)
    for pc in pcs:
        ids = pc._local_ids().reshape(pc.nzl + 2 * pc.halo, pc.nyl + 2 * pc.halo, dims[0])
        own = ids[pc.halo:pc.halo + pc.nzl, pc.halo:pc.halo + pc.nyl].ravel()
        assert (owner[own] == -1).all()
        owner[own] = pc.rank
    assert (owner >= 0).all()
    # a message's two ends name the same global cells in the same order
    for pc in pcs:
        send, recv = pc.exchange_lists()
        gid = pc._local_ids()
        peer = {"y_down": pc.y_down, "y_up": pc.y_up, "z_down": pc.z_down, "z_up": pc.z_up}
        for d, idx in recv.items():
            q = pcs[peer[d]]
            sent = q.exchange_lists()[0][PencilTransport.OPP[d]]
            assert np.array_equal(q._local_ids()[sent], gid[idx])
        # the ghost cells filled are exactly the side halos of the owned box
        h = pc.halo
        n_side = h * dims[0] * (pc.nyl + pc.nzl) * 2
        assert sum(v.shape[0] for v in recv.values()) == n_side
    interior, rims, whole = pcs[-1].split()
    cells = lambda b: (b[1] - b[0]) * (b[3] - b[2])  # noqa: E731
    if interior is not None:
        assert cells(interior) + sum(cells(r) for r in rims) == cells(whole)


def _pencil_rank(rank, grid, lim, rk, nsteps, transport, overlap=True, grad=False):
    from paper_2110_03044_gb300.decomp import HALO_ADJOINT, Pencil
    dims, h, mesh, th, u, dt = _case()
    pc = Pencil(dims, rank, grid, halo=HALO_ADJOINT if grad else 2)
    lm = oracle.OracleMesh(W.structured_mesh(*pc.local_dims, *h))
    ul = pc.local_faces(torch.from_numpy(u), 3).numpy()
    nx, nyl2 = dims[0], pc.nyl + 2 * pc.halo

    def box(y, y0, y1, z0, z1):
        return y.view(-1, nyl2, nx)[z0:z1, y0:y1, :]

    def stage(s, thn, x, y, y0, y1, z0, z1):
        xn = x.numpy()
        t = xn if thn is None else thn.numpy()
        full = torch.from_numpy(oracle.stage(lm, lim, rk, s, dt, t, xn, ul))
        box(y, y0, y1, z0, z1).copy_(box(full, y0, y1, z0, z1))

    bs = {0: 1.0, 1: 0.25, 2: 2.0 / 3.0}

    def stage_adjoint(s, x, mu, lam_a, lam_b, out, y0, y1, z0, z1):
        m = mu.numpy()
        yv = bs[s if rk == 3 else 0] * (m + dt * oracle.rhs_adjoint(lm, lim, x.numpy(), ul, m))
        if rk == 3 and s == 0:
            yv = yv + 0.75 * lam_a.numpy() + (1.0 / 3.0) * lam_b.numpy()
        box(out, y0, y1, z0, z1).copy_(box(torch.from_numpy(yv), y0, y1, z0, z1))

    tl = pc.local_cells(torch.from_numpy(th)).clone()
    # scratch: a huge finite sentinel rather than NaN.  The pencil's corner
    # ghost cells (ghost rows of ghost planes) are never exchanged: the
    # stencil never reads them, but the oracle's upstream sum runs over all
    # other faces of the upwind cell, orthogonal ones with weight 0, and
    # 0 x NaN would be NaN; 0 x 1e200 is 0, and any weighted read of an
    # unwritten cell still blows up
    nan = lambda: torch.full_like(tl, 1e200)  # noqa: E731
    if grad:
        from paper_2110_03044_gb300.decomp import gradient_rk
        tgt = np.random.default_rng(7).normal(size=mesh.n_cells)
        thT = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
        lam = pc.local_cells(torch.from_numpy(thT - tgt)).clone()
        out = gradient_rk(pc, transport, stage, stage_adjoint, rk, nsteps, 2, tl, lam, nan,
                          overlap=overlap)
    else:
        out = step_rk(pc, transport, stage, rk, nsteps, tl, nan(), nan(), overlap=overlap)
    ids = pc._local_ids().reshape(pc.nzl + 2 * pc.halo, nyl2, nx)
    own = ids[pc.halo:pc.halo + pc.nzl, pc.halo:pc.halo + pc.nyl].ravel()
    return own, pc.owned(out).reshape(-1).numpy().copy()


def _pencil_worker(rank, grid, port, lim, rk, nsteps, overlap, grad, q):
    import torch.distributed as dist

    from paper_2110_03044_gb300.decomp import PencilTransport
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=grid[0] * grid[1])
    try:
        q.put((rank,) + _pencil_rank(rank, grid, lim, rk, nsteps, PencilTransport(), overlap,
                                     grad))
    finally:
        dist.destroy_process_group()


def _pencil_gloo(grid, lim, rk, nsteps, overlap=True, grad=False):
    world = grid[0] * grid[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_pencil_worker,
                         args=(r, grid, port, lim, rk, nsteps, overlap, grad, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    dims = _case()[0]
    got = np.full(dims[0] * dims[1] * dims[2], np.nan)
    for _, ids, vals in out:
        got[ids] = vals
    return got


@pytest.mark.parametrize("grid,overlap", [((2, 2), True), ((3, 2), True), ((2, 1), False)])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1)])
def test_gloo_pencil_rollout_equals_one_rank(grid, overlap, lim, rk):
    from paper_2110_03044_gb300.decomp import PencilTransport
    dims, h, mesh, th, u, dt = _case()
    own, vals = _pencil_rank(0, (1, 1), lim, rk, 3, PencilTransport(), overlap=False)
    one = np.empty(mesh.n_cells)
    one[own] = vals
    got = _pencil_gloo(grid, lim, rk, 3, overlap)
    assert np.array_equal(got, one)  # bit for bit
    ref = oracle.step(mesh, lim, rk, dt, 3, u, th)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1)])
def test_gloo_pencil_gradient_equals_one_rank(lim, rk):
    from paper_2110_03044_gb300.decomp import PencilTransport
    dims, h, mesh, th, u, dt = _case()
    own, vals = _pencil_rank(0, (1, 1), lim, rk, 3, PencilTransport(), overlap=False, grad=True)
    one = np.empty(mesh.n_cells)
    one[own] = vals
    got = _pencil_gloo((2, 2), lim, rk, 3, grad=True)
    assert np.array_equal(got, one)  # bit for bit
    tgt = np.random.default_rng(7).normal(size=mesh.n_cells)
    _, g_ref = oracle.gradient(mesh, lim, rk, dt, 3, u, th, tgt)
    assert np.max(np.abs(got - g_ref)) <= 1e-12 * np.max(np.abs(g_ref))


def test_tall_pencil_rims_are_tile_tall():
    # a pencil of more than 32 rows keeps 8-row bands (whole stage tiles)
    from paper_2110_03044_gb300.decomp import Pencil
    pc = Pencil((8, 80, 20), 0, (1, 1))
    interior, rims, whole = pc.split()
    h = pc.halo
    assert interior == (h + 8, h + 72, h + 2, h + 18)
    cells = lambda b: (b[1] - b[0]) * (b[3] - b[2])  # noqa: E731
    assert cells(interior) + sum(cells(r) for r in rims) == cells(whole)
    covered = np.zeros((20 + 2 * h, 80 + 2 * h), dtype=int)
    for y0, y1, z0, z1 in [interior] + rims:
        covered[z0:z1, y0:y1] += 1
    assert (covered[h:h + 20, h:h + 80] == 1).all() and covered.sum() == 80 * 20
