"""The z-slab decomposition on the GPU: W ranks emulated in one process on one
GPU, each a host thread with its own local mesh, running the library's stage
kernel (fl_step_rk_stage) through the same step_rk loop the multi-GPU run
uses.  The exchange copies ghost planes between the ranks' device buffers
after a host barrier; every launch and copy goes to the one default stream,
in order, so no kernel waits on another.

The owned planes of the decomposed rollout must equal fl_step_rk on the
whole mesh bit for bit: FP64 (with the pre-scaled velocity, the arithmetic of
fl_step_rk), FP32 on the register tile and on the TMA kernel, Euler and
SSP-RK3.  The decomposed reverse sweep (fl_step_rk_stage_adjoint, three ghost
planes, the adjoint's halo exchanged before every adjoint stage) must give the
one-slab sweep's gradient bit for bit, and fl_step_rk_adjoint's and the
oracle's gradient to rounding."""
import threading

import numpy as np
import pytest
import torch

import workloads as W
from paper_2110_03044_gb300.decomp import Slab, SlabRollout

pytestmark = pytest.mark.gpu


class ThreadGroupTransport:
    """Exchange among W host threads sharing one GPU: the ghost planes of each
    rank are copied from its neighbours' owned planes between two barriers."""

    def __init__(self, world):
        self.world = world
        self.fields = [None] * world
        self.bar = threading.Barrier(world)

    def exchange(self, slab, x):
        P, h, n = slab.plane, slab.halo, slab.nz_local
        self.fields[slab.rank] = (slab, x)
        self.bar.wait()  # every rank's stage input is enqueued and registered
        sd, xd = self.fields[slab.down]
        su, xu = self.fields[slab.up]
        x[0:h * P].copy_(xd[sd.nz_local * P:(sd.nz_local + h) * P])
        x[(h + n) * P:(2 * h + n) * P].copy_(xu[h * P:2 * h * P])
        self.bar.wait()  # every copy is enqueued before any rank's next stage


def _decomposed(fl, world, dims, h, th, u, lim, dtype, rk, dt, nsteps):
    out = [None] * world
    err = []
    tr = ThreadGroupTransport(world)
    ug = torch.tensor(u, device="cuda")

    def rank(r):
        try:
            torch.cuda.set_device(0)
            slab = Slab(dims, r, world)
            ro = SlabRollout(slab, h, ug, lim, dtype, dt, transport=tr)
            tl = ro.local_field(torch.tensor(th, device="cuda"))
            ro.step(tl, rk, nsteps)
            torch.cuda.synchronize()
            out[r] = (slab.lo, slab.hi, slab.owned(tl).cpu())
            ro.close()
        except BaseException as e:  # noqa: BLE001 -- reported below
            err.append(e)
            tr.bar.abort()

    ts = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if err:
        raise err[0]
    P = dims[0] * dims[1]
    got = torch.empty(P * dims[2], dtype=dtype)
    for lo, hi, part in out:
        got[lo * P:hi * P] = part
    return got


@pytest.mark.parametrize("world", [1, 2, 3, 4])
@pytest.mark.parametrize("dims,dtype", [((40, 12, 24), torch.float64),
                                        ((40, 12, 24), torch.float32),
                                        ((128, 8, 20), torch.float32)])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1), ("smart", 3)])
def test_decomposed_rollout_equals_whole_mesh_bitwise(fl, world, dims, dtype, lim, rk):
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(5)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 6)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    nsteps = 3
    got = _decomposed(fl, world, dims, h, th, u, lim, dtype, rk, dt, nsteps)
    m = fl.Mesh.structured(*dims, *h)
    ref = torch.tensor(th, dtype=dtype, device="cuda")
    fl.step_rk(m, lim, ref, torch.tensor(u, dtype=dtype, device="cuda"), dt, nsteps,
               rk_order=rk)
    m.close()
    assert torch.equal(got, ref.cpu())


def test_stage_entry_point_composes_to_step_rk(fl):
    # three fl_step_rk_stage calls (FP64, pre-scaled velocity) give the bits
    # of one fl_step_rk SSP-RK3 step; without w_f the FP64 stage forms the
    # flux per face and agrees to rounding
    dims = (33, 10, 7)
    h = (0.1, 0.2, 0.3)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(8)
    th0 = torch.tensor(rng.uniform(-1, 1, mesh.n_cells), device="cuda")
    u = torch.tensor(0.3 * W.mixed_sign_velocity(mesh.n_faces, 9), device="cuda")
    dt = 0.05
    m = fl.Mesh.structured(*dims, *h)
    ref = th0.clone()
    fl.step_rk(m, "smart", ref, u, dt, 1, rk_order=3)
    for w in (torch.empty_like(u), None):
        if w is not None:
            fl.fl_velocity_prescale(m.handle, torch.float64, dt, u, w)
        th = th0.clone()
        a, b = torch.empty_like(th), torch.empty_like(th)
        fl.fl_step_rk_stage(m.handle, "smart", torch.float64, 3, 0, dt, None, th, a, u, w)
        fl.fl_step_rk_stage(m.handle, "smart", torch.float64, 3, 1, dt, th, a, b, u, w)
        fl.fl_step_rk_stage(m.handle, "smart", torch.float64, 3, 2, dt, th, b, th, u, w)
        if w is not None:
            assert torch.equal(th, ref)
        else:
            assert float((th - ref).abs().max() / ref.abs().max()) <= 1e-14
    with pytest.raises(fl.FLError) as e:  # y must not overlap x
        fl.fl_step_rk_stage(m.handle, "smart", torch.float64, 3, 0, dt, None, th, th, u, None)
    assert e.value.status == fl.FL_EINVAL
    with pytest.raises(fl.FLError):  # no stage 1 in forward Euler
        fl.fl_step_rk_stage(m.handle, "smart", torch.float64, 1, 1, dt, th, a, b, u, None)
    m.close()


def _decomposed_gradient(fl, world, dims, h, th, u, lam_T, lim, rk, dt, nsteps, every,
                         dtype=torch.float64):
    from paper_2110_03044_gb300.decomp import HALO_ADJOINT
    out = [None] * world
    err = []
    tr = ThreadGroupTransport(world)
    ug = torch.tensor(u, device="cuda")

    def rank(r):
        try:
            torch.cuda.set_device(0)
            slab = Slab(dims, r, world, halo=HALO_ADJOINT)
            ro = SlabRollout(slab, h, ug, lim, dtype, dt, transport=tr)
            tl = ro.local_field(torch.tensor(th, device="cuda"))
            ll = ro.local_field(torch.tensor(lam_T, device="cuda"))
            g = ro.gradient(tl, ll, rk, nsteps, every)
            torch.cuda.synchronize()
            out[r] = (slab.lo, slab.hi, slab.owned(g).cpu())
            ro.close()
        except BaseException as e:  # noqa: BLE001 -- reported below
            err.append(e)
            tr.bar.abort()

    ts = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if err:
        raise err[0]
    P = dims[0] * dims[1]
    got = torch.empty(P * dims[2], dtype=torch.float64)
    for lo, hi, part in out:
        got[lo * P:hi * P] = part
    return got.numpy()


@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 3), ("smart", 1)])
def test_decomposed_gradient_matches_whole_mesh_and_oracle(fl, lim, rk):
    # the reverse sweep on 3 slabs (three ghost planes, the adjoint's halo
    # exchanged before every adjoint stage): bit for bit the one-slab sweep,
    # and fl_step_rk_adjoint on the whole mesh and the oracle's gradient to
    # rounding
    import oracle
    dims = (24, 10, 18)
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(15)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 16)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    nsteps, every = 4, 3
    tgt = rng.normal(size=mesh.n_cells)
    thT = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
    got = _decomposed_gradient(fl, 3, dims, h, th, u, thT - tgt, lim, rk, dt, nsteps, every)
    one = _decomposed_gradient(fl, 1, dims, h, th, u, thT - tgt, lim, rk, dt, nsteps, every)
    assert np.array_equal(got, one)
    m = fl.Mesh.structured(*dims, *h)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, rk, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty(mesh.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_step_rk_adjoint(m.handle, lim, torch.float64, rk, dt, nsteps, every,
                          torch.tensor(th, device="cuda"), torch.tensor(u, device="cuda"),
                          torch.tensor(thT - tgt, device="cuda"), g, ws, nb)
    m.close()
    whole = g.cpu().numpy()
    scale = np.max(np.abs(whole))
    assert np.max(np.abs(got - whole)) <= 1e-12 * scale
    _, g_ref = oracle.gradient(mesh, lim, rk, dt, nsteps, u, th, tgt)
    assert np.max(np.abs(got - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))


def test_stage_adjoint_composes_to_the_step_adjoint(fl):
    # one SSP-RK3 step back through fl_step_rk_stage_adjoint equals
    # fl_step_rk_adjoint over one step (stage states from fl_step_rk_stage)
    dims = (33, 10, 7)
    h = (0.1, 0.2, 0.3)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(18)
    th0 = torch.tensor(rng.uniform(-1, 1, mesh.n_cells), device="cuda")
    u = torch.tensor(0.3 * W.mixed_sign_velocity(mesh.n_faces, 19), device="cuda")
    lam = torch.tensor(rng.normal(size=mesh.n_cells), device="cuda")
    dt = 0.05
    m = fl.Mesh.structured(*dims, *h)
    w = torch.empty_like(u)
    fl.fl_velocity_prescale(m.handle, torch.float64, dt, u, w)
    x1, x2, y = torch.empty_like(th0), torch.empty_like(th0), torch.empty_like(th0)
    f64 = torch.float64
    fl.fl_step_rk_stage(m.handle, "superbee", f64, 3, 0, dt, None, th0, x1, u, w)
    fl.fl_step_rk_stage(m.handle, "superbee", f64, 3, 1, dt, th0, x1, x2, u, w)
    m2, m1, out = torch.empty_like(th0), torch.empty_like(th0), torch.empty_like(th0)
    fl.fl_step_rk_stage_adjoint(m.handle, "superbee", f64, 3, 2, dt, x2, lam, None, None, m2, u, w)
    fl.fl_step_rk_stage_adjoint(m.handle, "superbee", f64, 3, 1, dt, x1, m2, None, None, m1, u, w)
    fl.fl_step_rk_stage_adjoint(m.handle, "superbee", f64, 3, 0, dt, th0, m1, m2, lam, out, u, w)
    nb = fl.fl_adjoint_workspace_size(m.handle, f64, 3, 1, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    ref = torch.empty_like(th0)
    fl.fl_step_rk_adjoint(m.handle, "superbee", f64, 3, dt, 1, 1, th0, u, lam, ref, ws, nb)
    assert float((out - ref).abs().max() / ref.abs().max()) <= 1e-14
    with pytest.raises(fl.FLError):  # out must not overlap mu
        fl.fl_step_rk_stage_adjoint(m.handle, "superbee", f64, 3, 1, dt, x1, m2, None, None, m2,
                                    u, w)
    m.close()


# ------------------------------------------------ plane-range stage kernels
@pytest.mark.parametrize("dims,dtype,pre", [((40, 12, 23), torch.float64, True),
                                            ((40, 12, 23), torch.float64, False),
                                            ((40, 12, 23), torch.float32, False),
                                            ((128, 8, 21), torch.float32, False)])
@pytest.mark.parametrize("lim", ["superbee", "vanleer", "smart"])
def test_stage_planes_compose_to_the_whole_stage(fl, dims, dtype, pre, lim):
    # the stage over three plane ranges (one of them a single plane, one at
    # each periodic end) gives the whole stage's bits on every plane it
    # covers and leaves every other plane of y as it was
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(21)
    P, nz = dims[0] * dims[1], dims[2]
    th0 = torch.tensor(rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3),
                       dtype=dtype, device="cuda")
    thn = torch.tensor(rng.uniform(-1, 1, mesh.n_cells), dtype=dtype, device="cuda")
    u = torch.tensor(0.3 * W.mixed_sign_velocity(mesh.n_faces, 22), dtype=dtype, device="cuda")
    dt = 0.3 * min(h) / float(u.abs().max()) / 3
    m = fl.Mesh.structured(*dims, *h)
    w = None
    if pre:
        w = torch.empty_like(u)
        fl.fl_velocity_prescale(m.handle, dtype, dt, u, w)
    for s in range(3):
        ref = torch.empty_like(th0)
        fl.fl_step_rk_stage(m.handle, lim, dtype, 3, s, dt, thn, th0, ref, u, w)
        sentinel = torch.full_like(th0, 7.25)
        for z0, z1 in [(0, 1), (5, 9), (nz - 3, nz)]:
            y = sentinel.clone()
            fl.fl_step_rk_stage_planes(m.handle, lim, dtype, 3, s, dt, z0, z1, thn, th0, y, u, w)
            torch.cuda.synchronize()
            assert torch.equal(y[z0 * P:z1 * P], ref[z0 * P:z1 * P])
            assert torch.equal(y[:z0 * P], sentinel[:z0 * P])
            assert torch.equal(y[z1 * P:], sentinel[z1 * P:])
        y = sentinel.clone()
        for z0, z1 in [(0, 1), (1, 12), (12, 12), (12, nz)]:
            fl.fl_step_rk_stage_planes(m.handle, lim, dtype, 3, s, dt, z0, z1, thn, th0, y, u, w)
        assert torch.equal(y, ref)
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", ["superbee", "vanleer", "smart"])
def test_stage_adjoint_planes_compose_to_the_whole_stage(fl, dtype, lim):
    dims = (36, 10, 17)
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(23)
    P, nz = dims[0] * dims[1], dims[2]

    def field():
        return torch.tensor(rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3),
                            dtype=dtype, device="cuda")

    x, mu, la, lb = field(), field(), field(), field()
    u = torch.tensor(0.3 * W.mixed_sign_velocity(mesh.n_faces, 24), dtype=dtype, device="cuda")
    dt = 0.3 * min(h) / float(u.abs().max()) / 3
    m = fl.Mesh.structured(*dims, *h)
    for s in range(3):
        ref = torch.empty_like(x)
        fl.fl_step_rk_stage_adjoint(m.handle, lim, dtype, 3, s, dt, x, mu, la, lb, ref, u)
        out = torch.full_like(x, -3.5)
        fl.fl_step_rk_stage_adjoint_planes(m.handle, lim, dtype, 3, s, dt, 4, 11, x, mu, la, lb,
                                           out, u)
        torch.cuda.synchronize()
        assert torch.equal(out[4 * P:11 * P], ref[4 * P:11 * P])
        assert bool((out[:4 * P] == -3.5).all()) and bool((out[11 * P:] == -3.5).all())
        for z0, z1 in [(0, 4), (11, nz)]:
            fl.fl_step_rk_stage_adjoint_planes(m.handle, lim, dtype, 3, s, dt, z0, z1, x, mu, la,
                                               lb, out, u)
        assert torch.equal(out, ref)
    m.close()


def test_stage_planes_argument_errors(fl):
    dims = (16, 8, 6)
    h = (0.1, 0.1, 0.1)
    m = fl.Mesh.structured(*dims, *h)
    n = 16 * 8 * 6
    x = torch.rand(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    u = torch.rand(3 * n, dtype=torch.float64, device="cuda")
    for z0, z1 in [(-1, 2), (3, 2), (0, 7)]:
        with pytest.raises(fl.FLError) as e:
            fl.fl_step_rk_stage_planes(m.handle, "superbee", torch.float64, 1, 0, 0.01, z0, z1,
                                       None, x, y, u)
        assert e.value.status == fl.FL_EINVAL
        with pytest.raises(fl.FLError) as e:
            fl.fl_step_rk_stage_adjoint_planes(m.handle, "superbee", torch.float64, 1, 0, 0.01,
                                               z0, z1, x, x.clone(), None, None, y, u)
        assert e.value.status == fl.FL_EINVAL
    # an empty range runs nothing
    fl.fl_step_rk_stage_planes(m.handle, "superbee", torch.float64, 1, 0, 0.01, 3, 3, None, x, y,
                               u)
    torch.cuda.synchronize()
    assert bool((y == 0).all())
    m.close()
    # a face-based mesh has no planes
    mesh = W.structured_mesh(4, 4, 4, 0.25, 0.25, 0.25)
    fm = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                            mesh.volumes)
    xf = torch.rand(mesh.n_cells, dtype=torch.float64, device="cuda")
    uf = torch.rand(mesh.n_faces, dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk_stage_planes(fm.handle, "superbee", torch.float64, 1, 0, 0.01, 0, 1, None,
                                   xf, torch.empty_like(xf), uf)
    assert e.value.status == fl.FL_EUNSUPPORTED
    fm.close()


def test_decomposed_diagnostics(fl):
    # mass: the ranks' owned-plane sums (fl_reduce_mass on the owned planes)
    # add up to the whole mesh's; max |u_f|: every rank's local faces give the
    # global maximum (a single process: no group, each rank's own value)
    import math
    dims = (40, 12, 24)
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(31)
    th = rng.uniform(-1, 1, mesh.n_cells)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 32)
    ug = torch.tensor(u, device="cuda")
    shares, maxima = [], []
    for r in range(3):
        slab = Slab(dims, r, 3)
        ro = SlabRollout(slab, h, ug, "superbee", torch.float64, 0.01)
        tl = ro.local_field(torch.tensor(th, device="cuda"))
        shares.append(ro.mass(tl))
        maxima.append(ro.max_abs_velocity())
        ro.close()
    want = math.fsum((th * mesh.volumes).tolist())
    assert abs(math.fsum(shares) - want) <= 1e-13 * max(1.0, abs(want))
    assert max(maxima) == float(np.max(np.abs(u)))


# ------------------------------------------------------------------ pencils
class ThreadPencilTransport:
    """The four-neighbour exchange of W pencils run by host threads on one
    GPU: each ghost region is gathered from the neighbour's field with
    fl_halo_pack on the neighbour's mesh and scattered with fl_halo_unpack,
    between two barriers."""

    def __init__(self, fl, world):
        self.fl = fl
        self.reg = [None] * world
        self.fields = [None] * world
        self.bar = threading.Barrier(world)
        self.idx = {}

    def _dev(self, key, a):
        if key not in self.idx:
            self.idx[key] = torch.as_tensor(a, dtype=torch.int32, device="cuda")
        return self.idx[key]

    def exchange(self, pc, x):
        from paper_2110_03044_gb300.decomp import PencilTransport
        self.fields[pc.rank] = x
        self.bar.wait()
        peer = {"y_down": pc.y_down, "y_up": pc.y_up, "z_down": pc.z_down, "z_up": pc.z_up}
        recv = pc.exchange_lists()[1]
        for d, ridx in recv.items():
            q = self.reg[peer[d]]
            sidx = q.slab.exchange_lists()[0][PencilTransport.OPP[d]]
            tmp = torch.empty(ridx.shape[0], dtype=x.dtype, device="cuda")
            self.fl.fl_halo_pack(q.mesh.handle, x.dtype, self.fields[peer[d]],
                                 self._dev(("s", peer[d], d), sidx), sidx.shape[0], tmp)
            self.fl.fl_halo_unpack(self.reg[pc.rank].mesh.handle, x.dtype, tmp,
                                   self._dev(("r", pc.rank, d), ridx), ridx.shape[0], x)
        self.bar.wait()


def _pencils(fl, grid, dims, h, th, u, lim, dtype, rk, dt, nsteps, lam_T=None, every=2):
    from paper_2110_03044_gb300.decomp import HALO_ADJOINT, Pencil, PencilRollout
    world = grid[0] * grid[1]
    tr = ThreadPencilTransport(fl, world)
    ug = torch.tensor(u, device="cuda")
    halo = HALO_ADJOINT if lam_T is not None else 2
    ros = [PencilRollout(Pencil(dims, r, grid, halo=halo), h, ug, lim, dtype, dt, transport=tr)
           for r in range(world)]
    for r, ro in enumerate(ros):
        tr.reg[r] = ro
    out = [None] * world
    err = []

    def rank(r):
        try:
            torch.cuda.set_device(0)
            ro = ros[r]
            tl = ro.local_field(torch.tensor(th, device="cuda"))
            if lam_T is None:
                res = ro.step(tl, rk, nsteps)
            else:
                res = ro.gradient(tl, ro.local_field(torch.tensor(lam_T, device="cuda")), rk,
                                  nsteps, every)
            torch.cuda.synchronize()
            pc = ro.slab
            ids = pc._local_ids().reshape(pc.nzl + 2 * pc.halo, pc.nyl + 2 * pc.halo, dims[0])
            own = ids[pc.halo:pc.halo + pc.nzl, pc.halo:pc.halo + pc.nyl].ravel()
            out[r] = (own, pc.owned(res).reshape(-1).cpu())
        except BaseException as e:  # noqa: BLE001 -- reported below
            err.append(e)
            tr.bar.abort()

    ts = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for ro in ros:
        ro.close()
    if err:
        raise err[0]
    got = torch.empty(dims[0] * dims[1] * dims[2], dtype=dtype)
    for own, vals in out:
        got[torch.as_tensor(own)] = vals
    return got


@pytest.mark.parametrize("grid", [(2, 2), (3, 2), (1, 4)])
@pytest.mark.parametrize("dims,dtype", [((40, 12, 24), torch.float64),
                                        ((40, 12, 24), torch.float32),
                                        ((128, 16, 20), torch.float32)])
@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1), ("smart", 3)])
def test_pencil_rollout_equals_whole_mesh_bitwise(fl, grid, dims, dtype, lim, rk):
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(25)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 26)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    got = _pencils(fl, grid, dims, h, th, u, lim, dtype, rk, dt, 3)
    m = fl.Mesh.structured(*dims, *h)
    ref = torch.tensor(th, dtype=dtype, device="cuda")
    fl.step_rk(m, lim, ref, torch.tensor(u, dtype=dtype, device="cuda"), dt, 3, rk_order=rk)
    m.close()
    assert torch.equal(got, ref.cpu())


@pytest.mark.parametrize("lim,rk", [("superbee", 3), ("vanleer", 1)])
def test_pencil_gradient_matches_whole_mesh(fl, lim, rk):
    import oracle
    dims = (24, 14, 18)
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(27)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, 28)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    nsteps, every = 4, 2
    tgt = rng.normal(size=mesh.n_cells)
    thT = oracle.step(mesh, lim, rk, dt, nsteps, u, th)
    got = _pencils(fl, (2, 2), dims, h, th, u, lim, torch.float64, rk, dt, nsteps, thT - tgt,
                   every).numpy()
    one = _pencils(fl, (1, 1), dims, h, th, u, lim, torch.float64, rk, dt, nsteps, thT - tgt,
                   every).numpy()
    assert np.array_equal(got, one)
    m = fl.Mesh.structured(*dims, *h)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, rk, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty(mesh.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_step_rk_adjoint(m.handle, lim, torch.float64, rk, dt, nsteps, every,
                          torch.tensor(th, device="cuda"), torch.tensor(u, device="cuda"),
                          torch.tensor(thT - tgt, device="cuda"), g, ws, nb)
    m.close()
    whole = g.cpu().numpy()
    assert np.max(np.abs(got - whole)) <= 1e-12 * np.max(np.abs(whole))


@pytest.mark.parametrize("dims,dtype,pre", [((40, 12, 23), torch.float64, True),
                                            ((40, 12, 23), torch.float32, False),
                                            ((128, 16, 21), torch.float32, False)])
def test_stage_box_composes_and_leaves_other_cells(fl, dims, dtype, pre):
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(29)
    nx, ny, nz = dims
    th0 = torch.tensor(rng.uniform(-1, 1, mesh.n_cells), dtype=dtype, device="cuda")
    thn = torch.tensor(rng.uniform(-1, 1, mesh.n_cells), dtype=dtype, device="cuda")
    u = torch.tensor(0.3 * W.mixed_sign_velocity(mesh.n_faces, 30), dtype=dtype, device="cuda")
    dt = 0.3 * min(h) / float(u.abs().max()) / 3
    m = fl.Mesh.structured(*dims, *h)
    w = None
    if pre:
        w = torch.empty_like(u)
        fl.fl_velocity_prescale(m.handle, dtype, dt, u, w)
    boxes = [(0, 5, 0, 7), (5, ny, 0, 7), (0, 3, 7, nz), (3, ny - 1, 7, nz), (ny - 1, ny, 7, nz)]
    for s in range(3):
        ref = torch.empty_like(th0)
        fl.fl_step_rk_stage(m.handle, "smart", dtype, 3, s, dt, thn, th0, ref, u, w)
        y = torch.full_like(th0, 4.5)
        fl.fl_step_rk_stage_box(m.handle, "smart", dtype, 3, s, dt, *boxes[1], thn, th0, y, u, w)
        torch.cuda.synchronize()
        v, vr = y.view(nz, ny, nx), ref.view(nz, ny, nx)
        assert torch.equal(v[0:7, 5:ny], vr[0:7, 5:ny])
        assert bool((v[7:] == 4.5).all()) and bool((v[0:7, 0:5] == 4.5).all())
        for b in boxes[:1] + boxes[2:]:
            fl.fl_step_rk_stage_box(m.handle, "smart", dtype, 3, s, dt, *b, thn, th0, y, u, w)
        assert torch.equal(y, ref)
        # the adjoint box kernel composes the same way
        mu = torch.sin(th0 * 3).contiguous()
        oref = torch.empty_like(th0)
        fl.fl_step_rk_stage_adjoint(m.handle, "smart", dtype, 3, s, dt, th0, mu, thn, th0, oref,
                                    u)
        out = torch.full_like(th0, -1.5)
        for b in boxes:
            fl.fl_step_rk_stage_adjoint_box(m.handle, "smart", dtype, 3, s, dt, *b, th0, mu, thn,
                                            th0, out, u)
        assert torch.equal(out, oref)
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk_stage_box(m.handle, "smart", dtype, 3, 0, dt, 0, ny + 1, 0, 1, None, th0,
                                torch.empty_like(th0), u, w)
    assert e.value.status == fl.FL_EINVAL
    m.close()


def test_fp32_decomposed_gradients_equal_one_rank(fl):
    # FP32 reverse sweeps: three slabs and a 2 x 2 pencil grid give the bits
    # of the one-rank sweep of the same decomposition, and the FP64 oracle's
    # gradient to FP32 rounding (inputs cast to FP32 first)
    import oracle
    dims = (24, 14, 18)
    h = tuple(0.7 / d for d in dims)
    mesh = W.structured_mesh(*dims, *h)
    rng = np.random.default_rng(33)
    th = (rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3))
    th = th.astype(np.float32).astype(np.float64)
    u = (0.3 * W.mixed_sign_velocity(mesh.n_faces, 34)).astype(np.float32).astype(np.float64)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    nsteps, every = 3, 2
    tgt = rng.normal(size=mesh.n_cells)
    thT = oracle.step(mesh, "superbee", 3, dt, nsteps, u, th)
    lam = (thT - tgt).astype(np.float32).astype(np.float64)
    _, g_ref = oracle.gradient(mesh, "superbee", 3, dt, nsteps, u, th, tgt)
    scale = np.max(np.abs(g_ref))
    f32 = torch.float32
    s3 = _decomposed_gradient(fl, 3, dims, h, th, u, lam, "superbee", 3, dt, nsteps, every, f32)
    s1 = _decomposed_gradient(fl, 1, dims, h, th, u, lam, "superbee", 3, dt, nsteps, every, f32)
    assert np.array_equal(s3, s1)
    assert np.max(np.abs(s3 - g_ref)) <= 1e-4 * scale
    p4 = _pencils(fl, (2, 2), dims, h, th, u, "superbee", f32, 3, dt, nsteps, lam, every)
    p1 = _pencils(fl, (1, 1), dims, h, th, u, "superbee", f32, 3, dt, nsteps, lam, every)
    assert torch.equal(p4, p1)
    assert np.max(np.abs(p4.double().numpy() - g_ref)) <= 1e-4 * scale
