"""Domain decomposition of a structured periodic box, z-slabs or (y, z)
pencils, with a halo exchange once per RK stage.

The paper's large runs split the mesh across processes and exchange the cells
next to each cut before every operator application, overlapping the exchange
with the interior's computation (Section 4, the MareNostrum 4 and
Lomonosov-2 runs).  Here each rank (one GPU) owns a block of the box and
holds it as its own structured mesh with HALO ghost layers on each cut
side.  HALO = 2: the upstream cell of a face is a second neighbour, so the
update of a cell reads the cells within two of its own along each axis.

Slab: rank r owns the z planes [lo, hi) and holds nz_local + 2 HALO planes.
Planes are contiguous in the cell layout c = i + nx (j + ny k), so a halo is
one contiguous slice: no packing kernel.  Pencil: rank ry + py rz of a py x
pz grid owns a box of rows and planes; its ghost rows are strided, so each
message is gathered and scattered through index lists by the library's
fl_halo_pack / fl_halo_unpack.  The stencil runs along the axes only, so a
pencil's corner ghost cells are never read and never exchanged.

A stage updates only the owned cells, through the library's range-limited
stage kernels (fl_step_rk_stage_planes for a slab's plane ranges,
fl_step_rk_stage_box for a pencil's boxes), on the local mesh treated as
periodic: every owned cell reads only cells inside the local array, so its
result is the one the whole mesh gives, bit for bit (same inputs, same
per-face arithmetic, same order of the six face terms of a cell).  A face on
a cut is evaluated by both ranks from the same exchanged values with the
same code, so the scheme stays conservative.  The ghost layers of a stage
result are never written; the next exchange fills them before anything reads
them.  The face velocities of the local mesh are cut from the global field
once at set-up.

Exchange: messages go through torch.distributed point-to-point calls (NCCL
between GPUs, gloo on the host), posted together and tagged by the side they
fill, so that two ranks that are each other's neighbours on both sides pair
them correctly; a rank that is its own neighbour copies its own cells.

Overlap: the exchange of a stage input is started first; the owned cells at
least two cells from every cut (the stage's reach) need no ghost cell and run
while the halos travel; after the wait, the cells next to the cuts run.  With
NCCL the messages travel on the communicator's stream while the interior
kernel runs on the rank's stream, and the wait orders the rim kernels after
them without blocking the host.

The reverse sweep (gradient_rk) exchanges the adjoint field the same way
before every adjoint stage; the adjoint stage reads the stage states three
cells deep, so a slab or pencil for the reverse sweep keeps HALO_ADJOINT = 3
ghost layers.  partition.py applies the same loops to graph partitions of
face-based meshes.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

HALO = 2


@dataclass
class Slab:
    """The z-planes of a periodic nx x ny x nz box that rank ``rank`` of
    ``world`` owns, and the shape of its local mesh."""
    dims: tuple
    rank: int
    world: int
    halo: int = HALO

    def __post_init__(self):
        nx, ny, nz = self.dims
        if self.world < 1 or not 0 <= self.rank < self.world:
            raise ValueError("bad rank %d of %d" % (self.rank, self.world))
        if nz < 2:
            raise ValueError("a z-slab decomposition needs nz >= 2")
        self.lo = nz * self.rank // self.world
        self.hi = nz * (self.rank + 1) // self.world
        if self.hi - self.lo < self.halo:
            raise ValueError("rank %d would own %d planes, fewer than the halo of %d"
                             % (self.rank, self.hi - self.lo, self.halo))
        self.down = (self.rank - 1) % self.world
        self.up = (self.rank + 1) % self.world

    @property
    def nz_local(self) -> int:
        return self.hi - self.lo

    @property
    def local_dims(self) -> tuple:
        nx, ny, _ = self.dims
        return (nx, ny, self.nz_local + 2 * self.halo)

    @property
    def plane(self) -> int:
        return self.dims[0] * self.dims[1]

    def global_planes(self):
        """Global z index of every local plane (ghost planes wrap)."""
        nz = self.dims[2]
        return [(self.lo - self.halo + k) % nz for k in range(self.nz_local + 2 * self.halo)]

    def owned(self, x):
        """The owned planes of a local cell field (a view)."""
        P = self.plane
        return x[self.halo * P:(self.halo + self.nz_local) * P]

    def split(self, reach=None):
        """(interior, rims, whole): the owned local planes at least ``reach``
        planes from both cuts as one range (None when there are none), the
        ranges of the other owned planes, and the range of all of them."""
        reach = REACH if reach is None else reach
        h, n = self.halo, self.nz_local
        if n <= 2 * reach:
            return None, [(h, h + n)], (h, h + n)
        return ((h + reach, h + n - reach), [(h, h + reach), (h + n - reach, h + n)],
                (h, h + n))

    def check_adjoint(self):
        if self.halo < HALO_ADJOINT:
            raise ValueError("the reverse sweep needs a halo of %d planes" % HALO_ADJOINT)

    # ------------------------------------------------------------ set-up
    def local_cells(self, glob):
        """A local cell field (ghost planes included) cut from a global one
        (torch tensor or numpy array, flat, c = i + nx (j + ny k))."""
        P = self.plane
        parts = [glob[g * P:(g + 1) * P] for g in self.global_planes()]
        return _cat(parts)

    def local_faces(self, glob, n_axes):
        """The local face field: each of the ``n_axes`` face blocks (one per
        axis of extent > 1, x, y, z order, |C| faces each) cut like a cell
        field; the local mesh has the same active axes (its nz > 1)."""
        C = self.dims[0] * self.dims[1] * self.dims[2]
        return _cat([self.local_cells(glob[b * C:(b + 1) * C]) for b in range(n_axes)])


def _cat(parts):
    try:
        import torch
        if isinstance(parts[0], torch.Tensor):
            return torch.cat(parts).contiguous()
    except ImportError:
        pass
    import numpy as np
    return np.concatenate(parts)


class _Done:
    """The handle of an exchange that has completed when it was started."""

    def wait(self):
        return None


class _Pending:
    """The handle of an exchange in flight: its point-to-point requests."""

    def __init__(self, reqs):
        self.reqs = reqs

    def wait(self):
        for r in self.reqs:
            r.wait()


def start_exchange(transport, slab: Slab, x):
    """Start the halo exchange of x and return a handle whose wait() ends it;
    a transport with no start() exchanges at once."""
    start = getattr(transport, "start", None)
    if start is not None:
        return start(slab, x)
    transport.exchange(slab, x)
    return _Done()


class LocalTransport:
    """Exchange for a single rank: its neighbours are itself."""

    def exchange(self, slab: Slab, x):
        P, h, n = slab.plane, slab.halo, slab.nz_local
        x[0:h * P].copy_(x[n * P:(n + h) * P])
        x[(h + n) * P:(2 * h + n) * P].copy_(x[h * P:2 * h * P])

    def start(self, slab: Slab, x):
        self.exchange(slab, x)
        return _Done()


class TorchTransport:
    """Exchange through the default torch.distributed process group
    (point-to-point sends and receives into the ghost-plane slices)."""

    UP, DOWN = 11, 12  # tags: planes travelling to the rank above / below

    def exchange(self, slab: Slab, x):
        self.start(slab, x).wait()

    def start(self, slab: Slab, x):
        """Post the four point-to-point operations of x's halo exchange and
        return their handle (NCCL: enqueued on the communicator's stream)."""
        import torch.distributed as dist
        if slab.world == 1:
            return LocalTransport().start(slab, x)
        P, h, n = slab.plane, slab.halo, slab.nz_local
        top = x[n * P:(n + h) * P]            # my highest owned planes -> rank above
        bottom = x[h * P:2 * h * P]           # my lowest owned planes -> rank below
        lower_ghost = x[0:h * P]              # <- the rank below's highest planes
        upper_ghost = x[(h + n) * P:(2 * h + n) * P]  # <- the rank above's lowest planes
        ops = [dist.P2POp(dist.isend, top, slab.up, tag=self.UP),
               dist.P2POp(dist.isend, bottom, slab.down, tag=self.DOWN),
               dist.P2POp(dist.irecv, lower_ghost, slab.down, tag=self.UP),
               dist.P2POp(dist.irecv, upper_ghost, slab.up, tag=self.DOWN)]
        return _Pending(dist.batch_isend_irecv(ops))


StageFn = Callable[[int, Optional[object], object, object, int, int], None]
StageAdjointFn = Callable[[int, object, object, Optional[object], Optional[object], object, int,
                           int], None]

# The adjoint stage reads mu within two planes and the stage state x within
# three (the four faces of an axis around a cell, each with its upstream
# cell): a decomposed reverse sweep keeps three ghost planes.
HALO_ADJOINT = 3

# How far a stage reads the field whose halo is exchanged before it: the
# forward stage reads x, the adjoint stage mu, within two planes.
REACH = 2

# Rows of a structured stage tile (the kernels' 32 x 8 tiles)
TILE_ROWS = 8


def exchange_and_run(slab, transport, x, run, overlap=True, reach=None):
    """Exchange x's halo and run ``run(*r)`` over every owned local range r
    of the domain ``slab`` (a Slab: plane ranges (z0, z1); a Pencil: boxes
    (y0, y1, z0, z1); a partition.GraphPart: cell ranges (c0, c1)).  With ``overlap`` the part that reads no halo value (for a slab,
    the planes at least ``reach`` planes from both cuts) runs while the
    exchange is in flight and the rest after it ends; without it (or when
    there is no such interior) everything runs after the exchange."""
    interior, rims, whole = slab.split(reach)
    if not overlap or interior is None:
        transport.exchange(slab, x)
        run(*whole)
        return
    pending = start_exchange(transport, slab, x)
    run(*interior)
    pending.wait()
    for r in rims:
        run(*r)


def step_rk(slab: Slab, transport, stage: StageFn, rk_order: int, nsteps: int, theta, a, b=None,
            overlap=True):
    """``nsteps`` steps of Euler (rk_order 1) or SSP-RK3 (3) on the local
    field ``theta`` (owned planes valid on entry and on return), exchanging
    the halo of every stage input.  ``stage(s, theta_n, x, y, z0, z1)`` runs
    stage s into the local planes [z0, z1) of y (the library's
    fl_step_rk_stage_planes on the local mesh); ``a`` and ``b`` are local
    scratch fields of the same size (``b`` for SSP-RK3 only).  ``overlap``
    runs each stage's interior while its input's halo is exchanged.  Returns
    the local field that holds the result (``theta``)."""
    def run_stage(s, thn, x, y):
        exchange_and_run(slab, transport, x, lambda *r: stage(s, thn, x, y, *r), overlap)

    if rk_order == 1:
        cur, nxt = theta, a
        for _ in range(nsteps):
            run_stage(0, None, cur, nxt)
            cur, nxt = nxt, cur
        if cur is not theta:
            slab.owned(theta).copy_(slab.owned(cur))
        return theta
    if rk_order != 3:
        raise ValueError("rk_order must be 1 or 3")
    for _ in range(nsteps):
        run_stage(0, None, theta, a)
        run_stage(1, theta, a, b)
        run_stage(2, theta, b, theta)  # y may be theta_n, never x
    return theta


def gradient_rk(slab: Slab, transport, stage: StageFn, stage_adjoint: StageAdjointFn,
                rk_order: int, nsteps: int, every: int, theta0, lam_T, new, overlap=True):
    """Reverse-mode sweep of a decomposed rollout: dJ/dtheta_0 from
    lam_T = dJ/dtheta_T, with checkpoints every ``every`` steps and each
    segment recomputed (its stage inputs stored with their exchanged ghost
    planes) before its adjoint stages run in reverse; the adjoint's halo is
    exchanged before every adjoint stage, the same exchange as the forward
    stages', and with ``overlap`` the interior of every forward and adjoint
    stage runs while it travels.  ``stage_adjoint(s, x, mu, lam_a, lam_b,
    out, z0, z1)`` is the library's fl_step_rk_stage_adjoint_planes on the
    local mesh; ``new()`` gives a fresh local field.  The slab needs
    ``halo >= HALO_ADJOINT``.  Returns the local dJ/dtheta_0 (owned planes
    valid)."""
    slab.check_adjoint()
    if rk_order not in (1, 3):
        raise ValueError("rk_order must be 1 or 3")

    def run_stage(s, thn, x, y, keep):
        exchange_and_run(slab, transport, x, lambda *r: stage(s, thn, x, y, *r), overlap)
        keep.append(x.clone())  # x with its exchanged ghost planes (a stage never writes x)

    def fwd_step(th, keep):
        """one step in place on th, appending its exchanged stage inputs"""
        if rk_order == 1:
            y = new()
            run_stage(0, None, th, y, keep)
            slab.owned(th).copy_(slab.owned(y))
            return
        a, b = new(), new()
        run_stage(0, None, th, a, keep)
        run_stage(1, th, a, b, keep)
        run_stage(2, th, b, th, keep)  # y is theta_n, never x

    def adj(s, x, mu, lam_a, lam_b, out):
        exchange_and_run(slab, transport, mu,
                         lambda *r: stage_adjoint(s, x, mu, lam_a, lam_b, out, *r), overlap)

    # forward, storing a checkpoint every `every` steps
    checkpoints = []
    th = theta0.clone()
    for n in range(nsteps):
        if n % every == 0:
            checkpoints.append(th.clone())
        fwd_step(th, [])
    lam = lam_T.clone()
    for c in range(len(checkpoints) - 1, -1, -1):
        seg = min(every, nsteps - c * every)
        th = checkpoints[c].clone()
        states = []
        for _ in range(seg):
            fwd_step(th, states)
        for n in range(seg - 1, -1, -1):
            if rk_order == 1:
                out = new()
                adj(0, states[n], lam, None, None, out)
                lam = out
                continue
            x0, x1, x2 = states[3 * n], states[3 * n + 1], states[3 * n + 2]
            m2, m1, out = new(), new(), new()
            adj(2, x2, lam, None, None, m2)
            adj(1, x1, m2, None, None, m1)
            adj(0, x0, m1, m2, lam, out)
            lam = out
    return lam


# ------------------------------------------------------------------ pencils
@dataclass
class Pencil:
    """Rank ``rank`` of a py x pz grid of ranks (grid = (py, pz), rank =
    ry + py rz) owns the rows [ylo, yhi) of the planes [zlo, zhi) of a
    periodic nx x ny x nz box and holds them, with ``halo`` ghost rows and
    planes on each side, as a local structured mesh of nx x (nyl + 2 halo) x
    (nzl + 2 halo) cells.  The stencil runs along the axes only, so the
    corner ghost cells (ghost rows of ghost planes) are never read and never
    exchanged.  Pencils cut the halo volume of slabs when there are many
    ranks, and allow more ranks than nz / halo."""
    dims: tuple
    rank: int
    grid: tuple
    halo: int = HALO

    def __post_init__(self):
        nx, ny, nz = self.dims
        py, pz = self.grid
        if py < 1 or pz < 1 or not 0 <= self.rank < py * pz:
            raise ValueError("bad rank %d of a %d x %d grid" % (self.rank, py, pz))
        if ny < 2 or nz < 2:
            raise ValueError("a pencil decomposition needs ny >= 2 and nz >= 2")
        self.ry, self.rz = self.rank % py, self.rank // py
        self.ylo, self.yhi = ny * self.ry // py, ny * (self.ry + 1) // py
        self.zlo, self.zhi = nz * self.rz // pz, nz * (self.rz + 1) // pz
        if min(self.yhi - self.ylo, self.zhi - self.zlo) < self.halo:
            raise ValueError("rank %d would own fewer rows or planes than the halo of %d"
                             % (self.rank, self.halo))
        self.y_down = (self.ry - 1) % py + py * self.rz
        self.y_up = (self.ry + 1) % py + py * self.rz
        self.z_down = self.ry + py * ((self.rz - 1) % pz)
        self.z_up = self.ry + py * ((self.rz + 1) % pz)
        self._idx = None

    @property
    def world(self) -> int:
        return self.grid[0] * self.grid[1]

    @property
    def nyl(self) -> int:
        return self.yhi - self.ylo

    @property
    def nzl(self) -> int:
        return self.zhi - self.zlo

    @property
    def local_dims(self) -> tuple:
        return (self.dims[0], self.nyl + 2 * self.halo, self.nzl + 2 * self.halo)

    def _local_ids(self):
        """Global flat id of every local cell (ghost rows and planes wrap)."""
        import numpy as np
        nx, ny, nz = self.dims
        h = self.halo
        rows = (self.ylo - h + np.arange(self.nyl + 2 * h)) % ny
        planes = (self.zlo - h + np.arange(self.nzl + 2 * h)) % nz
        return ((planes[:, None, None] * ny + rows[None, :, None]) * nx
                + np.arange(nx)[None, None, :]).ravel()

    def _box(self, j0, j1, k0, k1):
        """Local flat ids of the rows [j0, j1) of the local planes [k0, k1)."""
        import numpy as np
        nx, nyl2 = self.dims[0], self.nyl + 2 * self.halo
        k = np.arange(k0, k1)[:, None, None]
        j = np.arange(j0, j1)[None, :, None]
        return ((k * nyl2 + j) * nx + np.arange(nx)[None, None, :]).ravel().astype(np.int32)

    def exchange_lists(self):
        """(send, recv) index lists of the four messages: for each of
        'y_down', 'y_up', 'z_down', 'z_up', the local ids this rank sends to
        that neighbour and the local ids of the ghost cells it fills from it.
        The two ends of a message list their cells in the same (plane, row,
        column) order."""
        if self._idx is None:
            h, nyl, nzl = self.halo, self.nyl, self.nzl
            own_z, own_y = (h, h + nzl), (h, h + nyl)
            send = {"y_down": self._box(h, 2 * h, *own_z),
                    "y_up": self._box(nyl, nyl + h, *own_z),
                    "z_down": self._box(*own_y, h, 2 * h),
                    "z_up": self._box(*own_y, nzl, nzl + h)}
            recv = {"y_down": self._box(0, h, *own_z),
                    "y_up": self._box(h + nyl, nyl + 2 * h, *own_z),
                    "z_down": self._box(*own_y, 0, h),
                    "z_up": self._box(*own_y, h + nzl, nzl + 2 * h)}
            self._idx = (send, recv)
        return self._idx

    def owned(self, x):
        """The owned box of a local cell field (a strided view)."""
        h = self.halo
        v = x.view(self.nzl + 2 * h, self.nyl + 2 * h, self.dims[0])
        return v[h:h + self.nzl, h:h + self.nyl, :]

    def split(self, reach=None):
        """(interior, rims, whole) boxes (y0, y1, z0, z1) of the owned cells:
        the interior at least ``reach`` planes and ``reach`` rows (a tile's 8
        rows on pencils of more than 32 rows) from every cut, the rims the
        rest (two slabs of planes and two bands of rows)."""
        reach = REACH if reach is None else reach
        h, nyl, nzl = self.halo, self.nyl, self.nzl
        whole = (h, h + nyl, h, h + nzl)
        # the row bands are as tall as the stage tiles (8 rows) when the
        # pencil is tall enough: a 2-row band would leave 6 of a tile's 8
        # rows idle
        ry = max(reach, TILE_ROWS) if nyl > 4 * TILE_ROWS else reach
        if nyl <= 2 * ry or nzl <= 2 * reach:
            return None, [whole], whole
        zi = (h + reach, h + nzl - reach)
        interior = (h + ry, h + nyl - ry) + zi
        rims = [(h, h + nyl, h, h + reach), (h, h + nyl, h + nzl - reach, h + nzl),
                (h, h + ry) + zi, (h + nyl - ry, h + nyl) + zi]
        return interior, rims, whole

    def check_adjoint(self):
        if self.halo < HALO_ADJOINT:
            raise ValueError("the reverse sweep needs a halo of %d" % HALO_ADJOINT)

    def local_cells(self, glob):
        """A local cell field cut from a global one (torch tensor or numpy
        array, flat, c = i + nx (j + ny k))."""
        return glob[_index(glob, self._local_ids())]

    def local_faces(self, glob, n_axes):
        """The local face field: each of the ``n_axes`` face blocks cut like
        a cell field."""
        import numpy as np
        C = self.dims[0] * self.dims[1] * self.dims[2]
        ids = self._local_ids()
        return glob[_index(glob, np.concatenate([ids + b * C for b in range(n_axes)]))]


def _index(x, ids):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return torch.as_tensor(ids, dtype=torch.long, device=x.device)
    except ImportError:
        pass
    return ids


class PencilTransport:
    """The four-neighbour exchange of a Pencil through the default
    torch.distributed process group (or, for one rank in a direction, a
    copy of its own cells).  ``pack(x, index, out)`` gathers x[index] into
    out and ``unpack(buf, index, x)`` scatters buf into x[index]: the
    library's fl_halo_pack / fl_halo_unpack for device fields (see
    PencilRollout), index copies on the host."""

    TAGS = {"y_down": 31, "y_up": 32, "z_down": 33, "z_up": 34}
    OPP = {"y_down": "y_up", "y_up": "y_down", "z_down": "z_up", "z_up": "z_down"}

    def __init__(self, pack=None, unpack=None):
        self.pack = pack or (lambda x, idx, out: out.copy_(x[idx.long()]))
        self.unpack = unpack or (lambda buf, idx, x: x.index_copy_(0, idx.long(), buf))
        self._dev = {}

    def exchange(self, pc: Pencil, x):
        self.start(pc, x).wait()

    def _lists(self, pc, x):
        import torch
        key = (id(pc), x.dtype, x.device)
        if key not in self._dev:
            send, recv = pc.exchange_lists()
            mk = lambda a: torch.as_tensor(a, dtype=torch.int32, device=x.device)  # noqa: E731
            self._dev[key] = ({d: mk(a) for d, a in send.items()},
                              {d: mk(a) for d, a in recv.items()},
                              {d: torch.empty(a.shape[0], dtype=x.dtype, device=x.device)
                               for d, a in send.items()},
                              {d: torch.empty(a.shape[0], dtype=x.dtype, device=x.device)
                               for d, a in recv.items()})
        return self._dev[key]

    def start(self, pc: Pencil, x):
        import torch.distributed as dist
        send, recv, sbuf, rbuf = self._lists(pc, x)
        peer = {"y_down": pc.y_down, "y_up": pc.y_up, "z_down": pc.z_down, "z_up": pc.z_up}
        for d in send:
            self.pack(x, send[d], sbuf[d])
        ops, local = [], []
        for d in send:
            if peer[d] == pc.rank:
                local.append(d)  # one rank in this direction: its own cells
                continue
            # a message to the neighbour on side d fills its ghost cells on the
            # opposite side, and carries the tag of that side
            ops.append(dist.P2POp(dist.isend, sbuf[d], peer[d], tag=self.TAGS[self.OPP[d]]))
            ops.append(dist.P2POp(dist.irecv, rbuf[d], peer[d], tag=self.TAGS[d]))
        reqs = dist.batch_isend_irecv(ops) if ops else []
        return _PencilPending(self, x, recv, sbuf, rbuf, local, reqs)


class _PencilPending:
    def __init__(self, tr, x, recv, sbuf, rbuf, local, reqs):
        self.args = (tr, x, recv, sbuf, rbuf, local, reqs)

    def wait(self):
        tr, x, recv, sbuf, rbuf, local, reqs = self.args
        for r in reqs:
            r.wait()
        for d in recv:
            # a direction served by this rank itself: its ghost cells on side
            # d are its own cells sent towards the opposite side
            src = sbuf[PencilTransport.OPP[d]] if d in local else rbuf[d]
            tr.unpack(src, recv[d], x)


class SlabRollout:
    """A rank's part of a decomposed rollout on the GPU: the local mesh, its
    face velocities (and, in FP64, the pre-scaled velocity fl_step_rk uses),
    the stage scratch, and the library's plane-range stage kernels.  The
    owned planes of the result equal those of fl_step_rk on the whole mesh,
    bit for bit.  ``overlap`` runs each stage's interior planes while the
    halo of its input is exchanged."""

    def __init__(self, slab: Slab, h, u_global, limiter, dtype, dt, transport=None,
                 overlap=True):
        import torch

        from . import Mesh, fl_velocity_prescale
        self.slab = slab
        self.mesh = Mesh.structured(*slab.local_dims, *h)
        n_axes = sum(1 for d in slab.dims if d > 1)
        self.u = slab.local_faces(u_global, n_axes).to(dtype).contiguous()
        self.w = None
        if dtype == torch.float64 and dt > 0:
            self.w = torch.empty_like(self.u)
            fl_velocity_prescale(self.mesh.handle, dtype, dt, self.u, self.w)
        self.limiter, self.dtype, self.dt = limiter, dtype, dt
        self.transport = transport or TorchTransport()
        self.overlap = overlap
        self.h = tuple(h)
        self._owned_mesh = None

    def local_field(self, theta_global):
        return self.slab.local_cells(theta_global).to(self.dtype).contiguous()

    def _stage_fn(self, rk_order):
        from . import fl_step_rk_stage_planes

        def stage(s, thn, x, y, z0, z1):
            fl_step_rk_stage_planes(self.mesh.handle, self.limiter, self.dtype, rk_order, s,
                                    self.dt, z0, z1, thn, x, y, self.u, self.w)

        return stage

    def step(self, theta_local, rk_order, nsteps):
        import torch
        a = torch.empty_like(theta_local)
        b = torch.empty_like(theta_local) if rk_order == 3 else None
        return step_rk(self.slab, self.transport, self._stage_fn(rk_order), rk_order, nsteps,
                       theta_local, a, b, overlap=self.overlap)

    def gradient(self, theta_local, lam_T_local, rk_order, nsteps, every):
        """dJ/dtheta_0 on this rank's slab (see gradient_rk); the slab needs
        a halo of HALO_ADJOINT planes."""
        import torch

        from . import fl_step_rk_stage_adjoint_planes

        def stage_adjoint(s, x, mu, lam_a, lam_b, out, z0, z1):
            fl_step_rk_stage_adjoint_planes(self.mesh.handle, self.limiter, self.dtype, rk_order,
                                            s, self.dt, z0, z1, x, mu, lam_a, lam_b, out, self.u,
                                            self.w)

        return gradient_rk(self.slab, self.transport, self._stage_fn(rk_order), stage_adjoint,
                           rk_order, nsteps, every, theta_local, lam_T_local,
                           lambda: torch.empty_like(theta_local), overlap=self.overlap)

    def mass(self, theta_local):
        """sum_c V_c theta_c over the whole mesh (the conservation
        diagnostic): fl_reduce_mass over this rank's owned planes, summed
        over the ranks."""
        import torch

        from . import Mesh, fl_reduce_mass, fl_reduce_workspace_size
        from .replicas import sum_over_ranks
        if self._owned_mesh is None:
            nx, ny, _ = self.slab.dims
            self._owned_mesh = Mesh.structured(nx, ny, self.slab.nz_local, *self.h)
        ws = torch.empty(max(fl_reduce_workspace_size(), 1), dtype=torch.uint8,
                         device=theta_local.device)
        own = fl_reduce_mass(self._owned_mesh.handle, self.dtype, self.slab.owned(theta_local), ws)
        return sum_over_ranks(own, theta_local.device)

    def max_abs_velocity(self):
        """max_f |u_f| over the whole mesh (the CFL diagnostic): this rank's
        local faces (copies of ghost-plane faces change no maximum), then
        the maximum over the ranks."""
        return _max_abs_faces(self.u)

    def close(self):
        if self._owned_mesh is not None:
            self._owned_mesh.close()
        self.mesh.close()


def _max_abs_faces(u):
    import torch

    from . import fl_reduce_max_abs, fl_reduce_workspace_size
    from .replicas import max_over_ranks
    ws = torch.empty(max(fl_reduce_workspace_size(), 1), dtype=torch.uint8, device=u.device)
    return max_over_ranks(fl_reduce_max_abs(u.dtype, u, u.numel(), ws), u.device)


class PencilRollout(SlabRollout):
    """SlabRollout for a Pencil: the library's box-range stage kernels
    (fl_step_rk_stage_box / fl_step_rk_stage_adjoint_box) on the interior
    and the four rim boxes, and the four-neighbour exchange with its halo
    gathered and scattered by fl_halo_pack / fl_halo_unpack."""

    def __init__(self, pencil: Pencil, h, u_global, limiter, dtype, dt, transport=None,
                 overlap=True):
        from . import fl_halo_pack, fl_halo_unpack
        super().__init__(pencil, h, u_global, limiter, dtype, dt,
                         transport=transport or _no_transport, overlap=overlap)
        if transport is None:
            hdl = self.mesh.handle
            self.transport = PencilTransport(
                pack=lambda x, idx, out: fl_halo_pack(hdl, x.dtype, x, idx, idx.numel(), out),
                unpack=lambda buf, idx, x: fl_halo_unpack(hdl, x.dtype, buf, idx, idx.numel(),
                                                          x))

    def _stage_fn(self, rk_order):
        from . import fl_step_rk_stage_box

        def stage(s, thn, x, y, y0, y1, z0, z1):
            fl_step_rk_stage_box(self.mesh.handle, self.limiter, self.dtype, rk_order, s, self.dt,
                                 y0, y1, z0, z1, thn, x, y, self.u, self.w)

        return stage

    def gradient(self, theta_local, lam_T_local, rk_order, nsteps, every):
        """dJ/dtheta_0 on this rank's pencil (see gradient_rk); the pencil
        needs a halo of HALO_ADJOINT."""
        import torch

        from . import fl_step_rk_stage_adjoint_box

        def stage_adjoint(s, x, mu, lam_a, lam_b, out, y0, y1, z0, z1):
            fl_step_rk_stage_adjoint_box(self.mesh.handle, self.limiter, self.dtype, rk_order, s,
                                         self.dt, y0, y1, z0, z1, x, mu, lam_a, lam_b, out,
                                         self.u, self.w)

        return gradient_rk(self.slab, self.transport, self._stage_fn(rk_order), stage_adjoint,
                           rk_order, nsteps, every, theta_local, lam_T_local,
                           lambda: torch.empty_like(theta_local), overlap=self.overlap)

    def mass(self, theta_local):
        """sum_c V_c theta_c over the whole mesh: fl_reduce_mass over this
        rank's owned box (copied into one block), summed over the ranks."""
        import torch

        from . import Mesh, fl_reduce_mass, fl_reduce_workspace_size
        from .replicas import sum_over_ranks
        pc = self.slab
        if self._owned_mesh is None:
            self._owned_mesh = Mesh.structured(pc.dims[0], pc.nyl, pc.nzl, *self.h)
        ws = torch.empty(max(fl_reduce_workspace_size(), 1), dtype=torch.uint8,
                         device=theta_local.device)
        own = fl_reduce_mass(self._owned_mesh.handle, self.dtype,
                             pc.owned(theta_local).contiguous().view(-1), ws)
        return sum_over_ranks(own, theta_local.device)


class _NoTransport:
    def exchange(self, slab, x):
        raise RuntimeError("no transport")


_no_transport = _NoTransport()
