"""Domain decomposition of a structured periodic box into z-slabs, with a
halo exchange once per RK stage.

The paper's large runs split the mesh across processes and exchange the cells
next to each cut before every operator application, overlapping the exchange
with the interior's computation (Section 4, the MareNostrum 4 and
Lomonosov-2 runs).  Here each rank (one GPU) owns a contiguous range of z
planes [lo, hi) of an nx x ny x nz periodic box and holds it as its own
structured mesh of nz_local + 2 HALO planes: HALO ghost planes below, the
owned planes, HALO ghost planes above.  HALO = 2, because the upstream cell
of a face is a second neighbour, so the update of a cell reads the planes
within two of its own.

A stage runs the library's ordinary stage kernel (fl_step_rk_stage) on that
local mesh as if it were periodic in z: every owned plane reads only planes
inside the local array, so its result is the one the whole mesh would give,
bit for bit (same inputs, same per-face arithmetic, same order of the six
face terms of a cell); the ghost planes come out wrong (the local wrap) and
are overwritten by the next exchange before anything reads them.  A face on
a cut is evaluated by both ranks from the same exchanged values with the
same code, so both see the same flux and the scheme stays conservative.
The face velocities of the local mesh (ghost planes included) are copied
once from the global field at set-up.

Exchange per stage input x: the HALO lowest owned planes go to the rank
below (they become its upper ghost planes), the HALO highest owned planes to
the rank above (its lower ghost planes).  Planes are contiguous in the cell
layout c = i + nx (j + ny k), so a halo is one contiguous slice: no packing
kernel is needed.  Messages go through torch.distributed point-to-point
calls (NCCL between GPUs, gloo on the host), sends upward first and
receives from below first on every rank, with tags, so that with two ranks
(where the rank below is also the rank above) the messages pair correctly.
A rank whose neighbours are itself (one rank) copies its own planes.

The adjoint (gradient_rk) exchanges the adjoint field the same way before
every adjoint stage; it reads the stage states three planes deep, so a slab
for the reverse sweep keeps HALO_ADJOINT = 3 ghost planes.

Overlap (the paper's split runs hide the exchange behind the interior's
work): a stage updates only the owned planes, through the library's
plane-range stage (fl_step_rk_stage_planes).  The exchange of its input is
started first; the owned planes at least two planes away from both cuts (the
stage's reach) need no ghost plane and run while the halos travel; after the
wait, the two planes next to each cut run.  With NCCL the messages travel on
the communicator's own stream while the interior kernel runs on the rank's
stream, and the wait orders the rim kernels after the messages without
blocking the host.  The ghost planes of a stage result are never written:
the next exchange fills them before anything reads them.  A slab of fewer
than 2 x reach planes has no interior and runs its owned planes after the
wait.
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


def exchange_and_run(slab, transport, x, run, overlap=True, reach=None):
    """Exchange x's halo and run ``run(lo, hi)`` over every owned local range
    of the domain ``slab`` (a Slab: plane ranges; a partition.GraphPart: cell
    ranges).  With ``overlap`` the part that reads no halo value (for a slab,
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
    for lo, hi in rims:
        run(lo, hi)


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
        exchange_and_run(slab, transport, x, lambda z0, z1: stage(s, thn, x, y, z0, z1), overlap)

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
        exchange_and_run(slab, transport, x, lambda z0, z1: stage(s, thn, x, y, z0, z1), overlap)
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
                         lambda z0, z1: stage_adjoint(s, x, mu, lam_a, lam_b, out, z0, z1), overlap)

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
