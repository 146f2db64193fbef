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

Overlap: at 256^2 planes a halo is 2 x 65536 values per side (1 MiB in
FP64), against a stage of 16.8 M cells; the exchange is issued before the
stage and waited for, without splitting the stage into interior and rim.
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


class LocalTransport:
    """Exchange for a single rank: its neighbours are itself."""

    def exchange(self, slab: Slab, x):
        P, h, n = slab.plane, slab.halo, slab.nz_local
        x[0:h * P].copy_(x[n * P:(n + h) * P])
        x[(h + n) * P:(2 * h + n) * P].copy_(x[h * P:2 * h * P])


class TorchTransport:
    """Exchange through the default torch.distributed process group
    (point-to-point sends and receives into the ghost-plane slices)."""

    UP, DOWN = 11, 12  # tags: planes travelling to the rank above / below

    def exchange(self, slab: Slab, x):
        import torch.distributed as dist
        if slab.world == 1:
            return LocalTransport().exchange(slab, x)
        P, h, n = slab.plane, slab.halo, slab.nz_local
        top = x[n * P:(n + h) * P]            # my highest owned planes -> rank above
        bottom = x[h * P:2 * h * P]           # my lowest owned planes -> rank below
        lower_ghost = x[0:h * P]              # <- the rank below's highest planes
        upper_ghost = x[(h + n) * P:(2 * h + n) * P]  # <- the rank above's lowest planes
        ops = [dist.P2POp(dist.isend, top, slab.up, tag=self.UP),
               dist.P2POp(dist.isend, bottom, slab.down, tag=self.DOWN),
               dist.P2POp(dist.irecv, lower_ghost, slab.down, tag=self.UP),
               dist.P2POp(dist.irecv, upper_ghost, slab.up, tag=self.DOWN)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


StageFn = Callable[[int, Optional[object], object, object], None]
StageAdjointFn = Callable[[int, object, object, Optional[object], Optional[object], object], None]

# The adjoint stage reads mu within two planes and the stage state x within
# three (the four faces of an axis around a cell, each with its upstream
# cell): a decomposed reverse sweep keeps three ghost planes.
HALO_ADJOINT = 3


def step_rk(slab: Slab, transport, stage: StageFn, rk_order: int, nsteps: int, theta, a, b=None):
    """``nsteps`` steps of Euler (rk_order 1) or SSP-RK3 (3) on the local
    field ``theta`` (owned planes valid on entry and on return), exchanging
    the halo of every stage input.  ``stage(s, theta_n, x, y)`` runs stage s
    into y (the library's fl_step_rk_stage on the local mesh); ``a`` and ``b``
    are local scratch fields of the same size (``b`` for SSP-RK3 only).
    Returns the local field that holds the result (``theta``)."""
    if rk_order == 1:
        cur, nxt = theta, a
        for _ in range(nsteps):
            transport.exchange(slab, cur)
            stage(0, None, cur, nxt)
            cur, nxt = nxt, cur
        if cur is not theta:
            theta.copy_(cur)
        return theta
    if rk_order != 3:
        raise ValueError("rk_order must be 1 or 3")
    for _ in range(nsteps):
        transport.exchange(slab, theta)
        stage(0, None, theta, a)
        transport.exchange(slab, a)
        stage(1, theta, a, b)
        transport.exchange(slab, b)
        stage(2, theta, b, theta)  # y may be theta_n, never x
    return theta


def gradient_rk(slab: Slab, transport, stage: StageFn, stage_adjoint: StageAdjointFn,
                rk_order: int, nsteps: int, every: int, theta0, lam_T, new):
    """Reverse-mode sweep of a decomposed rollout: dJ/dtheta_0 from
    lam_T = dJ/dtheta_T, with checkpoints every ``every`` steps and each
    segment recomputed (its stage inputs stored with their exchanged ghost
    planes) before its adjoint stages run in reverse; the adjoint's halo is
    exchanged before every adjoint stage, the same exchange as the forward
    stages'.  ``stage_adjoint(s, x, mu, lam_a, lam_b, out)`` is the
    library's fl_step_rk_stage_adjoint on the local mesh; ``new()`` gives a
    fresh local field.  The slab needs ``halo >= HALO_ADJOINT``.  Returns the
    local dJ/dtheta_0 (owned planes valid)."""
    if slab.halo < HALO_ADJOINT:
        raise ValueError("the reverse sweep needs a halo of %d planes" % HALO_ADJOINT)
    if rk_order not in (1, 3):
        raise ValueError("rk_order must be 1 or 3")

    def fwd_step(th, keep):
        """one step in place on th, appending its exchanged stage inputs"""
        transport.exchange(slab, th)
        keep.append(th.clone())
        if rk_order == 1:
            y = new()
            stage(0, None, th, y)
            th.copy_(y)
            return
        a, b = new(), new()
        stage(0, None, th, a)
        transport.exchange(slab, a)
        keep.append(a.clone())
        stage(1, th, a, b)
        transport.exchange(slab, b)
        keep.append(b.clone())
        stage(2, th, b, th)

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
            transport.exchange(slab, lam)
            if rk_order == 1:
                out = new()
                stage_adjoint(0, states[n], lam, None, None, out)
                lam = out
                continue
            x0, x1, x2 = states[3 * n], states[3 * n + 1], states[3 * n + 2]
            m2, m1, out = new(), new(), new()
            stage_adjoint(2, x2, lam, None, None, m2)
            transport.exchange(slab, m2)
            stage_adjoint(1, x1, m2, None, None, m1)
            transport.exchange(slab, m1)
            stage_adjoint(0, x0, m1, m2, lam, out)
            lam = out
    return lam


class SlabRollout:
    """A rank's part of a decomposed rollout on the GPU: the local mesh, its
    face velocities (and, in FP64, the pre-scaled velocity fl_step_rk uses),
    the stage scratch, and the library's stage kernel.  The owned planes of
    the result equal those of fl_step_rk on the whole mesh, bit for bit."""

    def __init__(self, slab: Slab, h, u_global, limiter, dtype, dt, transport=None):
        import torch

        from . import Mesh, fl_velocity_prescale, fl_step_rk_stage
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
        self._stage = fl_step_rk_stage

    def local_field(self, theta_global):
        return self.slab.local_cells(theta_global).to(self.dtype).contiguous()

    def step(self, theta_local, rk_order, nsteps):
        import torch
        a = torch.empty_like(theta_local)
        b = torch.empty_like(theta_local) if rk_order == 3 else None

        def stage(s, thn, x, y):
            self._stage(self.mesh.handle, self.limiter, self.dtype, rk_order, s, self.dt, thn, x,
                        y, self.u, self.w)

        return step_rk(self.slab, self.transport, stage, rk_order, nsteps, theta_local, a, b)

    def gradient(self, theta_local, lam_T_local, rk_order, nsteps, every):
        """dJ/dtheta_0 on this rank's slab (see gradient_rk); the slab needs
        a halo of HALO_ADJOINT planes."""
        import torch

        from . import fl_step_rk_stage_adjoint

        def stage(s, thn, x, y):
            self._stage(self.mesh.handle, self.limiter, self.dtype, rk_order, s, self.dt, thn, x,
                        y, self.u, self.w)

        def stage_adjoint(s, x, mu, lam_a, lam_b, out):
            fl_step_rk_stage_adjoint(self.mesh.handle, self.limiter, self.dtype, rk_order, s,
                                     self.dt, x, mu, lam_a, lam_b, out, self.u, self.w)

        return gradient_rk(self.slab, self.transport, stage, stage_adjoint, rk_order, nsteps,
                           every, theta_local, lam_T_local, lambda: torch.empty_like(theta_local))

    def close(self):
        self.mesh.close()
