"""Graph partitioning of a face-based mesh, with a two-ring halo exchanged
once per RK stage.

The paper's split runs of unstructured meshes give each process one part of
the cell graph and refresh, before every operator application, the copies of
the neighbouring parts' cells that its stencils read (Section 4).  The update
of a cell reads its faces' other cells and, behind the upwind cell of each
face, that cell's neighbours: the stencil reaches two cells deep in the cell
graph.  So a part keeps two rings of halo cells:

* ring 1: the cells of other parts adjacent to an owned cell.  The upwind
  cell of a face of an owned cell is an owned cell or a ring-1 cell, so a
  ring-1 cell brings all its faces (its upstream stencil must be whole);
* ring 2: the other cells of the ring-1 cells' faces.  Their own face lists
  are cut, which is harmless: no stencil of an owned cell is taken at them.

The local mesh (the library's fl_mesh_create_local) lists its cells as
[interior | rim | halo]: interior cells have no halo cell within two cells
(their update reads owned values only), rim cells do, and the halo cells
come grouped by the part that owns them, each group in ascending global id,
so that a neighbour's values land in one contiguous slice of a local field.
Local faces are the faces of the owned and ring-1 cells in ascending global
id: a cell then sums its faces in the whole mesh's order, and an owned cell
gets the whole mesh's bits.

Partitioner: recursive bisection of the cell graph along breadth-first
level structures.  A part is split by a breadth-first search from a
pseudo-peripheral cell of it (the last cell reached by a search from any
cell), the first share of the visiting order going to one side: that side is
a connected ball of the graph and the other its complement, found without
coordinates or an external library.  The shares follow the number of ranks
on each side, so any number of ranks works.

Exchange per stage input x: for every neighbour part, the owned values it
holds as halo are gathered into a send buffer (the library's fl_halo_pack on
the GPU) and sent; the halo slice that part fills is received in place.
Messages are torch.distributed point-to-point operations posted together
(NCCL between GPUs, gloo on the host).  Interior cells update while they
travel, the rim after (decomp.exchange_and_run).  The reverse sweep runs the
same exchange on the adjoint field: the face-based adjoint of an owned cell
reads the adjoint and the stage state within two cells as well.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np


# ------------------------------------------------------------ the cell graph
def cell_graph(n_cells: int, face_cells) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """CSR of the cell graph: (ptr, neighbour, face) with the neighbours of
    cell c in neighbour[ptr[c]:ptr[c + 1]], across faces face[...] listed in
    ascending face id."""
    fc = np.asarray(face_cells, dtype=np.int64).reshape(-1, 2)
    F = fc.shape[0]
    src = np.concatenate([fc[:, 0], fc[:, 1]])
    dst = np.concatenate([fc[:, 1], fc[:, 0]])
    fid = np.concatenate([np.arange(F), np.arange(F)])
    order = np.lexsort((fid, src))
    ptr = np.zeros(n_cells + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    np.cumsum(ptr, out=ptr)
    return ptr, dst[order], fid[order]


def _adjacency(n_cells: int, face_cells):
    """The cell graph as a symmetric sparse matrix (scipy CSR)."""
    from scipy.sparse import coo_matrix
    fc = np.asarray(face_cells, dtype=np.int64).reshape(-1, 2)
    r = np.concatenate([fc[:, 0], fc[:, 1]])
    c = np.concatenate([fc[:, 1], fc[:, 0]])
    a = coo_matrix((np.ones(r.shape[0], dtype=np.int8), (r, c)), shape=(n_cells, n_cells))
    return a.tocsr()


def _level_order(adj, cells):
    """The cells of one part in the breadth-first order from a
    pseudo-peripheral cell (the last cell reached from the part's first
    cell), component after component."""
    from scipy.sparse.csgraph import breadth_first_order, connected_components
    sub = adj[cells][:, cells]
    ncomp, labels = connected_components(sub, directed=False)
    out = []
    firsts = np.unique(labels, return_index=True)[1]  # each component's lowest cell
    for comp in np.argsort(firsts):
        seed = int(firsts[comp])
        far = int(breadth_first_order(sub, seed, directed=False, return_predecessors=False)[-1])
        out.append(cells[breadth_first_order(sub, far, directed=False,
                                             return_predecessors=False)])
    return np.concatenate(out) if out else cells[:0]


def partition_graph(n_cells: int, face_cells, world: int) -> np.ndarray:
    """part[c] in [0, world) for every cell: recursive bisection along
    breadth-first level structures (see the module notes)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    adj = _adjacency(n_cells, face_cells)
    part = np.zeros(n_cells, dtype=np.int32)

    def split(cells, r0, k):
        if k == 1 or len(cells) == 0:
            part[cells] = r0
            return
        k1 = k // 2
        order = _level_order(adj, cells)
        n1 = len(order) * k1 // k
        split(order[:n1], r0, k1)
        split(order[n1:], r0 + k1, k - k1)

    split(np.arange(n_cells, dtype=np.int64), 0, world)
    return part


# ------------------------------------------------------------- one local part
@dataclass
class GraphPart:
    """Rank ``rank``'s part of a partitioned face-based mesh: its local cell
    and face lists (global ids) and its exchange lists."""
    rank: int
    world: int
    owned_ids: np.ndarray          # global ids, interior then rim
    n_interior: int
    halo_ids: np.ndarray           # global ids, grouped by owner part
    face_ids: np.ndarray           # global ids of the local faces, ascending
    face_cells: np.ndarray         # [n_faces_local, 2] local cell ids
    recv: List[Tuple[int, int, int]] = field(default_factory=list)   # (src, offset, count)
    send: List[Tuple[int, np.ndarray]] = field(default_factory=list)  # (dst, local ids)

    @property
    def n_owned(self) -> int:
        return int(self.owned_ids.shape[0])

    @property
    def n_cells(self) -> int:
        return self.n_owned + int(self.halo_ids.shape[0])

    @property
    def cell_ids(self) -> np.ndarray:
        return np.concatenate([self.owned_ids, self.halo_ids])

    def split(self, reach=None):
        """(interior, rims, whole) cell ranges of the owned cells (see
        decomp.exchange_and_run); the interior reads no halo cell."""
        n_i, n_o = self.n_interior, self.n_owned
        rims = [(n_i, n_o)] if n_o > n_i else []
        if n_i == 0:
            return None, [(0, n_o)], (0, n_o)
        return (0, n_i), rims, (0, n_o)

    def check_adjoint(self):
        return None  # the two rings serve the reverse sweep as well

    def owned(self, x):
        return x[:self.n_owned]

    def local_cells(self, glob):
        """A local cell field (owned, then halo) cut from a global one."""
        return glob[_index_like(glob, self.cell_ids)]

    def local_faces(self, glob):
        """A local face field cut from a global one."""
        return glob[_index_like(glob, self.face_ids)]

    def reordered(self, cell_perm, face_perm) -> "GraphPart":
        """This part in the internal order of its local mesh, created with
        FL_RENUMBER: cell_perm[i] / face_perm[f] (fl_mesh_permutation) is the
        internal index of local cell i / face f.  The library reorders the
        interior and the rim among themselves and keeps the halo, so the
        receive slices stand; the send lists and the local ids follow."""
        cp = np.asarray(cell_perm, dtype=np.int64)
        fp = np.asarray(face_perm, dtype=np.int64)
        n_o = self.n_owned
        if not np.array_equal(cp[n_o:], np.arange(n_o, self.n_cells)):
            raise ValueError("the halo cells must keep their places")
        inv = np.empty_like(cp)
        inv[cp] = np.arange(cp.shape[0])
        invf = np.empty_like(fp)
        invf[fp] = np.arange(fp.shape[0])
        return GraphPart(rank=self.rank, world=self.world,
                         owned_ids=self.owned_ids[inv[:n_o]], n_interior=self.n_interior,
                         halo_ids=self.halo_ids, face_ids=self.face_ids[invf],
                         face_cells=cp[self.face_cells[invf]].astype(np.int32),
                         recv=list(self.recv),
                         send=[(d, cp[ids].astype(np.int32)) for d, ids in self.send])


def _index_like(x, ids):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return torch.as_tensor(ids, dtype=torch.long, device=x.device)
    except ImportError:
        pass
    return ids


def build_parts(n_cells: int, face_cells, part: np.ndarray, world: int = None) -> List[GraphPart]:
    """The local part of every rank for the partition ``part`` (ranks
    0 .. world - 1; by default the highest rank ``part`` names); a rank that
    owns no cell gets an empty part."""
    fc = np.asarray(face_cells, dtype=np.int64).reshape(-1, 2)
    if world is None:
        world = int(part.max()) + 1 if n_cells else 1
    ptr, nbr, fid = cell_graph(n_cells, fc)
    deg = np.diff(ptr)
    owner_of_edge = np.repeat(np.arange(n_cells), deg)
    parts = []
    halos = []
    for r in range(world):
        own = part == r
        # ring 1: other parts' cells next to an owned cell; ring 2: the other
        # cells of the ring-1 cells' faces
        e_own = own[owner_of_edge]
        ring1 = np.zeros(n_cells, dtype=bool)
        ring1[nbr[e_own & ~own[nbr]]] = True
        e_r1 = ring1[owner_of_edge]
        ring2 = np.zeros(n_cells, dtype=bool)
        ring2[nbr[e_r1]] = True
        ring2 &= ~own & ~ring1
        # rim: owned cells within two cells of a halo cell
        near1 = np.zeros(n_cells, dtype=bool)
        near1[owner_of_edge[e_own & ring1[nbr]]] = True
        near2 = near1.copy()
        e_n1 = near1[owner_of_edge]
        near2[nbr[e_n1]] = True
        rim = own & near2
        interior = own & ~rim
        owned_ids = np.concatenate([np.flatnonzero(interior), np.flatnonzero(rim)])
        halo_mask = ring1 | ring2
        hids = np.flatnonzero(halo_mask)
        hids = hids[np.lexsort((hids, part[hids]))]  # by owner part, then id
        halos.append(hids)
        local_ids = np.concatenate([owned_ids, hids])
        g2l = np.full(n_cells, -1, dtype=np.int64)
        g2l[local_ids] = np.arange(local_ids.shape[0])
        fmask = own[fc[:, 0]] | own[fc[:, 1]] | ring1[fc[:, 0]] | ring1[fc[:, 1]]
        fids = np.flatnonzero(fmask)
        lfc = g2l[fc[fids]]
        assert (lfc >= 0).all()
        parts.append(GraphPart(rank=r, world=world, owned_ids=owned_ids,
                               n_interior=int(interior.sum()), halo_ids=hids, face_ids=fids,
                               face_cells=lfc.astype(np.int32)))
    # exchange lists: what rank q receives from rank r is r's owned cells in
    # q's halo, in the order of q's halo group for r
    loc_in_owner = np.empty(n_cells, dtype=np.int64)  # index among its owner's cells
    for p in parts:
        loc_in_owner[p.owned_ids] = np.arange(p.n_owned)
    for q in range(world):
        hids = halos[q]
        src = part[hids]
        off = 0
        for r in range(world):
            cnt = int((src == r).sum())
            if cnt == 0:
                continue
            parts[q].recv.append((r, off, cnt))
            parts[r].send.append((q, loc_in_owner[hids[off:off + cnt]].astype(np.int32)))
            off += cnt
    for p in parts:
        p.send.sort(key=lambda t: t[0])
    return parts


def local_mesh_arrays(mesh, gp: GraphPart):
    """(n_cells, n_owned, n_interior, face_cells, normals, areas, volumes,
    distances or None) of the local mesh of part ``gp`` cut from a global
    face-based mesh with the attributes of workloads.Mesh."""
    nrm = np.asarray(mesh.normals, dtype=np.float64).reshape(-1, 3)[gp.face_ids]
    ar = np.asarray(mesh.areas, dtype=np.float64)[gp.face_ids]
    vol = np.asarray(mesh.volumes, dtype=np.float64)[gp.cell_ids]
    dist = getattr(mesh, "distances", None)
    if dist is not None:
        dist = np.asarray(dist, dtype=np.float64)[gp.face_ids]
    return gp.n_cells, gp.n_owned, gp.n_interior, gp.face_cells, nrm, ar, vol, dist


# ------------------------------------------------------------------ exchange
class LocalGraphTransport:
    """Exchange for a single part: it has no halo."""

    def exchange(self, gp: GraphPart, x):
        if gp.halo_ids.shape[0]:
            raise ValueError("a single part has no neighbour to exchange with")

    def start(self, gp: GraphPart, x):
        from .decomp import _Done
        self.exchange(gp, x)
        return _Done()


class GraphTransport:
    """Exchange through the default torch.distributed process group.
    ``pack(x, index, out)`` gathers x[index] into out: the library's
    fl_halo_pack for device fields (see GraphRollout), an index copy on the
    host."""

    TAG = 21

    def __init__(self, pack=None, index_device=None):
        self.pack = pack or _host_pack
        self.index_device = index_device
        self._idx = {}
        self._buf = {}

    def exchange(self, gp: GraphPart, x):
        self.start(gp, x).wait()

    def start(self, gp: GraphPart, x):
        import torch
        import torch.distributed as dist

        from .decomp import _Pending
        ops = []
        for dst, ids in gp.send:
            key = (id(gp), dst, x.dtype, x.device)
            if key not in self._idx:
                self._idx[key] = torch.as_tensor(ids, dtype=torch.int32,
                                                 device=self.index_device or x.device)
                self._buf[key] = torch.empty(ids.shape[0], dtype=x.dtype, device=x.device)
            buf = self._buf[key]
            self.pack(x, self._idx[key], buf)
            ops.append(dist.P2POp(dist.isend, buf, dst, tag=self.TAG))
        n0 = gp.n_owned
        for src, off, cnt in gp.recv:
            ops.append(dist.P2POp(dist.irecv, x[n0 + off:n0 + off + cnt], src, tag=self.TAG))
        if not ops:
            from .decomp import _Done
            return _Done()
        return _Pending(dist.batch_isend_irecv(ops))


def _host_pack(x, index, out):
    out.copy_(x[index.long()])


class ThreadGroupGraphTransport:
    """The exchange of ``world`` parts run in one process on one GPU, one
    host thread per part (tests and single-GPU measurement).  A part's halo
    slice from neighbour r is gathered straight from r's field by
    fl_halo_pack on r's local mesh, between two barriers; every launch goes
    to the one stream in order, so no kernel waits on another.  Register
    every part's GraphRollout before the threads start."""

    def __init__(self, world):
        import threading
        self.world = world
        self.reg = [None] * world
        self.fields = [None] * world
        self.bar = threading.Barrier(world)
        self._idx = {}

    def register(self, rollout):
        self.reg[rollout.gp.rank] = rollout

    def exchange(self, gp: GraphPart, x):
        import torch

        from . import fl_halo_pack
        self.fields[gp.rank] = x
        self.bar.wait()  # every part's stage input is enqueued and registered
        n0 = gp.n_owned
        for src, off, cnt in gp.recv:
            ro = self.reg[src]
            key = (src, gp.rank)
            if key not in self._idx:
                self._idx[key] = torch.as_tensor(dict(ro.gp.send)[gp.rank], dtype=torch.int32,
                                                 device=x.device)
            fl_halo_pack(ro.mesh.handle, x.dtype, self.fields[src], self._idx[key], cnt,
                         x[n0 + off:n0 + off + cnt])
        self.bar.wait()  # every gather is enqueued before any part's next stage


# ---------------------------------------------------- a rank's rollout (GPU)
class GraphRollout:
    """A rank's part of a partitioned rollout on the GPU: the local mesh
    (fl_mesh_create_local), its face velocities (and, in FP64, the
    pre-scaled velocity fl_step_rk uses), and the library's cell-range stage
    kernels; the halo goes through fl_halo_pack and torch.distributed.
    ``renumber`` lets the library reorder the interior and the rim into
    compact blocks (the part's lists follow its internal order); without it
    the owned cells give the whole mesh's bits."""

    def __init__(self, mesh, gp: GraphPart, u_global, limiter, dtype, dt, transport=None,
                 overlap=True, renumber=False):
        import torch

        from . import (FL_RENUMBER, Mesh, fl_halo_pack, fl_mesh_create_local,
                       fl_mesh_permutation, fl_velocity_prescale)
        C, n_o, n_i, fcl, nrm, ar, vol, dist = local_mesh_arrays(mesh, gp)
        self.mesh = Mesh(fl_mesh_create_local(C, n_o, n_i, fcl, nrm, ar, vol, dist,
                                              FL_RENUMBER if renumber else 0))
        if renumber:
            # fields are built in the library's internal order directly
            cp, fp, _ = fl_mesh_permutation(self.mesh.handle)
            gp = gp.reordered(cp, fp)
        self.gp = gp
        self.u = gp.local_faces(u_global).to(dtype).contiguous()
        self.w = None
        if dtype == torch.float64 and dt > 0:
            self.w = torch.empty_like(self.u)
            fl_velocity_prescale(self.mesh.handle, dtype, dt, self.u, self.w)
        self.limiter, self.dtype, self.dt = limiter, dtype, dt
        if transport is None:
            h = self.mesh.handle
            transport = GraphTransport(pack=lambda x, idx, out: fl_halo_pack(
                h, x.dtype, x, idx, idx.numel(), out))
        self.transport = transport
        self.overlap = overlap

    def local_field(self, theta_global):
        return self.gp.local_cells(theta_global).to(self.dtype).contiguous()

    def _stage_fn(self, rk_order):
        from . import fl_step_rk_stage_cells

        def stage(s, thn, x, y, c0, c1):
            fl_step_rk_stage_cells(self.mesh.handle, self.limiter, self.dtype, rk_order, s,
                                   self.dt, c0, c1, thn, x, y, self.u, self.w)

        return stage

    def step(self, theta_local, rk_order, nsteps):
        import torch

        from .decomp import step_rk
        a = torch.empty_like(theta_local)
        b = torch.empty_like(theta_local) if rk_order == 3 else None
        return step_rk(self.gp, self.transport, self._stage_fn(rk_order), rk_order, nsteps,
                       theta_local, a, b, overlap=self.overlap)

    def gradient(self, theta_local, lam_T_local, rk_order, nsteps, every):
        """dJ/dtheta_0 on this rank's owned cells (decomp.gradient_rk)."""
        import torch

        from . import fl_step_rk_stage_adjoint_cells
        from .decomp import gradient_rk

        def stage_adjoint(s, x, mu, lam_a, lam_b, out, c0, c1):
            fl_step_rk_stage_adjoint_cells(self.mesh.handle, self.limiter, self.dtype, rk_order,
                                           s, self.dt, c0, c1, x, mu, lam_a, lam_b, out, self.u,
                                           self.w)

        return gradient_rk(self.gp, self.transport, self._stage_fn(rk_order), stage_adjoint,
                           rk_order, nsteps, every, theta_local, lam_T_local,
                           lambda: torch.empty_like(theta_local), overlap=self.overlap)

    def mass(self, theta_local):
        """sum_c V_c theta_c over the whole mesh: this rank's owned cells
        (fl_reduce_mass on the local mesh) summed over the ranks."""
        import torch

        from . import fl_reduce_mass, fl_reduce_workspace_size
        from .replicas import sum_over_ranks
        ws = torch.empty(max(fl_reduce_workspace_size(), 1), dtype=torch.uint8,
                         device=theta_local.device)
        return sum_over_ranks(fl_reduce_mass(self.mesh.handle, self.dtype, theta_local, ws),
                              theta_local.device)

    def max_abs_velocity(self):
        """max_f |u_f| over the whole mesh: this rank's local faces, then the
        maximum over the ranks."""
        from .decomp import _max_abs_faces
        return _max_abs_faces(self.u)

    def close(self):
        self.mesh.close()


__all__ = ["cell_graph", "partition_graph", "GraphPart", "build_parts", "local_mesh_arrays",
           "LocalGraphTransport", "GraphTransport", "ThreadGroupGraphTransport", "GraphRollout"]
