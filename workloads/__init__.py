"""Seeded synthetic inputs for the flux-limited convection path.

This module only *describes* inputs: mesh topology/geometry as plain arrays,
velocity fields on faces, initial scalar fields and targets.  It contains none
of the limiter / flux / time-step arithmetic, so both the CPU oracle and the
CUDA library can consume what it produces without sharing any of the method.

Conventions shared by every generator (they describe the data, not the method):

* Structured periodic box ``nx x ny x nz`` with spacings ``hx, hy, hz``; cell
  ``c = i + nx*(j + ny*k)``, centre ``((i+1/2)hx, (j+1/2)hy, (k+1/2)hz)``.
* Faces exist only along axes whose extent is > 1.  For each such axis (x, y, z
  in that order) there is one block of ``|C|`` faces; face ``axis_block*|C| + c``
  sits between ``c0 = c`` and ``c1 = c + e_axis`` (periodic wrap) and its unit
  normal is ``+e_axis`` (points from c0 to c1).
* ``u_f`` is the normal velocity component along the stored normal.

The velocity fields are built as discrete curls of a vector potential sampled
on mesh edges, so the face fluxes are divergence-free cell by cell up to
round-off (each edge sample enters two faces of every cell with opposite sign).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    """Explicit face-based mesh description (host arrays, user ordering)."""

    n_cells: int
    face_cells: np.ndarray  # int32 [F, 2]  (c0, c1); normal points c0 -> c1
    normals: np.ndarray  # float64 [F, 3] unit normals
    areas: np.ndarray  # float64 [F]
    volumes: np.ndarray  # float64 [C]
    dims: tuple | None = None  # (nx, ny, nz) for structured meshes
    h: tuple | None = None  # (hx, hy, hz)
    extra: dict = field(default_factory=dict)
    distances: np.ndarray | None = None  # float64 [F]: c0-c1 centre distance
                                         # (non-uniform meshes; None = uniform)

    @property
    def n_faces(self) -> int:
        if self.face_cells is None:  # a structured box given by dims and h only
            return int(self.n_cells) * len(active_axes(self.dims))
        return int(self.face_cells.shape[0])


def active_axes(dims):
    return [a for a in range(3) if dims[a] > 1]


def structured_mesh(nx: int, ny: int = 1, nz: int = 1, hx: float = 1.0,
                    hy: float = 1.0, hz: float = 1.0) -> Mesh:
    """Periodic structured box written out as explicit face arrays."""
    dims = (nx, ny, nz)
    n = nx * ny * nz
    c = np.arange(n, dtype=np.int64)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    hs = (hx, hy, hz)
    fc, nrm, ar = [], [], []
    for a in active_axes(dims):
        if a == 0:
            nb = ((i + 1) % nx) + nx * (j + ny * k)
        elif a == 1:
            nb = i + nx * (((j + 1) % ny) + ny * k)
        else:
            nb = i + nx * (j + ny * ((k + 1) % nz))
        fc.append(np.stack([c, nb], axis=1))
        nv = np.zeros((n, 3))
        nv[:, a] = 1.0
        nrm.append(nv)
        others = [hs[b] for b in range(3) if b != a]
        ar.append(np.full(n, others[0] * others[1]))
    if fc:
        face_cells = np.concatenate(fc).astype(np.int32)
        normals = np.concatenate(nrm)
        areas = np.concatenate(ar)
    else:
        face_cells = np.zeros((0, 2), np.int32)
        normals = np.zeros((0, 3))
        areas = np.zeros(0)
    volumes = np.full(n, hx * hy * hz)
    return Mesh(n, face_cells, normals, areas, volumes, dims=dims, h=hs)


def structured_box(nx: int, ny: int = 1, nz: int = 1, hx: float = 1.0, hy: float = 1.0,
                   hz: float = 1.0) -> Mesh:
    """A periodic structured box by its sizes and spacings only, without the
    explicit face arrays of structured_mesh (which take 40 bytes per face:
    23 GB at 576^3).  For the GPU library, which needs dims and h alone; the
    oracle needs structured_mesh."""
    return Mesh(nx * ny * nz, None, None, None, None, dims=(nx, ny, nz), h=(hx, hy, hz))


def stretched_mesh(wx, wy=(1.0,), wz=(1.0,)) -> Mesh:
    """Periodic tensor-product box with cell widths ``wx`` [nx], ``wy`` [ny],
    ``wz`` [nz] along the axes, as explicit face arrays with the face
    distances of a non-uniform mesh: the face between cells i and i+1 along
    an axis has distance (w_i + w_{i+1}) / 2 (periodic)."""
    wx, wy, wz = (np.asarray(w, dtype=np.float64) for w in (wx, wy, wz))
    nx, ny, nz = len(wx), len(wy), len(wz)
    dims = (nx, ny, nz)
    n = nx * ny * nz
    c = np.arange(n, dtype=np.int64)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    ws = (wx[i], wy[j], wz[k])
    widths = (wx, wy, wz)
    idx = (i, j, k)
    fc, nrm, ar, dist = [], [], [], []
    for a in active_axes(dims):
        if a == 0:
            nb = ((i + 1) % nx) + nx * (j + ny * k)
        elif a == 1:
            nb = i + nx * (((j + 1) % ny) + ny * k)
        else:
            nb = i + nx * (j + ny * ((k + 1) % nz))
        fc.append(np.stack([c, nb], axis=1))
        nv = np.zeros((n, 3))
        nv[:, a] = 1.0
        nrm.append(nv)
        others = [ws[b] for b in range(3) if b != a]
        ar.append(others[0] * others[1])
        w = widths[a]
        dist.append(0.5 * (w[idx[a]] + w[(idx[a] + 1) % dims[a]]))
    if fc:
        face_cells = np.concatenate(fc).astype(np.int32)
        normals = np.concatenate(nrm)
        areas = np.concatenate(ar)
        distances = np.concatenate(dist)
    else:
        face_cells = np.zeros((0, 2), np.int32)
        normals = np.zeros((0, 3))
        areas = np.zeros(0)
        distances = np.zeros(0)
    volumes = ws[0] * ws[1] * ws[2]
    return Mesh(n, face_cells, normals, areas, volumes, dims=dims, distances=distances)


def stretched_widths(n, length, ratio, seed):
    """``n`` seeded cell widths summing to ``length`` whose largest / smallest
    ratio is at most ``ratio`` (a smooth stretching plus seeded jitter)."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    base = 1.0 + 0.5 * (ratio - 1.0) * (1.0 + np.sin(2.0 * np.pi * x))
    w = base * rng.uniform(0.9, 1.1, n)
    w = np.clip(w, 1.0, ratio)
    return w * (length / w.sum())


# --------------------------------------------------------------------------
# general (non-hexahedral) periodic meshes
# --------------------------------------------------------------------------
def _lattice_id(v, n):
    v = np.mod(v, n)
    return v[..., 0] + n * (v[..., 1] + n * v[..., 2])


def _box_origins(n):
    o = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    return o.transpose(2, 1, 0, 3).reshape(-1, 3)  # x fastest


def polyhedral_mesh(n, h, face_groups, volumes):
    """Face-based periodic mesh of the box [0, n h)^3 from cells given by
    their faces: ``face_groups`` is a list of (cell index [m], polygon
    vertices [m, nv, 3]) in integer lattice coordinates (unwrapped, so each
    polygon is geometrically intact).  Faces are matched by their wrapped
    vertex sets; every face must be shared by exactly two cells.  The normal
    is the unit Newell normal, oriented from c0 (first occurrence) to c1."""
    c0s, c1s, nrms, areas = [], [], [], []
    centroid_sum = np.zeros((len(volumes), 3))
    centroid_cnt = np.zeros(len(volumes))
    for cells, poly in face_groups:
        np.add.at(centroid_sum, cells, poly.mean(axis=1) * h)
        np.add.at(centroid_cnt, cells, 1.0)
    cen = centroid_sum / centroid_cnt[:, None]
    for cells, poly in face_groups:
        m, nv, _ = poly.shape
        keys = np.sort(_lattice_id(poly, n), axis=1)
        _, inv, cnt = np.unique(keys, axis=0, return_inverse=True, return_counts=True)
        inv = inv.ravel()
        if not np.all(cnt == 2):
            raise ValueError("a face is not shared by exactly two cells")
        order = np.argsort(inv, kind="stable")
        first, second = order[0::2], order[1::2]
        P = poly[first].astype(np.float64) * h
        nrm = np.zeros((len(first), 3))
        for a in range(nv):
            p, q = P[:, a], P[:, (a + 1) % nv]
            nrm[:, 0] += (p[:, 1] - q[:, 1]) * (p[:, 2] + q[:, 2])
            nrm[:, 1] += (p[:, 2] - q[:, 2]) * (p[:, 0] + q[:, 0])
            nrm[:, 2] += (p[:, 0] - q[:, 0]) * (p[:, 1] + q[:, 1])
        a2 = np.linalg.norm(nrm, axis=1)
        unit = nrm / a2[:, None]
        c0 = cells[first]
        outward = np.einsum("ij,ij->i", unit, P.mean(axis=1) - cen[c0]) > 0
        unit[~outward] *= -1.0
        unit[unit == 0.0] = 0.0  # no negative zeros
        c0s.append(c0)
        c1s.append(cells[second])
        nrms.append(unit)
        areas.append(0.5 * a2)
    fc = np.stack([np.concatenate(c0s), np.concatenate(c1s)], axis=1).astype(np.int32)
    return Mesh(len(volumes), fc, np.concatenate(nrms), np.concatenate(areas),
                np.asarray(volumes, dtype=np.float64))


def tet_mesh(n, h=None):
    """Periodic box of n^3 cubes, each split into the 6 tetrahedra of the
    Kuhn (Freudenthal) triangulation around its main diagonal, which match
    across cube faces: 6 n^3 cells with 4 triangular faces each."""
    h = 1.0 / n if h is None else h
    e = np.eye(3, dtype=np.int64)
    tets = []
    for p in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        v1 = e[p[0]]
        v2 = v1 + e[p[1]]
        tets.append(np.stack([np.zeros(3, dtype=np.int64), v1, v2, np.ones(3, dtype=np.int64)]))
    tets = np.stack(tets)                                       # [6, 4, 3]
    o = _box_origins(n)
    verts = (o[:, None, None, :] + tets[None]).reshape(-1, 4, 3)
    nc = verts.shape[0]
    poly = np.stack([verts[:, [1, 2, 3]], verts[:, [0, 2, 3]], verts[:, [0, 1, 3]],
                     verts[:, [0, 1, 2]]], axis=1).reshape(-1, 3, 3)
    cells = np.repeat(np.arange(nc), 4)
    return polyhedral_mesh(n, h, [(cells, poly)], np.full(nc, h ** 3 / 6.0))


def prism_mesh(n, h=None):
    """Periodic box of n^3 cubes, each split along its xy diagonal into two
    triangular prisms: 2 n^3 cells with 2 triangular and 3 quadrilateral
    faces each (axis-aligned and diagonal quads)."""
    h = 1.0 / n if h is None else h
    tris = np.array([[[0, 0], [1, 0], [1, 1]], [[0, 0], [1, 1], [0, 1]]], dtype=np.int64)
    o = _box_origins(n)
    nc = 2 * o.shape[0]
    tri_polys, quad_polys, tri_cells, quad_cells = [], [], [], []
    for t in range(2):
        base = np.concatenate([tris[t], np.zeros((3, 1), dtype=np.int64)], axis=1)   # z = 0
        top = base + np.array([0, 0, 1])
        cell = 2 * np.arange(o.shape[0]) + t
        tri_polys += [o[:, None, :] + base[None], o[:, None, :] + top[None]]
        tri_cells += [cell, cell]
        for a in range(3):
            b = (a + 1) % 3
            q = np.stack([base[a], base[b], top[b], top[a]])
            quad_polys.append(o[:, None, :] + q[None])
            quad_cells.append(cell)
    groups = [(np.concatenate(tri_cells), np.concatenate(tri_polys)),
              (np.concatenate(quad_cells), np.concatenate(quad_polys))]
    return polyhedral_mesh(n, h, groups, np.full(nc, h ** 3 / 2.0))


def permuted_mesh(mesh: Mesh, seed: int, flip_fraction: float = 0.5):
    """Relabel cells and faces with seeded random permutations and flip the
    orientation of a seeded subset of faces (c0<->c1, normal negated).

    Returns ``(new_mesh, cell_perm, face_perm, flip)`` where
    ``new_cell_id = cell_perm[old_cell_id]`` and the new face ``face_perm[f]``
    is old face ``f``; ``flip[f]`` tells whether old face ``f`` was flipped.
    Fields map as ``theta_new[cell_perm] = theta_old`` and
    ``u_new[face_perm] = where(flip, -u_old, u_old)``.
    """
    rng = np.random.default_rng(seed)
    C, F = mesh.n_cells, mesh.n_faces
    cell_perm = rng.permutation(C).astype(np.int64)
    face_perm = rng.permutation(F).astype(np.int64)
    flip = rng.random(F) < flip_fraction
    fc = cell_perm[mesh.face_cells.astype(np.int64)]
    fc = np.where(flip[:, None], fc[:, ::-1], fc)
    nrm = np.where(flip[:, None], -mesh.normals, mesh.normals)
    new_fc = np.empty_like(fc)
    new_fc[face_perm] = fc
    new_n = np.empty_like(nrm)
    new_n[face_perm] = nrm
    new_a = np.empty_like(mesh.areas)
    new_a[face_perm] = mesh.areas
    new_v = np.empty_like(mesh.volumes)
    new_v[cell_perm] = mesh.volumes
    new_d = None
    if mesh.distances is not None:
        new_d = np.empty_like(mesh.distances)
        new_d[face_perm] = mesh.distances
    out = Mesh(C, new_fc.astype(np.int32), new_n, new_a, new_v, distances=new_d)
    return out, cell_perm, face_perm, flip


def permute_cell_field(theta, cell_perm):
    out = np.empty_like(theta)
    out[cell_perm] = theta
    return out


def permute_face_field(u, face_perm, flip):
    out = np.empty_like(u)
    out[face_perm] = np.where(flip, -u, u)
    return out


# --------------------------------------------------------------------------
# velocity fields (discrete curl of an edge-sampled vector potential)
# --------------------------------------------------------------------------
def _coords(dims, h):
    nx, ny, nz = dims
    hx, hy, hz = h
    c = np.arange(nx * ny * nz, dtype=np.int64)
    i = (c % nx).astype(np.float64)
    j = ((c // nx) % ny).astype(np.float64)
    k = (c // (nx * ny)).astype(np.float64)
    return i, j, k, hx, hy, hz


def _coords_b(dims, h):
    """The cell indices i, j, k as broadcastable float arrays of shapes
    (1, 1, nx), (1, ny, 1), (nz, 1, 1): element-wise expressions of them give
    the (nz, ny, nx) field of the flat arrays of _coords, value for value, with
    one full-size array per result instead of one per coordinate."""
    nx, ny, nz = dims
    i = np.arange(nx, dtype=np.float64).reshape(1, 1, nx)
    j = np.arange(ny, dtype=np.float64).reshape(1, ny, 1)
    k = np.arange(nz, dtype=np.float64).reshape(nz, 1, 1)
    return i, j, k, h[0], h[1], h[2]


def _full(a, dims):
    nx, ny, nz = dims
    return np.broadcast_to(a, (nz, ny, nx)).ravel()


def curl_face_velocity(dims, h, potential):
    """Face normal velocities ``u_f`` (layout of :func:`structured_mesh`) from the
    discrete curl of a vector potential ``A = potential(axis, x, y, z)``.

    A_x lives on x-edges (x_i, y_{j+1/2}, z_{k+1/2}), A_y on y-edges
    (x_{i+1/2}, y_j, z_{k+1/2}), A_z on z-edges (x_{i+1/2}, y_{j+1/2}, z_k);
    the flux through a face is the circulation of A around its four edges
    (Stokes), divided by the face area.
    """
    # the coordinates broadcast over the (nz, ny, nx) grid (the potentials are
    # element-wise, so each value is the flat evaluation's, bit for bit)
    i, j, k, hx, hy, hz = _coords_b(dims, h)
    xc, yc, zc = (i + 0.5) * hx, (j + 0.5) * hy, (k + 0.5) * hz
    xp, yp, zp = (i + 1.0) * hx, (j + 1.0) * hy, (k + 1.0) * hz
    xm, ym, zm = i * hx, j * hy, k * hz
    A = potential
    out = []
    axes = active_axes(dims)
    if 0 in axes:  # x-face (x_{i+1/2}, y_j, z_k): dAz/dy - dAy/dz
        circ = (hz * (A(2, xp, yp, zc) - A(2, xp, ym, zc))
                - hy * (A(1, xp, yc, zp) - A(1, xp, yc, zm)))
        out.append(_full(circ / (hy * hz), dims))
    if 1 in axes:  # y-face (x_i, y_{j+1/2}, z_k): dAx/dz - dAz/dx
        circ = (hx * (A(0, xc, yp, zp) - A(0, xc, yp, zm))
                - hz * (A(2, xp, yp, zc) - A(2, xm, yp, zc)))
        out.append(_full(circ / (hx * hz), dims))
    if 2 in axes:  # z-face (x_i, y_j, z_{k+1/2}): dAy/dx - dAx/dy
        circ = (hy * (A(1, xp, yc, zp) - A(1, xm, yc, zp))
                - hx * (A(0, xc, yp, zp) - A(0, xc, ym, zp)))
        out.append(_full(circ / (hx * hy), dims))
    return np.concatenate(out) if out else np.zeros(0)


def taylor_green_potential(axis, x, y, z):
    """Stream function psi = sin x sin y cos z as the z-component of A; its
    curl is the Taylor-Green field (sin x cos y cos z, -cos x sin y cos z, 0)."""
    if axis != 2:
        return np.zeros_like(x)
    return np.sin(x) * np.sin(y) * np.cos(z)


def fourier_potential(rng, n_modes=8, kmax=4):
    """Random vector potential: ``n_modes`` Fourier modes with integer wave
    vectors in {-kmax..kmax}^3 minus 0, N(0,1) amplitudes per component and
    U(0, 2pi) phases."""
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, 3)
        if np.any(k != 0):
            ks.append(k.astype(np.float64))
    amps = rng.normal(0.0, 1.0, (n_modes, 3))
    phases = rng.uniform(0.0, TWO_PI, n_modes)

    def A(axis, x, y, z):
        s = np.zeros_like(x)
        for m in range(n_modes):
            s = s + amps[m, axis] * np.sin(ks[m][0] * x + ks[m][1] * y + ks[m][2] * z + phases[m])
        return s

    return A


# --------------------------------------------------------------------------
# scalar fields
# --------------------------------------------------------------------------
def sine_sum_field(dims, h, rng, n_modes=4, kmax=3, amp=0.25):
    i, j, k, hx, hy, hz = _coords(dims, h)
    x, y, z = (i + 0.5) * hx, (j + 0.5) * hy, (k + 0.5) * hz
    th = np.zeros(x.shape)
    for _ in range(n_modes):
        while True:
            kv = rng.integers(-kmax, kmax + 1, 3)
            if np.any(kv != 0):
                break
        a = rng.uniform(0.0, amp)
        ph = rng.uniform(0.0, TWO_PI)
        th = th + a * np.sin(kv[0] * x + kv[1] * y + kv[2] * z + ph)
    return th


def cube_step(dims, h, lo=0.5 * math.pi, hi=1.5 * math.pi):
    i, j, k, hx, hy, hz = _coords(dims, h)
    x, y, z = (i + 0.5) * hx, (j + 0.5) * hy, (k + 0.5) * hz
    inside = (x >= lo) & (x <= hi) & (y >= lo) & (y <= hi) & (z >= lo) & (z <= hi)
    return inside.astype(np.float64)


def sine_plus_cube(dims, h, seed):
    rng = np.random.default_rng(seed)
    return sine_sum_field(dims, h, rng) + cube_step(dims, h)


def max_abs(u):
    return float(np.max(np.abs(u))) if u.size else 0.0


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mesh: Mesh
    theta0: np.ndarray
    u: np.ndarray
    dt: float
    nsteps: int
    rk_order: int
    limiter: str
    extra: dict = field(default_factory=dict)


def config_1d(n=1000, seed=0):
    """1D periodic advection: N uniform cells of width 1/N, u = 1, square wave
    (1 on [0.25, 0.5]) plus a Gaussian bump at 0.75, CFL 0.5, forward Euler,
    van Leer, 1000 steps."""
    h = 1.0 / n
    mesh = structured_mesh(n, 1, 1, h, 1.0, 1.0)
    x = (np.arange(n) + 0.5) * h
    th = ((x >= 0.25) & (x <= 0.5)).astype(np.float64) + np.exp(-((x - 0.75) / 0.05) ** 2)
    u = np.ones(n)
    return Workload("1d_n%d_vanleer_euler" % n, mesh, th, u, 0.5 * h, 1000, 1, "vanleer")


def config_taylor_green(n=256, seed=1, cfl=0.4, nsteps=100, limiter="superbee"):
    """3D periodic cube n^3 on [0, 2pi]^3, Taylor-Green velocity from the
    discrete curl of an edge-sampled stream function, sine-sum plus cube-step
    scalar, SSP-RK3 at CFL 0.4."""
    h = TWO_PI / n
    mesh = structured_mesh(n, n, n, h, h, h)
    u = curl_face_velocity((n, n, n), (h, h, h), taylor_green_potential)
    th = sine_plus_cube((n, n, n), (h, h, h), seed)
    dt = cfl * h / max_abs(u)
    return Workload("tg%d" % n, mesh, th, u, dt, nsteps, 3, limiter)


def deformation_potential(n):
    """Vector potential of the reversing 3D deformation flow of Section 4.1
    (eq. rhodonea) on [0, 1]^3 at t = 0:
        A = (0, -sin^2(pi x) sin(2 pi y) sin^2(pi z) / pi,
                 sin^2(pi x) sin^2(pi y) sin(2 pi z) / pi),
    whose curl is the paper's (u, v, w) without the factor cos(pi t / T).
    Sample coordinates are snapped to the n-cell half-integer lattice and
    wrapped into [0, 1), so every sample on the periodic seam is exactly zero
    and no discrete flux crosses the domain boundary."""
    def snap(x):
        return np.mod(np.rint(2.0 * x * n) / 2.0, n) / n

    def A(axis, x, y, z):
        if axis == 0:
            return np.zeros_like(x)
        xs, ys, zs = snap(x), snap(y), snap(z)
        sx, sy, sz = np.sin(math.pi * xs), np.sin(math.pi * ys), np.sin(math.pi * zs)
        if axis == 1:
            return -(sx * sx) * np.sin(TWO_PI * ys) * (sz * sz) / math.pi
        return (sx * sx) * (sy * sy) * np.sin(TWO_PI * zs) / math.pi
    return A


def sphere_indicator(n, centre=(0.35, 0.35, 0.35), radius=0.15):
    """1 in the cells of [0, 1]^3 (n^3) whose centre lies in the sphere, else 0."""
    h = 1.0 / n
    i, j, k, _, _, _ = _coords_b((n, n, n), (h, h, h))
    x, y, z = (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return _full(r2 <= radius * radius, (n, n, n)).astype(np.float64)


def max_outflow_rate(dims, h, u):
    """max over cells of sum_{outflow faces} |u_f| A_f / V_c (1 / time units)
    for a structured mesh's face velocities (layout of structured_mesh)."""
    nx, ny, nz = dims
    C = nx * ny * nz
    rate = np.zeros((nz, ny, nx))
    for b, ax in enumerate(active_axes(dims)):
        uf = u[b * C:(b + 1) * C].reshape(nz, ny, nx)
        roll_axis = 2 - ax  # x varies fastest
        out_plus = np.maximum(uf, 0.0)                          # through the + face
        out_minus = np.maximum(-np.roll(uf, 1, axis=roll_axis), 0.0)  # through the - face
        rate += (out_plus + out_minus) / h[ax]
    return float(rate.max())


def modulation_factors(nsteps, dt, rk, period, t0=0.0):
    """cos(pi t / T) at the stage times of nsteps Euler (t_n) or SSP-RK3
    (t_n, t_n + dt, t_n + dt / 2) steps, flattened as [n * stages + s]."""
    t = t0 + dt * np.arange(nsteps, dtype=np.float64)
    if rk == 1:
        st = t[:, None]
    else:
        st = np.stack([t, t + dt, t + 0.5 * dt], axis=1)
    return np.cos(math.pi * st / period).ravel()


def config_deformation(n=72, courant=0.5, period=3.0, rk=1, limiter="superbee", faces=True):
    """Section 4.1: a sphere (r = 0.15 at (0.35, 0.35, 0.35)) in [0, 1]^3 on
    n^3 hexahedra, deformed by eq. rhodonea for t in [0, T], T = 3, forward
    Euler (Algorithm 5) with superbee.  The velocity at time t is
    cos(pi t / T) u_f with u_f the discrete curl of deformation_potential;
    dt makes the largest per-cell outflow Courant number `courant` and divides
    T into a whole number of steps (the flow reverses, so theta(T) returns
    to the sphere up to the scheme's error).  faces=False leaves out the
    explicit face arrays (structured_box: for the GPU alone, large n)."""
    h = 1.0 / n
    mesh = structured_mesh(n, n, n, h, h, h) if faces else structured_box(n, n, n, h, h, h)
    u = curl_face_velocity((n, n, n), (h, h, h), deformation_potential(n))
    th = sphere_indicator(n)
    dt = courant / max_outflow_rate((n, n, n), (h, h, h), u)
    nsteps = int(math.ceil(period / dt))
    dt = period / nsteps
    return Workload("deformation%d" % n, mesh, th, u, dt, nsteps, rk, limiter,
                    extra={"period": period, "g": modulation_factors(nsteps, dt, rk, period)})


def batched_box_dims(n_boxes=64, seed=3, lo=32, hi=128):
    rng = np.random.default_rng(seed)
    return [tuple(int(v) for v in d) for d in rng.integers(lo, hi + 1, (n_boxes, 3))]


def random_box(dims, seed, cfl=0.4):
    """One batched instance: periodic box [0, 2pi]^3 with its own solenoidal
    velocity (curl of an 8-mode Fourier potential, normalised to max|u_f| = 1)
    and its own sine-plus-cube scalar."""
    rng = np.random.default_rng(seed)
    h = tuple(TWO_PI / d for d in dims)
    mesh = structured_mesh(*dims, *h)
    A = fourier_potential(rng)
    u = curl_face_velocity(dims, h, A)
    u = u / max_abs(u)
    th = sine_sum_field(dims, h, rng) + cube_step(dims, h)
    dt = cfl * min(h) / max_abs(u)
    return mesh, th, u, dt


def smooth_target(dims, h, seed, n_modes=4, kmax=2):
    rng = np.random.default_rng(seed + 1000)
    return sine_sum_field(dims, h, rng, n_modes=n_modes, kmax=kmax, amp=0.5)


def random_field(n, seed, scale=1.0):
    return np.random.default_rng(seed).normal(0.0, scale, n)


# Values whose pairwise differences give the gradient ratio's exact edge
# cases: equal neighbours (d_u = 0, d_U = 0), ratios exactly on the limiters'
# kinks (1/5, 1/2, 1, 2, 5 and their negatives: e.g. 0, 1, 6 gives 1/5 and
# 0, 5, 6 gives 5), signed zeros, and subnormal neighbours of 0 whose
# difference makes r overflow to +-inf.
QUANTIZED_VALUES = (0.0, -0.0, 0.5, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, -1.0, -0.5)


def quantized_field(n, seed, dtype="f64", repeat=0.4):
    """Cell values drawn from QUANTIZED_VALUES plus +-1 and +2 smallest
    subnormals of the dtype; a fraction ``repeat`` of the cells copies the
    value of the cell before it (plateaus), so equal neighbours are common
    along every axis."""
    tiny = float(np.finfo(np.float64 if dtype == "f64" else np.float32).smallest_subnormal)
    vals = np.array(QUANTIZED_VALUES + (tiny, 2.0 * tiny, -tiny))
    rng = np.random.default_rng(seed)
    th = vals[rng.integers(0, len(vals), n)]
    rep = rng.random(n) < repeat
    for i in np.flatnonzero(rep):
        if i > 0:
            th[i] = th[i - 1]
    return th


def edge_velocity(n_faces, seed, scale=0.3):
    """Face velocities of both signs with exact +0 and -0 entries (both select
    the -1 side) among random magnitudes."""
    rng = np.random.default_rng(seed)
    u = scale * rng.uniform(-1.0, 1.0, n_faces)
    r = rng.random(n_faces)
    u[r < 0.08] = 0.0
    u[(r >= 0.08) & (r < 0.12)] = -0.0
    return u


def mixed_sign_velocity(n_faces, seed, zero_fraction=0.1):
    """Random face velocities with both signs and some exact zeros (and one
    negative zero) for upwind-selection tests."""
    rng = np.random.default_rng(seed)
    u = rng.normal(0.0, 1.0, n_faces)
    u[rng.random(n_faces) < zero_fraction] = 0.0
    if n_faces > 2:
        u[1] = -0.0
    return u
