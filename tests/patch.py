"""Local patches of a periodic Cartesian mesh, for checking full-size GPU
results cell by cell with the oracle: the cells within L-infinity distance
``radius`` of a centre cell, with every face between two patch cells.  Any
value the stencil computes at distance <= radius - 2*(stages) ... is exact."""
import numpy as np

import workloads as W


def patch(dims, h, centre, radius):
    nx, ny, nz = dims
    C = nx * ny * nz
    r = range(-radius, radius + 1)
    cells = []
    loc = {}
    for dk in r:
        for dj in r:
            for di in r:
                i = (centre[0] + di) % nx
                j = (centre[1] + dj) % ny
                k = (centre[2] + dk) % nz
                loc[(di, dj, dk)] = len(cells)
                cells.append(i + nx * (j + ny * k))
    axes = W.active_axes(dims)
    fc, nrm, ar, fidx = [], [], [], []
    for (di, dj, dk), lc in loc.items():
        for blk, a in enumerate(axes):
            nb = [di, dj, dk]
            nb[a] += 1
            nb = tuple(nb)
            if nb not in loc:
                continue
            fc.append((lc, loc[nb]))
            n = [0.0, 0.0, 0.0]
            n[a] = 1.0
            nrm.append(n)
            others = [h[b] for b in range(3) if b != a]
            ar.append(others[0] * others[1])
            fidx.append(blk * C + cells[lc])
    mesh = W.Mesh(len(cells), np.array(fc, np.int32), np.array(nrm), np.array(ar),
                  np.full(len(cells), h[0] * h[1] * h[2]))
    return mesh, np.array(cells), np.array(fidx), loc[(0, 0, 0)]
