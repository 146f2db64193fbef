"""The padded layout of the batched FP32 tile (decomposition kind 2,
fl_struct_pad4.cuh) restated on the host: for box shapes with rows that end
anywhere in a warp's run, planes of one row and boxes of one plane, every
load and store of the tile's index arithmetic stays inside the padded copy,
every neighbour a cell's stencil reads is written by the stage that produces
it (its own cells plus the ghost images) with the periodic image of the right
cell, and each cell is stored once at its own place.  This checks the layout
and its ghost-write rules; the kernel's arithmetic is checked on the GPU
against the oracle (tests/test_gpu_batched.py)."""
import random

import pytest

RUN, GX = 128, 2


def geom(nx, ny, nz):
    P = (nx + 4 + 3) // 4 * 4
    gy = 2 if ny > 1 else 0
    gz = 2 if nz > 1 else 0
    PY, PZ = ny + 2 * gy, nz + 2 * gz
    return P, PY, PZ, gy, gz


def pos_of(nx, ny, nz, i):
    """the (x, y, z) cell whose periodic image padded index i holds"""
    P, PY, PZ, gy, gz = geom(nx, ny, nz)
    xp = i % P
    t = i // P
    yp, zp = t % PY, t // PY
    return ((xp - GX) % nx, (yp - gy) % ny, (zp - gz) % nz)


def run(nx, ny, nz, W, zchunk):
    """errors of one box shape and tiling (empty when the layout holds)"""
    P, PY, PZ, gy, gz = geom(nx, ny, nz)
    PP = P * PY
    vol = PP * PZ
    rows = ny * P
    tiles_x = -(-rows // (RUN * W))
    act_y, act_z = ny > 1, nz > 1
    errs = []
    written = {}  # padded index -> (x, y, z) cell whose value is stored there

    def chk(i, what):
        if not 0 <= i < vol:
            errs.append((what, i, vol))
    reads = []  # (padded index, expected image) for valid cells
    for seg in range(tiles_x):
        for zc in range(-(-nz // zchunk)):
            z0 = zc * zchunk
            z1 = min(z0 + zchunk, nz)
            for w in range(W):
                run0 = (seg * W + w) * RUN
                if run0 >= rows:
                    continue
                for lane in range(32):
                    live = run0 + 4 * lane < rows
                    f0 = run0 + 4 * lane if live else rows - 4
                    yrow, c0 = divmod(f0, P)
                    xb = c0 - GX
                    val = [live and 0 <= xb + v < nx for v in range(4)]
                    ybase = gy * P + f0
                    at = lambda kz: (kz + gz) * PP + ybase
                    # init loads
                    for v in range(4):
                        chk(at(z0) + v, 'init')
                    if act_z:
                        for dz in (-2, -1, 1, 2):
                            for v in range(4):
                                chk(at(z0 + dz) + v, 'initz')
                    for k in range(z0, z1):
                        o = at(k)
                        more = k + 1 < z1
                        ld = [o]
                        if act_z and more:
                            ld.append(o + 3 * PP)
                        if act_y:
                            ld += [o - 2 * P, o - P, o + P, o + 2 * P]
                        for b in ld:
                            for v in range(4):
                                chk(b + v, 'load')
                        if lane == 0 and c0 >= 4:
                            chk(o - 2, 'hl'); chk(o - 1, 'um1')
                        if lane == 31 and c0 + 4 < P:
                            chk(o + 5, 'hr')
                        # reads of valid cells: x window, y, z
                        for v in range(4):
                            if not val[v]:
                                continue
                            x, y, z = xb + v, yrow, k
                            for dx in (-2, -1, 1, 2):
                                reads.append((o + v + dx, ((x + dx) % nx, y, z)))
                            if act_y:
                                for dy in (-2, -1, 1, 2):
                                    reads.append((o + v + dy * P, (x, (y + dy) % ny, z)))
                            if act_z:
                                for dz in (-2, -1, 1, 2):
                                    reads.append((o + v + dz * PP, (x, y, (z + dz) % nz)))
                        # stores
                        def put(oo):
                            for v in range(4):
                                if val[v]:
                                    chk(oo + v, 'st')
                                    written[oo + v] = (xb + v, yrow, k)
                        put(o)
                        if act_y and yrow < 2:
                            put(o + ny * P)
                        if act_y and yrow >= ny - 2:
                            put(o - ny * P)
                        if act_z and k < 2:
                            put(o + nz * PP)
                        if act_z and k >= nz - 2:
                            put(o - nz * PP)
                        if xb < 2 or xb + 3 >= nx - 2:
                            for v in range(4):
                                if val[v] and xb + v < 2:
                                    chk(o + v + nx, 'gx+'); written[o + v + nx] = (xb + v, yrow, k)
                                if val[v] and xb + v >= nx - 2:
                                    chk(o + v - nx, 'gx-'); written[o + v - nx] = (xb + v, yrow, k)
    # every written padded index holds the image the layout assigns it
    for i, c in written.items():
        if pos_of(nx, ny, nz, i) != c:
            errs.append(('wrong image written', i, c, pos_of(nx, ny, nz, i)))
            break
    # every read of a valid cell is an index the stage writes, holding its image
    for i, c in reads:
        if i not in written:
            errs.append(('read never written', i, c))
            break
        if written[i] != c:
            errs.append(('read wrong', i, c, written[i]))
            break
        if pos_of(nx, ny, nz, i) != c:
            errs.append(('layout image', i, c))
            break
    # each cell stored at its interior position exactly once
    n_int = sum(1 for i, c in written.items()
                if i == ((c[2] + gz) * PY + c[1] + gy) * P + c[0] + GX)
    if n_int != nx * ny * nz:
        errs.append(('interior count', n_int, nx * ny * nz))
    return errs




SHAPES = [(8, 1, 1), (8, 8, 8), (9, 2, 2), (33, 17, 9), (21, 14, 1), (31, 1, 1), (127, 5, 3),
          (128, 3, 2), (13, 2, 5), (10, 7, 4), (8, 3, 1), (11, 1, 4)]
random.seed(3)
SHAPES += [(random.randint(8, 130), random.randint(1, 24), random.randint(1, 5)) for _ in range(6)]


@pytest.mark.parametrize("shape", SHAPES)
def test_padded_layout_reads_what_the_stage_writes(shape):
    for W in (1, 2, 8):
        for zc in (1, 3, 16):
            assert run(*shape, W, zc) == [], (shape, W, zc)


def test_ghost_image_geometry():
    # the row pitch leaves two ghost columns after the cells and is a multiple of 4
    for nx in range(8, 140):
        P, PY, PZ, gy, gz = geom(nx, 5, 1)
        assert P % 4 == 0 and P >= nx + 4 and P < nx + 8
        assert (gy, gz, PY, PZ) == (2, 0, 9, 1)
