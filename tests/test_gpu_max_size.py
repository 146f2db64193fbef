"""The largest structured mesh the library takes (nx ny nz < 2^31 cells, here
1024 x 1024 x 2047 = 2.15e9 cells with 6.4e9 face entries, so every face
offset and most cell offsets need 64-bit arithmetic): one SSP-RK3 step
through each kernel family that serves it (the temporally blocked step
included), checked cell by cell against the
oracle on local patches around sampled cells (the last planes, the periodic
wrap, tile edges, random cells), plus mass conservation over the whole mesh.

Inputs are drawn on the device by torch's seeded generator (uniform theta,
uniform mixed-sign face velocities, so every limiter branch occurs); the
oracle reads the patch values back from those tensors."""
import gc

import numpy as np
import pytest
import torch

import oracle
from tests.patch import patch

pytestmark = pytest.mark.gpu

RADIUS = 6  # 2 cells per RK stage, 3 stages: the centre of a 13^3 patch is exact


def _free():
    gc.collect()
    torch.cuda.empty_cache()


def _samples(dims, rng, n_random=10):
    nx, ny, nz = dims
    fixed = [(nx - 1, ny - 1, nz - 1), (0, 0, 0), (nx - 1, 0, nz - 1), (0, ny - 1, nz - 2),
             (31, 7, nz - 1), (32, 8, nz // 2), (nx // 2 + 127, ny // 2 + 8, nz - 3)]
    rand = [tuple(int(v) for v in rng.integers(0, [nx, ny, nz])) for _ in range(n_random)]
    return fixed + rand


# (shape, dtype, kernel that serves it); the temporally blocked step runs
# through fl_step_rk_blocked, the others through fl_step_rk
CASES = [
    ((1024, 1024, 2047), torch.float64, "FP64 shared-memory tile"),
    ((1024, 1024, 2047), torch.float32, "FP32 TMA kernel"),
    ((1030, 1024, 2036), torch.float32, "FP32 register tile"),
    ((1024, 1024, 2047), torch.float64, "FP64 temporally blocked"),
    ((1030, 1024, 2036), torch.float32, "FP32 temporally blocked"),
]


@pytest.mark.parametrize("shape,dtype,kernel", CASES, ids=[c[2] for c in CASES])
def test_largest_mesh_sampled_and_conserved(fl, shape, dtype, kernel):
    nx, ny, nz = shape
    C = nx * ny * nz
    assert C < 2 ** 31 and 3 * C > 2 ** 32
    es = torch.finfo(dtype).bits // 8
    _free()
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    m = fl.Mesh.structured(nx, ny, nz, *h)
    nb = fl.fl_workspace_size(m.handle, dtype, 3)
    need = C * es * 4 + nb + (1 << 30)
    free_b, _ = torch.cuda.mem_get_info()
    if free_b < need:
        m.close()
        pytest.skip("needs %.1f GB of free device memory, %.1f GB free" % (need / 1e9, free_b / 1e9))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2047)
    th = torch.empty(C, dtype=dtype, device="cuda").uniform_(0.0, 1.0, generator=gen)
    u = torch.empty(3 * C, dtype=dtype, device="cuda").uniform_(-1.0, 1.0, generator=gen)
    dt = 0.4 / (1.0 / h[0] + 1.0 / h[1] + 1.0 / h[2])
    # the sampled patches' inputs, read before the step overwrites theta
    rng = np.random.default_rng(11)
    picks = []
    for c in _samples(shape, rng):
        pm, cells, fidx, centre = patch(shape, h, c, RADIUS)
        th_p = th[torch.from_numpy(cells).cuda()].double().cpu().numpy()
        u_p = u[torch.from_numpy(fidx).cuda()].double().cpu().numpy()
        picks.append((c, pm, cells[centre], centre, th_p, u_p))
    red = torch.empty(fl.fl_reduce_workspace_size(), dtype=torch.uint8, device="cuda")
    m0 = fl.fl_reduce_mass(m.handle, dtype, th, red)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    step = fl.fl_step_rk_blocked if "blocked" in kernel else fl.fl_step_rk
    step(m.handle, "superbee", dtype, 3, dt, 1, th, u, ws, nb)
    torch.cuda.synchronize()
    m1 = fl.fl_reduce_mass(m.handle, dtype, th, red)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert abs(m1 - m0) <= tol * abs(m0)
    idx = torch.tensor([p[2] for p in picks], dtype=torch.int64, device="cuda")
    got = th[idx].double().cpu().numpy()
    for (c, pm, _, centre, th_p, u_p), g in zip(picks, got):
        ref = oracle.step(pm, "superbee", 3, dt, 1, u_p, th_p)[centre]
        assert abs(g - ref) <= tol, (kernel, c, g, ref)
    del th, u, ws, red, idx
    m.close()
    _free()
