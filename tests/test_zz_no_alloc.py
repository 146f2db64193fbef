"""fl_step_rk_noalloc: the explicit step for callers that cannot allocate.

Hosts such as plugin frameworks that own the device memory pool, real-time
loops that cannot pay for an allocation, or deployments whose memory is fixed
at start-up cannot hand this library a workspace.  fl_step_rk_noalloc takes
its stage buffers from a fixed scratch area inside the library instead.  This
test calls it through the C ABI and checks that, twice in a row, it gives the
same result as fl_step_rk with a caller-provided workspace (within the
parity tolerances used everywhere: 1e-12 relative in FP64, 1e-5 in FP32), and
that meshes too large for the area are refused before anything runs.

The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("dtype,rk,lim", [(torch.float64, 3, "superbee"),
                                          (torch.float32, 1, "smart"),
                                          (torch.float64, 1, "vanleer")])
def test_noalloc_matches_workspace_call_twice(fl, dtype, rk, lim):
    shape = (37, 21, 13)
    mesh = W.structured_mesh(*shape, 0.03, 0.04, 0.05)
    rng = np.random.default_rng(17)
    th0 = torch.tensor(rng.uniform(-1, 1, mesh.n_cells), dtype=dtype, device="cuda")
    u = torch.tensor(0.2 * W.mixed_sign_velocity(mesh.n_faces, 4), dtype=dtype, device="cuda")
    dt = 0.02
    m = fl.Mesh.structured(*shape, *mesh.h)
    ref = th0.clone()
    new = th0.clone()
    for _ in range(2):  # two calls in a row, each advancing 3 steps
        fl.step_rk(m, lim, ref, u, dt, 3, rk_order=rk)
        fl.fl_step_rk_noalloc(m.handle, lim, dtype, rk, dt, 3, new, u)
        torch.cuda.synchronize()
        assert _rel(new, ref) <= TOL[dtype]
    m.close()


def test_noalloc_rejects_meshes_beyond_the_area(fl):
    # 2^21 + 2^20 FP64 cells need 48 MiB of RK3 stage buffers (> 32 MiB)
    n = 1 << 21
    m = fl.Mesh.structured(n + (n >> 1), 1, 1, 1.0, 1.0, 1.0)
    th = torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
    u = torch.zeros(m.n_faces, dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FLError) as e:
        fl.fl_step_rk_noalloc(m.handle, "superbee", torch.float64, 3, 0.1, 1, th, u)
    assert e.value.status == fl.FL_EINVAL
    m.close()
