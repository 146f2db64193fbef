"""Time-modulated flow (stage velocity g * u_f) through fl_step_rk_modulated,
against the oracle's step_modulated, and the deformation benchmark of
Section 4.1 (eq. rhodonea) run on the GPU.

Per step the GPU starts from the oracle's theta^n; the bar is 1e-12 (FP64)
and 1e-5 (FP32) relative in max norm.  Factor sequences cover g = 1 (the
pre-scaled FP64 path without modulation), fractional and negative factors
(reversed upwind sides), and exact zeros."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.test_gpu_unstructured import Dev

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
GSEQ = [1.0, 0.6, -0.8, 0.0, -1.0, 1.0, 0.25, -0.3, 0.9]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _case(shape, seed):
    h = (0.7 / shape[0], 0.9 / shape[1], 1.1 / shape[2])
    mesh = W.structured_mesh(*shape, *h)
    rng = np.random.default_rng(seed)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, seed + 1)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    return mesh, th, u, dt


def _cast(x, dtype):
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


# (37, 21, 13): plain tiles with ragged edges; (128, 8, 5): the FP32 TMA
# kernel for g >= 0; (33, 1, 1): a 1D line (not the resident kernel here)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("shape", [(37, 21, 13), (128, 8, 5), (33, 1, 1)])
def test_modulated_step_parity(fl, shape, lim, rk, dtype):
    mesh, th, u, dt = _case(shape, seed=11)
    th, u = _cast(th, dtype), _cast(u, dtype)
    S = 1 if rk == 1 else 3
    m = fl.Mesh.structured(*shape, *mesh.h)
    ud = torch.tensor(u, dtype=dtype, device="cuda")
    cur = th
    nsteps = 3
    for n in range(nsteps):
        g = np.array([GSEQ[(n * S + s) % len(GSEQ)] for s in range(S)])
        ref = oracle.step_modulated(mesh, lim, rk, dt, 1, u, g, cur)
        gt = torch.tensor(cur, dtype=dtype, device="cuda")
        fl.step_rk_modulated(m, lim, gt, ud, dt, 1, g, rk_order=rk)
        got = gt.cpu().double().numpy()
        assert _rel(got, ref) <= TOL[dtype], (n, g)
        cur = ref if dtype == torch.float64 else got
    # several steps in one call follow the factor sequence in order
    G = np.array([GSEQ[i % len(GSEQ)] for i in range(nsteps * S)])
    ref = oracle.step_modulated(mesh, lim, rk, dt, nsteps, u, G, th)
    gt = torch.tensor(th, dtype=dtype, device="cuda")
    fl.step_rk_modulated(m, lim, gt, ud, dt, nsteps, G, rk_order=rk)
    assert _rel(gt.cpu().double().numpy(), ref) <= 100 * TOL[dtype]
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", ["vanleer", "superbee", "smart"])
def test_modulated_face_based_mesh(fl, lim, dtype):
    base = W.structured_mesh(12, 9, 7, 0.1, 0.12, 0.15)
    pm, cp, fp, flip = W.permuted_mesh(base, seed=5)
    rng = np.random.default_rng(6)
    th = _cast(rng.uniform(-1, 1, pm.n_cells), dtype)
    u = _cast(0.3 * W.mixed_sign_velocity(pm.n_faces, 7), dtype)
    dt = 0.02
    d = Dev(fl, pm)
    ud = d.faces_in(u, dtype)
    for rk in (1, 3):
        S = 1 if rk == 1 else 3
        G = np.array(GSEQ[:2 * S])
        ref = oracle.step_modulated(pm, lim, rk, dt, 2, u, G, th)
        gt = d.cells_in(th, dtype)
        fl.step_rk_modulated(d.m, lim, gt, ud, dt, 2, G, rk_order=rk)
        assert _rel(d.cells_out(gt), ref) <= 10 * TOL[dtype]
    d.m.close()


def test_modulated_unit_factor_equals_plain_step(fl):
    # with every factor 1 the modulated call is fl_step_rk bit for bit
    mesh, th, u, dt = _case((40, 24, 9), seed=3)
    m = fl.Mesh.structured(40, 24, 9, *mesh.h)
    ud = torch.tensor(u, device="cuda")
    for rk in (1, 3):
        a = torch.tensor(th, device="cuda")
        b = a.clone()
        fl.step_rk(m, "superbee", a, ud, dt, 4, rk_order=rk)
        fl.step_rk_modulated(m, "superbee", b, ud, dt, 4, np.ones(4 * (1 if rk == 1 else 3)),
                             rk_order=rk)
        assert torch.equal(a, b)
    m.close()


def test_modulated_rejects_bad_factors(fl):
    mesh, th, u, dt = _case((16, 8, 4), seed=1)
    m = fl.Mesh.structured(16, 8, 4, *mesh.h)
    ud = torch.tensor(u, device="cuda")
    t = torch.tensor(th, device="cuda")
    with pytest.raises(fl.FLError):
        fl.step_rk_modulated(m, "superbee", t, ud, dt, 2, [1.0, float("nan")], rk_order=1)
    with pytest.raises(ValueError):
        fl.step_rk_modulated(m, "superbee", t, ud, dt, 2, [1.0, 1.0], rk_order=3)
    assert torch.equal(t, torch.tensor(th, device="cuda"))
    m.close()


def test_deformation_benchmark_72(fl):
    """Section 4.1 at 72^3: superbee, forward Euler, t in [0, 3].  Sampled
    steps match the oracle from the oracle's state; the full GPU run
    conserves mass to rounding, stays in [0, 1] and returns the sphere with
    the oracle's L1 error (the two trajectories differ only by rounding,
    which the limiter can amplify locally, so the L1 errors agree to 1 %)."""
    n = 72
    wl = W.config_deformation(n)
    g = wl.extra["g"]
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    ud = torch.tensor(wl.u, device="cuda")
    om = oracle.OracleMesh(wl.mesh)
    # the oracle's trajectory, with three sampled per-step checks on the way
    samples = {0, wl.nsteps // 2, wl.nsteps - 1}
    cur = wl.theta0
    done = 0
    for k in sorted(samples):
        cur = oracle.step_modulated(om, "superbee", 1, wl.dt, k - done, wl.u, g[done:k], cur)
        done = k
        ref = oracle.step_modulated(om, "superbee", 1, wl.dt, 1, wl.u, g[k:k + 1], cur)
        gt = torch.tensor(cur, device="cuda")
        fl.step_rk_modulated(m, "superbee", gt, ud, wl.dt, 1, g[k:k + 1], rk_order=1)
        assert _rel(gt.cpu().numpy(), ref) <= 1e-12, k
    ref_T = oracle.step_modulated(om, "superbee", 1, wl.dt, wl.nsteps - done, wl.u, g[done:], cur)
    gt = torch.tensor(wl.theta0, device="cuda")
    fl.step_rk_modulated(m, "superbee", gt, ud, wl.dt, wl.nsteps, g, rk_order=1)
    got = gt.cpu().numpy()
    m0 = wl.theta0.sum()
    assert abs(got.sum() - m0) <= 1e-12 * m0
    assert got.min() >= -1e-12 and got.max() <= 1.0 + 1e-12
    l1_gpu = np.sum(np.abs(got - wl.theta0)) / n ** 3
    l1_ref = np.sum(np.abs(ref_T - wl.theta0)) / n ** 3
    print("deformation 72^3: L1(theta(T) - theta(0)) GPU %.6e oracle %.6e; max |GPU - oracle| %.2e"
          % (l1_gpu, l1_ref, np.max(np.abs(got - ref_T))))
    assert abs(l1_gpu - l1_ref) <= 0.01 * l1_ref
    m.close()
