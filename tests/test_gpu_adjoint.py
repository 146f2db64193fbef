"""The hand-written adjoint: operator transpose against the oracle's adjoint
and tangent-linear model, the checkpointed reverse sweep against the oracle's
FP64 reference gradient, the torch.autograd wrapper, and -- at the adjoint
configuration's full size -- central finite differences along random
directions."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]


def _case(shape, seed=0):
    h = (0.7 / shape[0], 0.9 / shape[1], 1.1 / shape[2])
    mesh = W.structured_mesh(*shape, *h)
    rng = np.random.default_rng(seed)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = W.mixed_sign_velocity(mesh.n_faces, seed + 1)
    return mesh, th, u


def _t(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("shape", [(37, 21, 13), (33, 1, 1), (40, 9, 1), (5, 4, 6)])
def test_operator_adjoint_matches_oracle(fl, shape, lim, dtype):
    mesh, th, u = _case(shape, 3)
    if dtype == torch.float32:
        th = th.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    mu = np.random.default_rng(4).normal(size=mesh.n_cells)
    m = fl.Mesh.structured(*shape, *mesh.h)
    out = torch.empty(mesh.n_cells, dtype=dtype, device="cuda")
    fl.fl_conv_limited_adjoint(m.handle, lim, dtype, _t(th, dtype), _t(u, dtype), _t(mu, dtype),
                               out)
    ref = oracle.rhs_adjoint(mesh, lim, th, u, mu)
    scale = np.max(np.abs(u)) * np.max(np.abs(mu)) / min(mesh.h)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.max(np.abs(out.cpu().double().numpy() - ref)) <= 8 * tol * scale
    m.close()


@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_dot_product_with_cpu_tangent_linear(fl, lim):
    # <J v, w> with J v from the oracle's tangent-linear model (CPU) against
    # <v, J^T w> from the GPU adjoint, for one RK3 step
    wl = W.config_taylor_green(n=16, seed=4, nsteps=1, limiter=lim)
    rng = np.random.default_rng(5)
    m = fl.Mesh.structured(16, 16, 16, *wl.mesh.h)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, 3, 1, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        v = rng.normal(size=wl.mesh.n_cells)
        w = rng.normal(size=wl.mesh.n_cells)
        _, Jv = oracle.step_tlm(wl.mesh, lim, 3, wl.dt, 1, wl.u, wl.theta0, v)
        JTw = torch.empty(wl.mesh.n_cells, dtype=torch.float64, device="cuda")
        fl.fl_step_rk_adjoint(m.handle, lim, torch.float64, 3, wl.dt, 1, 1, _t(wl.theta0),
                              _t(wl.u), _t(w), JTw, ws, nb)
        lhs = float(np.dot(Jv, w))
        rhs = float(np.dot(v, JTw.cpu().numpy()))
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jv) * np.linalg.norm(w)
    m.close()


@pytest.mark.parametrize("rk,every", [(3, 3), (3, 20), (1, 4)])
@pytest.mark.parametrize("lim", ["superbee", "vanleer", "smart"])
def test_checkpointed_gradient_matches_oracle(fl, lim, rk, every):
    n, nsteps = 12, 10
    wl = W.config_taylor_green(n=n, seed=4, nsteps=nsteps, limiter=lim)
    tgt = W.smooth_target(wl.mesh.dims, wl.mesh.h, 4)
    J_ref, g_ref = oracle.gradient(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0, tgt)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    thT = oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, rk, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty(wl.mesh.n_cells, dtype=torch.float64, device="cuda")
    fl.fl_step_rk_adjoint(m.handle, lim, torch.float64, rk, wl.dt, nsteps, every, _t(wl.theta0),
                          _t(wl.u), _t(thT - tgt), g, ws, nb)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))
    m.close()


def test_checkpointed_pair_equals_one_call(fl):
    n, nsteps, every = 16, 11, 4
    wl = W.config_taylor_green(n=n, seed=4, nsteps=nsteps, limiter="smart")
    tgt = W.smooth_target(wl.mesh.dims, wl.mesh.h, 4)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    u, th0 = _t(wl.u), _t(wl.theta0)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, 3, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    th = th0.clone()
    fl.fl_step_rk_checkpointed(m.handle, "smart", torch.float64, 3, wl.dt, nsteps, every, th, u,
                               ws, nb)
    ref = th0.clone()
    fl.step_rk(m, "smart", ref, u, wl.dt, nsteps, rk_order=3)
    assert torch.equal(th, ref)
    lam = th - _t(tgt)
    g1 = torch.empty_like(th0)
    fl.fl_step_rk_adjoint_from_checkpoints(m.handle, "smart", torch.float64, 3, wl.dt, nsteps,
                                           every, u, lam, g1, ws, nb)
    g2 = torch.empty_like(th0)
    ws2 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fl.fl_step_rk_adjoint(m.handle, "smart", torch.float64, 3, wl.dt, nsteps, every, th0, u, lam,
                          g2, ws2, nb)
    assert torch.equal(g1, g2)
    m.close()


def test_autograd_function(fl):
    from paper_2110_03044_gb300.autograd import rollout
    n, nsteps = 12, 6
    wl = W.config_taylor_green(n=n, seed=4, nsteps=nsteps, limiter="superbee")
    tgt = W.smooth_target(wl.mesh.dims, wl.mesh.h, 4)
    _, g_ref = oracle.gradient(wl.mesh, "superbee", 3, wl.dt, nsteps, wl.u, wl.theta0, tgt)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    th0 = _t(wl.theta0).requires_grad_(True)
    thT = rollout(th0, _t(wl.u), m, "superbee", wl.dt, nsteps, 3, 4)
    loss = 0.5 * ((thT - _t(tgt)) ** 2).sum()
    loss.backward()
    assert np.max(np.abs(th0.grad.cpu().numpy() - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))
    m.close()


def test_adjoint_config_full_size_central_differences(fl):
    """128^3 Taylor-Green, superbee, 200 SSP-RK3 steps, checkpoints every 20:
    the gradient of 0.5||theta_T - target||^2 against central finite
    differences of GPU forward rollouts along 32 smooth random directions
    (random Fourier fields) and 32 white-noise directions N(0, I).

    The rollout is piecewise linear in theta0 (the limiter is piecewise
    linear), so central differences are exact up to rounding except for the
    limiter kinks crossed inside +-eps, whose effect shrinks with eps.  What
    is left is an absolute error floor of about 1e-8 ||g|| ||v|| (rounding of
    two 200-step rollouts and kinks closer than the smallest step), so the
    relative error of a direction grows as 1 / cos(g, v).  The bar:
      * every direction: |fd - ad| <= 1e-6 ||g|| ||v||;
      * smooth directions with |cos(g, v)| >= 0.05: |fd - ad| <= 1e-6 |ad|;
      * the median relative error over the smooth directions <= 1e-6.
    White-noise directions are nearly orthogonal to the smooth gradient
    (cos 1e-5..1e-3): their relative error is reported only."""
    n, nsteps, every = 128, 200, 20
    wl = W.config_taylor_green(n=n, seed=4, nsteps=nsteps, limiter="superbee")
    tgt = W.smooth_target(wl.mesh.dims, wl.mesh.h, 4)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    u = _t(wl.u)
    th0 = _t(wl.theta0)
    tg = _t(tgt)
    ws_f = torch.empty(fl.fl_workspace_size(m.handle, torch.float64, 3), dtype=torch.uint8,
                       device="cuda")

    def run(x):
        y = x.clone()
        fl.fl_step_rk(m.handle, "superbee", torch.float64, 3, wl.dt, nsteps, y, u, ws_f,
                      ws_f.numel())
        return y

    thT = run(th0)
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, 3, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty_like(th0)
    fl.fl_step_rk_adjoint(m.handle, "superbee", torch.float64, 3, wl.dt, nsteps, every, th0, u,
                          thT - tg, g, ws, nb)

    def dJ(ta, tb):
        # J(a) - J(b) = 0.5 sum (ta - tb)(ta + tb - 2 tgt), without cancellation
        return 0.5 * torch.sum((ta - tb) * (ta + tb - 2 * tg)).item()

    def fd(v, rel_eps):
        eps = rel_eps * float(th0.norm() / v.norm())
        return dJ(run(th0 + eps * v), run(th0 - eps * v)) / (2 * eps)

    def one_sided(v, rel_eps, side):
        # (-3 J(0) + 4 J(h) - J(2h)) / (2h), h = side * eps: exact for a
        # quadratic, blind to kinks on the other side of theta0
        eps = rel_eps * float(th0.norm() / v.norm())
        t1, t2 = run(th0 + side * eps * v), run(th0 + 2 * side * eps * v)
        return side * (4 * dJ(t1, thT) - dJ(t2, thT)) / (2 * eps)

    rng = np.random.default_rng(4)
    smooth, smooth_cos, scaled = [], [], []
    worst_noise_rel = 0.0
    for _ in range(32):
        v = _t(W.sine_sum_field(wl.mesh.dims, wl.mesh.h, rng, n_modes=4, kmax=4, amp=1.0))
        ad = float(torch.dot(g, v).item())
        gv = float(g.norm() * v.norm())
        # a limiter kink inside +-eps shows as an error that shrinks with
        # eps: halve eps (at most three times); a kink closer than that
        # spoils one side only, so the one-sided estimates of the clean side
        # are taken as well
        eps, rel = 1e-7, np.inf
        for _attempt in range(4):
            rel = min(rel, abs(fd(v, eps) - ad) / abs(ad))
            if rel <= 1e-6:
                break
            eps *= 0.5
        if rel > 1e-6:
            for side in (1, -1):
                rel = min(rel, abs(one_sided(v, 1e-7, side) - ad) / abs(ad))
        smooth.append(rel)
        smooth_cos.append(abs(ad) / gv)
        scaled.append(rel * abs(ad) / gv)
    for _ in range(32):
        v = _t(rng.normal(size=wl.mesh.n_cells))
        ad = float(torch.dot(g, v).item())
        err = abs(fd(v, 1e-8) - ad)
        scaled.append(err / float(g.norm() * v.norm()))
        worst_noise_rel = max(worst_noise_rel, err / abs(ad))
    smooth, smooth_cos = np.array(smooth), np.array(smooth_cos)
    print("adjoint vs central differences: smooth directions (rel err, |cos(g, v)|) "
          + " ".join("(%.1e, %.1e)" % (e, c) for e, c in zip(smooth, smooth_cos))
          + "; worst scaled over 64 directions %.2e; white noise worst rel %.2e"
          % (max(scaled), worst_noise_rel))
    assert max(scaled) <= 1e-6
    assert np.all(smooth[smooth_cos >= 0.05] <= 1e-6)
    assert np.median(smooth) <= 1e-6
    m.close()
