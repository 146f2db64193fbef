"""Pins for the oracle's derivatives: the tangent-linear model against
central finite differences of the forward oracle (exact up to rounding for
the piecewise-linear limiters while no branch flips), and the adjoint against
the tangent-linear model through the dot-product identity
<J v, w> = <v, J^T w>."""
import numpy as np
import pytest

import oracle
import workloads as W


def _setup(n=6, seed=4, lim="superbee"):
    wl = W.config_taylor_green(n=n, seed=seed, nsteps=4, limiter=lim)
    return wl


@pytest.mark.parametrize("lim", ["minmod", "superbee", "smart", "vanleer"])
@pytest.mark.parametrize("rk", [1, 3])
def test_tlm_matches_central_differences(lim, rk):
    wl = _setup(lim=lim)
    rng = np.random.default_rng(11)
    v = rng.normal(size=wl.mesh.n_cells)
    nsteps = 3
    th_t, dth = oracle.step_tlm(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0, v)
    eps = 1e-6
    plus = oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0 + eps * v)
    minus = oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0 - eps * v)
    fd = (plus - minus) / (2 * eps)
    np.testing.assert_array_equal(th_t, oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u,
                                                    wl.theta0))
    tol = 1e-6 if lim == "vanleer" else 1e-7
    err = np.linalg.norm(fd - dth) / np.linalg.norm(dth)
    assert err < tol, err


@pytest.mark.parametrize("lim", ["minmod", "superbee", "smart", "vanleer", "upwind", "central"])
def test_operator_adjoint_dot_product(lim):
    wl = _setup(lim=lim)
    mesh = oracle.OracleMesh(wl.mesh)
    rng = np.random.default_rng(2)
    th = wl.theta0
    v = rng.normal(size=mesh.C)
    w = rng.normal(size=mesh.C)
    # J v through the tangent-linear model of one Euler step with dt = 1:
    # (theta + R(theta))' = v + R'(theta) v
    _, d = oracle.step_tlm(mesh, lim, 1, 1.0, 1, wl.u, th, v)
    Jv = d - v
    JTw = oracle.rhs_adjoint(mesh, lim, th, wl.u, w)
    lhs, rhs = np.dot(Jv, w), np.dot(v, JTw)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Jv) * np.linalg.norm(w)


@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", ["superbee", "vanleer"])
def test_gradient_matches_tlm_and_fd(rk, lim):
    wl = _setup(n=6, lim=lim)
    tgt = W.smooth_target(wl.mesh.dims, wl.mesh.h, 4)
    nsteps = 5
    J, g = oracle.gradient(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0, tgt)
    thT = oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0)
    assert abs(J - 0.5 * np.sum((thT - tgt) ** 2)) <= 1e-12 * J
    rng = np.random.default_rng(4)
    for _ in range(4):
        v = rng.normal(size=wl.mesh.n_cells)
        _, dth = oracle.step_tlm(wl.mesh, lim, rk, wl.dt, nsteps, wl.u, wl.theta0, v)
        dJ_tlm = np.dot(thT - tgt, dth)
        dJ_adj = np.dot(g, v)
        assert abs(dJ_adj - dJ_tlm) <= 1e-12 * np.linalg.norm(g) * np.linalg.norm(v)
        eps = 1e-6
        Jp = 0.5 * np.sum((oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u,
                                       wl.theta0 + eps * v) - tgt) ** 2)
        Jm = 0.5 * np.sum((oracle.step(wl.mesh, lim, rk, wl.dt, nsteps, wl.u,
                                       wl.theta0 - eps * v) - tgt) ** 2)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - dJ_adj) <= 1e-6 * abs(dJ_adj) + 1e-9


@pytest.mark.parametrize("rk", [1, 3])
def test_central_tlm_is_the_linear_map_through_flat_faces(rk):
    # Psi = 1 for every r: the central scheme is linear in theta, d_u == 0
    # faces included (their guarded value theta_C equals theta_C + d_u / 2),
    # so its tangent-linear model applied to v is the forward step of v
    # itself -- on a field full of plateaus (many faces with d_u == 0)
    wl = _setup(n=7, lim="central")
    th = W.quantized_field(wl.mesh.n_cells, 5)
    v = np.random.default_rng(6).normal(size=wl.mesh.n_cells)
    _, dth = oracle.step_tlm(wl.mesh, "central", rk, wl.dt, 2, wl.u, th, v)
    lin = oracle.step(wl.mesh, "central", rk, wl.dt, 2, wl.u, v)
    assert np.max(np.abs(dth - lin)) <= 1e-13 * np.max(np.abs(lin))


@pytest.mark.parametrize("lim", ["minmod", "superbee", "smart", "vanleer", "upwind", "central"])
def test_tlm_at_an_overflowing_ratio_is_its_finite_limit(lim):
    # a subnormal d_u beside a normal d_U makes r = d_U / d_u overflow to inf;
    # the face sits on the limiter's flat cap, where theta_f = theta_C +
    # Psi_cap d_u / 2: the derivative is that of the same branch at a tiny
    # normal d_u (r finite), and the adjoint stays the TLM's transpose
    n = 12
    mesh = W.structured_mesh(n, 1, 1, 1.0 / n, 1.0, 1.0)
    u = np.full(n, 0.7)
    th = np.linspace(-1.0, 1.0, n)
    th[3], th[4], th[5] = -1.0, 0.0, 5e-324   # face 4|5: d_u subnormal, d_U = 1
    th_n = th.copy()
    th_n[5] = 1e-300                            # same branch, r = 1e300
    v = np.random.default_rng(9).normal(size=n)
    _, d_inf = oracle.step_tlm(mesh, lim, 1, 0.01, 1, u, th, v)
    _, d_fin = oracle.step_tlm(mesh, lim, 1, 0.01, 1, u, th_n, v)
    assert np.all(np.isfinite(d_inf))
    assert np.max(np.abs(d_inf - d_fin)) <= 1e-14 * np.max(np.abs(d_fin))
    w = np.random.default_rng(10).normal(size=n)
    om = oracle.OracleMesh(mesh)
    _, d1 = oracle.step_tlm(om, lim, 1, 1.0, 1, u, th, v)
    JTw = oracle.rhs_adjoint(om, lim, th, u, w)
    assert np.all(np.isfinite(JTw))
    assert abs(np.dot(d1 - v, w) - np.dot(v, JTw)) <= 1e-13 * np.linalg.norm(d1 - v) * \
        np.linalg.norm(w)


@pytest.mark.parametrize("lim", ["minmod", "superbee", "smart", "vanleer"])
def test_tlm_at_an_underflowing_ratio_keeps_its_branch(lim):
    # r = d_U / d_u > 0 below 2^-1075 rounds to 0, but the face lies on the
    # limiter's first increasing piece (Psi' > 0), as at any small positive
    # r: the derivative's branch is decided from d_U and d_u exactly
    n = 12
    mesh = W.structured_mesh(n, 1, 1, 1.0 / n, 1.0, 1.0)
    u = np.full(n, 0.7)
    th = np.linspace(-1.0, 1.0, n)
    th[3], th[4], th[5] = 0.0, 5e-324, 4.0   # face 4|5: d_U subnormal, d_u = 4
    th_n = th.copy()
    th_n[4] = 1e-300                           # same piece, r = 2.5e-301
    v = np.random.default_rng(12).normal(size=n)
    _, d_tiny = oracle.step_tlm(mesh, lim, 1, 0.01, 1, u, th, v)
    _, d_norm = oracle.step_tlm(mesh, lim, 1, 0.01, 1, u, th_n, v)
    assert np.max(np.abs(d_tiny - d_norm)) <= 1e-14 * np.max(np.abs(d_norm))
