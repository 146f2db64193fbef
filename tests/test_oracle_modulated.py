"""Pins of the oracle's time-modulated step (stage velocity g * u_f, the form
of the reversing deformation flow of Section 4.1, eq. rhodonea) and of the
deformation benchmark itself: what scaling a velocity field must and must not
change, exact round trips of the upwind scheme, and the benchmark's exact
mass conservation and reversal under refinement."""
import numpy as np
import pytest

import oracle
import workloads as W

LIMS = ["upwind", "central", "minmod", "vanleer", "superbee", "smart"]


def _case(seed=0, shape=(9, 7, 5)):
    h = (0.7 / shape[0], 0.9 / shape[1], 1.1 / shape[2])
    mesh = W.structured_mesh(*shape, *h)
    rng = np.random.default_rng(seed)
    th = rng.uniform(-1, 1, mesh.n_cells) + (rng.random(mesh.n_cells) < 0.3)
    u = 0.3 * W.mixed_sign_velocity(mesh.n_faces, seed + 1)
    dt = 0.3 * min(h) / np.max(np.abs(u)) / 3
    return mesh, th, u, dt


@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", LIMS)
def test_unit_factor_is_the_plain_step(lim, rk):
    mesh, th, u, dt = _case()
    S = 1 if rk == 1 else 3
    a = oracle.step(mesh, lim, rk, dt, 3, u, th)
    b = oracle.step_modulated(mesh, lim, rk, dt, 3, u, np.ones(3 * S), th)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("rk", [1, 3])
@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("g", [-1.0, 2.0, -0.5])
def test_factor_equals_scaled_velocity(lim, rk, g):
    # g u is exact for these g, so the modulated step must equal the plain
    # step with the scaled field bit for bit -- the selection follows the
    # sign of g u (g < 0 reverses every upwind side) and the flux its size
    mesh, th, u, dt = _case(seed=2)
    S = 1 if rk == 1 else 3
    a = oracle.step(mesh, lim, rk, dt, 2, g * u, th)
    b = oracle.step_modulated(mesh, lim, rk, dt, 2, u, np.full(2 * S, g), th)
    assert np.array_equal(a, b)


def test_zero_factor_is_identity():
    # no flow: Euler leaves theta exactly; SSP-RK3 up to its stage blends
    mesh, th, u, dt = _case(seed=3)
    out = oracle.step_modulated(mesh, "superbee", 1, dt, 4, u, np.zeros(4), th)
    assert np.array_equal(out, th)
    out = oracle.step_modulated(mesh, "superbee", 3, dt, 4, u, np.zeros(12), th)
    assert np.max(np.abs(out - th)) <= 16 * np.spacing(np.max(np.abs(th)))


def test_per_stage_factors_follow_the_stage_order():
    # SSP-RK3 with factors (1, 0, 0): stage 2 and 3 see no flow, so the step
    # is theta + 1/4 ... = 3/4 th + 1/4 th1 then 1/3 th + 2/3 th2 (no flux):
    # th2 = 3/4 th + 1/4 th1, y = 1/3 th + 2/3 th2
    mesh, th, u, dt = _case(seed=4)
    th1 = oracle.step(mesh, "minmod", 1, dt, 1, u, th)
    th2 = 0.75 * th + 0.25 * th1
    want = th / 3.0 + 2.0 / 3.0 * th2
    got = oracle.step_modulated(mesh, "minmod", 3, dt, 1, u, [1.0, 0.0, 0.0], th)
    assert np.max(np.abs(got - want)) <= 4e-16 * np.max(np.abs(th)) * 4


def test_upwind_round_trip_at_cfl_one():
    # Psi = 0, u = 1, CFL 1: N steps forward then N with g = -1 shift the
    # profile by N cells and back (each step exact up to one rounding)
    n = 256
    h = 1.0 / n
    mesh = W.structured_mesh(n, 1, 1, h, 1.0, 1.0)
    x = (np.arange(n) + 0.5) * h
    th0 = np.sin(2 * np.pi * x) + (x > 0.3) * (x < 0.6)
    g = np.concatenate([np.ones(40), -np.ones(40)])
    out = oracle.step_modulated(mesh, "upwind", 1, h, 80, np.ones(n), g, th0)
    assert np.max(np.abs(out - th0)) <= 1e-13
    half = oracle.step_modulated(mesh, "upwind", 1, h, 40, np.ones(n), g[:40], th0)
    assert np.max(np.abs(half - np.roll(th0, 40))) <= 1e-13


def test_deformation_conserves_bounds_and_reverses():
    # Section 4.1: mass is conserved exactly; superbee with forward Euler at a
    # per-cell outflow Courant number of 1/2 keeps the indicator in [0, 1];
    # the flow returns the sphere at t = T, the error shrinking with h
    l1 = []
    for n in (16, 32):
        wl = W.config_deformation(n)
        assert wl.nsteps * wl.dt == pytest.approx(3.0, rel=1e-14)
        th = oracle.step_modulated(wl.mesh, "superbee", 1, wl.dt, wl.nsteps, wl.u,
                                   wl.extra["g"], wl.theta0)
        m0 = wl.theta0.sum()
        assert abs(th.sum() - m0) <= 1e-13 * m0
        assert th.min() >= -1e-12 and th.max() <= 1.0 + 1e-12
        l1.append(np.sum(np.abs(th - wl.theta0)) / n ** 3)
    assert l1[1] < l1[0]


def test_deformation_velocity_is_closed_and_solenoidal():
    n = 24
    wl = W.config_deformation(n)
    C = n ** 3
    u = wl.u
    div = np.zeros((n, n, n))
    for b, ax in enumerate((2, 1, 0)):
        uf = u[b * C:(b + 1) * C].reshape(n, n, n)
        div += uf - np.roll(uf, 1, axis=ax)
    assert np.max(np.abs(div)) <= 1e-14 * np.max(np.abs(u)) * n
    # no flux through the periodic seam: the box is closed
    assert np.all(u[:C].reshape(n, n, n)[:, :, -1] == 0.0)
    assert np.all(u[C:2 * C].reshape(n, n, n)[:, -1, :] == 0.0)
    assert np.all(u[2 * C:].reshape(n, n, n)[-1] == 0.0)
    # the cell-centre face samples follow eq. rhodonea at t = 0 to O(h^2)
    h = 1.0 / n
    i = np.arange(n)
    xf = (i + 1.0) * h
    xc = (i + 0.5) * h
    ux = u[:C].reshape(n, n, n)
    exact = 2 * np.sin(np.pi * xf)[None, None, :] ** 2 * np.sin(2 * np.pi * xc)[None, :, None] \
        * np.sin(2 * np.pi * xc)[:, None, None]
    assert np.max(np.abs(ux - exact)) <= 20 * h * h
