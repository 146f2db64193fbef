"""Pins for the oracle's limiter functions: values fixed by the closed forms
at tabulated r, Sweby's second-order TVD region (Section 3, Harten/Sweby
conditions) and the consistency of the piecewise (branch) form used by the
derivatives."""
import numpy as np
import pytest

import oracle

R_TAB = [-1.0, 0.0, 0.25, 0.5, 1.0, 1.5, 2.0, 3.0, 10.0]
# Values of each limiter at R_TAB, from the mathematical closed forms.
TABLE = {
    "minmod": [0, 0, 0.25, 0.5, 1, 1, 1, 1, 1],
    "vanleer": [0, 0, 0.4, 2.0 / 3.0, 1, 1.2, 4.0 / 3.0, 1.5, 20.0 / 11.0],
    "superbee": [0, 0, 0.5, 1, 1, 1.5, 2, 2, 2],
    "smart": [0, 0, 0.4375, 0.625, 1, 1.375, 1.75, 2.5, 4],
    "upwind": [0] * 9,
    "central": [1] * 9,
}


@pytest.mark.parametrize("lim", sorted(TABLE))
def test_tabulated_values_exact(lim):
    got = oracle.psi(lim, R_TAB)
    assert np.array_equal(got, np.array(TABLE[lim], dtype=np.float64)), (lim, got)


@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee", "smart"])
def test_second_order_point(lim):
    # every second-order limiter passes through Psi(1) = 1 (Sweby)
    assert oracle.psi(lim, [1.0])[0] == 1.0


@pytest.mark.parametrize("lim", ["minmod", "vanleer", "superbee"])
def test_sweby_tvd_region(lim):
    r = np.concatenate([np.linspace(-5, 10, 20001), np.logspace(-8, 8, 2001)])
    p = oracle.psi(lim, r)
    assert np.all(p >= 0.0)
    bound = np.minimum(2.0 * np.maximum(r, 0.0), 2.0)
    assert np.all(p <= bound * (1 + 1e-15))
    # second-order region: between minmod and superbee for r > 0
    lo = np.maximum(0.0, np.minimum(1.0, r))
    hi = np.maximum(0.0, np.maximum(np.minimum(1.0, 2.0 * r), np.minimum(r, 2.0)))
    pos = r > 0
    assert np.all(p[pos] >= lo[pos] * (1 - 1e-15))
    assert np.all(p[pos] <= hi[pos] * (1 + 1e-15))


def test_smart_leaves_sweby_region():
    # SMART's cap 4 lies above Sweby's bound 2: the reason boundedness is not
    # gated for it.
    assert oracle.psi("smart", [10.0])[0] == 4.0


@pytest.mark.parametrize("lim", ["upwind", "central", "minmod", "vanleer", "superbee", "smart"])
def test_branch_form_matches_closed_form(lim):
    r = np.concatenate([np.linspace(-3, 12, 30001), [0.2, 0.5, 1.0, 2.0, 5.0]])
    p_closed = oracle.psi(lim, r)
    p_branch, d = oracle.psi_branch(lim, r)
    np.testing.assert_allclose(p_branch, p_closed, rtol=1e-15, atol=0)
    # derivative of the branch = central difference away from the kinks
    h = 1e-6
    kinks = np.array([0.0, 0.2, 0.5, 1.0, 2.0, 5.0])
    far = np.min(np.abs(r[:, None] - kinks[None, :]), axis=1) > 10 * h
    fd = (oracle.psi(lim, r + h) - oracle.psi(lim, r - h)) / (2 * h)
    np.testing.assert_allclose(d[far], fd[far], atol=2e-7)


def test_infinite_ratio_limits():
    inf = np.array([np.inf, -np.inf])
    assert list(oracle.psi("minmod", inf)) == [1.0, 0.0]
    assert list(oracle.psi("vanleer", inf)) == [2.0, 0.0]
    assert list(oracle.psi("superbee", inf)) == [2.0, 0.0]
    assert list(oracle.psi("smart", inf)) == [4.0, 0.0]


@pytest.mark.parametrize("lim", ["upwind", "central", "minmod", "vanleer", "superbee", "smart"])
def test_branch_form_at_infinite_ratio(lim):
    # r = +-inf lies on the flat end pieces: the branch form gives the closed
    # form's limit with a zero derivative (no 0 * inf in the tangent-linear
    # model's Psi - Psi' r)
    inf = np.array([np.inf, -np.inf])
    p, d = oracle.psi_branch(lim, inf)
    np.testing.assert_array_equal(p, oracle.psi(lim, inf))
    np.testing.assert_array_equal(d, [0.0, 0.0])
