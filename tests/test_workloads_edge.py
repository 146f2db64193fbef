"""The edge-case generators produce the inputs they are meant to: on a line of
quantized values the raw differences give exact ties of the gradient ratio at
the limiters' kinks, zero differences, and subnormal differences next to
normal ones (an overflowing ratio); the velocities hold +0 and -0."""
import math

import numpy as np

import workloads as W


def _ratios(th):
    d = np.diff(np.concatenate([th, th[:1]]))  # d[i] = th[i+1] - th[i] (periodic)
    up = np.roll(d, 1)  # the upstream difference for a positive flow
    return d, up


def test_quantized_field_hits_the_ratio_edge_cases():
    th = W.quantized_field(20000, 3)
    d, up = _ratios(th)
    assert np.any(d == 0) and np.any(up == 0)
    nz = (d != 0) & (up != 0) & np.isfinite(up / np.where(d == 0, 1, d))
    r = {float(x) for x in (up[nz] / d[nz]) if math.isfinite(x)}
    for kink in (0.2, 0.5, 1.0, 2.0, 5.0, -1.0):
        assert kink in r, kink
    tiny = np.finfo(np.float64).smallest_subnormal
    sub = (np.abs(d) > 0) & (np.abs(d) <= 2 * tiny) & (np.abs(up) >= 0.5)
    assert np.any(sub)  # r = d_U / d_u overflows
    assert np.any(np.signbit(th) & (th == 0))  # a negative zero


def test_quantized_field_fp32_subnormals():
    th = W.quantized_field(5000, 4, "f32")
    tiny32 = float(np.finfo(np.float32).smallest_subnormal)
    assert np.any(th == tiny32)
    assert np.array_equal(th.astype(np.float32).astype(np.float64), th)


def test_edge_velocity_signed_zeros():
    u = W.edge_velocity(5000, 5)
    z = u == 0
    assert np.any(z & np.signbit(u)) and np.any(z & ~np.signbit(u))
    assert np.any(u > 0) and np.any(u < 0)
