"""Building blocks of the stage kernels, run on the device through a
small probe compiled against the library's own header (fl_face.cuh):

* the van Leer quotient p q / (p + q), computed by Newton-Raphson division
  instead of an IEEE division: in FP64 (from an FP32 seed) against CUDA's
  __ddiv_rn, relative error below 2^-47; in FP32 against __fdiv_rn, below
  2^-22; and identical to the IEEE quotient where the divisor's range sends
  it to the IEEE division;
* SMART's piece test on the integer pipe (r >= 5, r <= 1/5 for r = p / q):
  against the exact decision in rational arithmetic, including ties, inputs
  one ulp either side of the boundaries, and subnormal operands;
* the FP64 limiter terms formed off the FP64 pipe: van Leer's p q / (p + q)
  in paired FP32 against the exact rational quotient (relative error below
  2^-45), and SMART's middle piece (q + 3p) / 8 in 64-bit integers, which
  must be the correctly rounded value."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2110_03044_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    from paper_2110_03044_gb300._build_lib import ARCH, _nvcc
    out = str(tmp_path_factory.mktemp("probe") / "face_arith_probe.so")
    cmd = [_nvcc()] + ARCH + ["-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                              "-I" + CSRC, os.path.join(HERE, "cuda", "face_arith_probe.cu"),
                              "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.probe_quot.argtypes = [P, P, P, P, ctypes.c_int]
    lib.probe_quot32.argtypes = [P, P, P, P, ctypes.c_int]
    lib.probe_smart.argtypes = [P, P, P, ctypes.c_int]
    lib.probe_limiter_term.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int]
    lib.probe_sub_exact.argtypes = [P, P, P, P, ctypes.c_int]
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _quot(probe, n, s):
    n = np.ascontiguousarray(n, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    q = np.empty_like(n)
    ref = np.empty_like(n)
    assert probe.probe_quot(_ptr(n), _ptr(s), _ptr(q), _ptr(ref), len(n)) == 0
    return q, ref


def _exponent_field(x):
    return (np.asarray(x, np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)


def test_van_leer_quotient_against_ieee_division(probe):
    rng = np.random.default_rng(3)
    k = 200000
    p = rng.uniform(0.5, 1.0, k) * 10.0 ** rng.integers(-150, 150, k)
    q = rng.uniform(0.5, 1.0, k) * 10.0 ** rng.integers(-150, 150, k)
    # the limiter's own operands: n = p q, s = p + q
    n, s = p * q, p + q
    got, ref = _quot(probe, n, s)
    E = _exponent_field(s)
    fast = (E >= 2) & (E <= 2044) & np.isfinite(n)
    assert fast.all()
    normal = fast & (np.abs(ref) >= np.finfo(np.float64).tiny)
    rel = np.abs(got[normal] - ref[normal]) / np.abs(ref[normal])
    assert rel.max() <= 2.0 ** -47, rel.max()
    # tiny quotients round at subnormal spacing: within 4 of its units
    sub = fast & ~normal
    assert np.all(np.abs(got[sub] - ref[sub]) <= 4 * 2.0 ** -1074 + 2.0 ** -47 * np.abs(ref[sub]))


def test_van_leer_quotient_range_edges_take_ieee_division(probe):
    tiny = np.finfo(np.float64).tiny
    big = np.finfo(np.float64).max
    s = np.array([tiny / 8, tiny, 1.5 * tiny, 2 * tiny, 3.99 * tiny,  # E = 0, 1, 1, 2, 2
                  2.0 ** 1021, 1.9 * 2.0 ** 1021, 2.0 ** 1022, big, np.inf, 5.0])
    n = np.array([1e-320, 3e-310, 1.0, 2.5e-300, 7.0, 1e300, 2.0, 1.5e307, big, 1.0, np.inf])
    got, ref = _quot(probe, n, s)
    E = _exponent_field(s)
    slow = (E < 2) | (E > 2044) | ~np.isfinite(n)
    assert slow.sum() >= 6
    np.testing.assert_array_equal(got[slow], ref[slow])
    rel = np.abs(got[~slow] - ref[~slow]) / np.abs(ref[~slow])
    assert rel.max() <= 2.0 ** -47


def test_van_leer_quotient_fp32_against_ieee_division(probe):
    rng = np.random.default_rng(4)
    k = 200000
    p = (rng.uniform(0.5, 1.0, k) * 10.0 ** rng.integers(-18, 18, k)).astype(np.float32)
    q = (rng.uniform(0.5, 1.0, k) * 10.0 ** rng.integers(-18, 18, k)).astype(np.float32)
    # the range edges: sums below 2^-125 or above 2^62 take the IEEE division
    edge_p = np.array([2.0 ** -127, 2.0 ** -126, 1e-38, 2.0 ** 61, 2.0 ** 62, 1e20, 3e38],
                      np.float32)
    edge_q = np.array([2.0 ** -128, 2.0 ** -127, 1e-38, 2.0 ** 61, 1.0, 1e19, 1e30], np.float32)
    p = np.concatenate([p, edge_p])
    q = np.concatenate([q, edge_q])
    with np.errstate(over="ignore", under="ignore"):
        n, s = p * q, p + q
    got = np.empty_like(n)
    ref = np.empty_like(n)
    assert probe.probe_quot32(_ptr(n), _ptr(s), _ptr(got), _ptr(ref), len(n)) == 0
    slow = ~((s >= np.float32(2.0 ** -125)) & (s <= np.float32(2.0 ** 62)))
    assert slow.sum() >= 5
    np.testing.assert_array_equal(got[slow], ref[slow])
    normal = ~slow & (np.abs(ref) >= np.finfo(np.float32).tiny)
    rel = np.abs(got[normal].astype(np.float64) - ref[normal]) / np.abs(ref[normal])
    assert rel.max() <= 2.0 ** -22, rel.max()
    sub = ~slow & ~normal
    assert np.all(np.abs(got[sub] - ref[sub]) <= 4 * 2.0 ** -149)


def _exact_piece(p, q):
    # ties go to the lower piece: r = 5 is the middle piece, r = 1/5 piece 2
    fp, fq = Fraction(float(p)), Fraction(float(q))
    if fp > 5 * fq:
        return 1
    if fq >= 5 * fp:
        return 2
    return 3


def test_smart_piece_is_the_exact_decision(probe):
    rng = np.random.default_rng(5)
    p = [rng.uniform(0.5, 1.0, 4000) * 10.0 ** rng.integers(-300, 300, 4000)]
    q = [p[0] * 10.0 ** rng.uniform(-2, 2, 4000)]
    # one to four ulps either side of q = 5p and p = 5q, and the ties
    base = rng.uniform(1.0, 2.0, 500) * 2.0 ** rng.integers(-1000, 1000, 500)
    for step in range(-4, 5):
        five = base * 5.0
        for _ in range(abs(step)):
            five = np.nextafter(five, np.inf if step > 0 else -np.inf)
        p += [base, five]
        q += [five, base]
    ties = 2.0 ** rng.integers(-1000, 1000, 200).astype(np.float64)
    p += [ties, 5 * ties]
    q += [5 * ties, ties]
    # subnormal operands (and normal ones beside them)
    sub = rng.integers(1, 2 ** 40, 600).astype(np.float64) * 2.0 ** -1074
    p += [sub[:300], sub[300:] * 5, np.full(100, 2.0 ** -1020)]
    q += [sub[300:], sub[:300], sub[:100]]
    p = np.concatenate(p)
    q = np.concatenate(q)
    assert np.all(p > 0) and np.all(q > 0) and np.all(np.isfinite(p)) and np.all(np.isfinite(q))
    piece = np.empty(len(p), np.int32)
    assert probe.probe_smart(_ptr(p), _ptr(q), _ptr(piece), len(p)) == 0
    want = np.array([_exact_piece(a, b) for a, b in zip(p, q)], np.int32)
    bad = np.nonzero(piece != want)[0]
    assert bad.size == 0, [(p[i], q[i], piece[i], want[i]) for i in bad[:5]]
    assert {1, 2, 3} <= set(want.tolist())


def _term(probe, p, q, mode):
    p = np.ascontiguousarray(p, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    g = np.empty(len(p), np.uint64)
    assert probe.probe_limiter_term(_ptr(p), _ptr(q), _ptr(g), len(p), mode) == 0
    return g.view(np.float64)


def test_van_leer_paired_fp32_quotient_against_exact(probe):
    rng = np.random.default_rng(7)
    k = 30000
    p = rng.uniform(1.0, 2.0, k) * 2.0 ** rng.integers(-1000, 1000, k)
    # the other operand within 2^-70 .. 2^70 of p (all exponent gaps, including
    # the d >= 60 shortcut), equal to p, or one ulp from it
    q = p * 2.0 ** rng.uniform(-70, 70, k)
    q[:500] = p[:500]
    q[500:1000] = np.nextafter(p[500:1000], np.inf)
    ok = (q > 2.0 ** -1018) & (q < 2.0 ** 1020)
    p, q = p[ok], q[ok]
    g = _term(probe, p, q, 0)
    worst = 0.0
    for a, b, x in zip(p, q, g):
        fa, fb = Fraction(float(a)), Fraction(float(b))
        exact = fa * fb / (fa + fb)
        worst = max(worst, float(abs(Fraction(float(x)) - exact) / exact))
    assert worst <= 2.0 ** -45, worst


def test_smart_middle_piece_is_correctly_rounded(probe):
    rng = np.random.default_rng(8)
    k = 30000
    q = rng.uniform(1.0, 2.0, k) * 2.0 ** rng.integers(-1000, 1000, k)
    p = q * rng.uniform(0.2, 5.0, k)
    # exact ties of the rounding: q + 3p one bit beyond 53 significant bits
    t = 2.0 ** rng.integers(-900, 900, 300).astype(np.float64)
    p = np.concatenate([p, t, t * (1 + 2.0 ** -52)])
    q = np.concatenate([q, t * (1 + 2.0 ** -51), t])
    g = _term(probe, p, q, 1)
    want = np.array([float((Fraction(float(b)) + 3 * Fraction(float(a))) / 8)
                     for a, b in zip(p, q)])
    bad = np.nonzero(g != want)[0]
    assert bad.size == 0, [(p[i], q[i], g[i], want[i]) for i in bad[:5]]


def test_integer_pipe_difference_has_the_bits_of_the_fp64_subtraction(probe):
    # sub_exact forms exact differences (Sterbenz pairs) on the integer pipe
    # and hands every other pair to __dsub_rn: all results carry the bits of
    # __dsub_rn, zeros' signs included
    rng = np.random.default_rng(41)
    n = 200_000
    base = rng.uniform(-4, 4, n) * 2.0 ** rng.integers(-40, 40, n)
    near = base * rng.uniform(0.45, 2.2, n)                 # ratios around Sterbenz's range
    ulps = np.nextafter(base, np.inf) + rng.integers(-3, 4, n) * np.spacing(base)
    pw = 2.0 ** rng.integers(-1000, 1000, n)
    edge = np.array([0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 1.5, 3.0, 2.0 ** -1022, 2.0 ** -1021,
                     2.0 ** -1074, 5e-324 * 7, 1.7976931348623157e308, np.inf, -np.inf, np.nan,
                     2.0 ** 53, 2.0 ** 53 + 2, 1 + 2.0 ** -52, 2 - 2.0 ** -52, 4 - 2.0 ** -51])
    ea, eb = np.meshgrid(edge, edge)
    a = np.concatenate([base, base, base, pw, pw * 1.5, ea.ravel()])
    b = np.concatenate([near, ulps, -near, pw * (1 + 2.0 ** -52), pw * 0.75, eb.ravel()])
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    d = np.empty_like(a)
    ref = np.empty_like(a)
    assert probe.probe_sub_exact(_ptr(a), _ptr(b), _ptr(d), _ptr(ref), len(a)) == 0
    assert np.array_equal(d.view(np.uint64), ref.view(np.uint64))
    # most of the near pairs are Sterbenz pairs: the integer path is exercised
    exact = (np.sign(base) == np.sign(near)) & (np.abs(near) <= 2 * np.abs(base)) & \
            (np.abs(base) <= 2 * np.abs(near))
    assert exact.mean() > 0.5
