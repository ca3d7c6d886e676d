"""Double-word arithmetic of the bus kernel (csrc/dword.cuh), built for the
host from the same header: conversions exact to their stated precision, and
the sum, product and fused product-sum within their error bounds, checked
against exact rational arithmetic.  (The GPU test
test_gpu_dword.py compares the device's results with these bit for bit.)"""
import ctypes as C
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2310_13145_b300", "csrc")
U2 = 2.0 ** -48  # u^2 for u = 2^-24


def build_host(tmpdir):
    so = os.path.join(str(tmpdir), "dword_host.so")
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC, "-o", so,
                           os.path.join(HERE, "dword_host.cpp")])
    lib = C.CDLL(so)
    dp = C.POINTER(C.c_double)
    lib.dw_host_ops.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp]
    return lib


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    return build_host(tmp_path_factory.mktemp("dword"))


def run_ops(lib, op, x, y=None, z=None):
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros_like(x) if y is None else np.ascontiguousarray(y, np.float64)
    z = np.zeros_like(x) if z is None else np.ascontiguousarray(z, np.float64)
    out = np.zeros((x.size, 4))
    dp = C.POINTER(C.c_double)
    lib.dw_host_ops(op, x.size, x.ctypes.data_as(dp), y.ctypes.data_as(dp), z.ctypes.data_as(dp),
                    out.ctypes.data_as(dp))
    return out


def sample(n, seed, lo=-6, hi=6):
    """Log-uniform magnitudes in [10^lo, 10^hi] with random signs and full
    53-bit significands."""
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(lo, hi, n) * (1.0 + rng.random(n) * 1e-3)


def dwval(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def test_from_d_split(host):
    x = np.concatenate([sample(20000, 1, -30, 30), [1.0, -1.0, 2.0 ** -126, 3.0, np.pi, 1.0 + 2.0 ** -30,
                                                    1.0 + 2.0 ** -52, np.nextafter(2.0, 0.0), 0.1]])
    o = run_ops(host, 0, x)
    h, back = o[:, 0], o[:, 2]
    l = o[:, 3].astype(np.uint32).view(np.float32).astype(np.float64)  # exact, subnormals included
    # h is x truncated to 24 significant bits: same sign, |h| <= |x| < |h| + ulp(h)
    ulp_h = np.abs(h) * 2.0 ** -23
    assert np.all(np.sign(h) == np.sign(x))
    assert np.all(np.abs(h) <= np.abs(x)) and np.all(np.abs(x) - np.abs(h) < 2.0 * ulp_h)
    # l carries the next 24 bits: |l| < ulp(h), of x's sign (or zero)
    assert np.all(np.abs(l) < 2.0 * ulp_h)
    assert np.all((l == 0) | (np.sign(l) == np.sign(x)))
    # together ~48 bits: |x - (h + l)| < 2^-47 |x| (+ 2^-126 where the low
    # part would be subnormal), and h + l is exact in FP64
    assert np.all(np.abs(x - (h + l)) <= 2.0 ** -47 * np.abs(x) + 2.0 ** -126)
    big = np.abs(x) >= 2.0 ** -102
    assert np.all(np.abs(x - (h + l))[big] <= 2.0 ** -47 * np.abs(x[big]))
    assert np.array_equal(back, h + np.where(np.abs(l) < 2.0 ** -126, 0.0, l))
    # near the bottom of the range the low part becomes a subnormal float,
    # still exact: the window of 24 bits below h's is kept down to 2^-102
    t = np.ldexp(1.0 + np.random.default_rng(4).integers(1, 2 ** 52, 400) * 2.0 ** -52,
                 np.repeat(np.arange(-110, -90), 20))
    ot = run_ops(host, 0, t)
    lo = ot[:, 3].astype(np.uint32).view(np.float32).astype(np.float64)  # l from its bit pattern
    keep = np.abs(t) >= 2.0 ** -102
    ex = np.floor(np.log2(np.abs(t))).astype(int)
    r = t - ot[:, 0]                                               # exact: the bits below h
    w = np.ldexp(np.trunc(np.ldexp(r, 47 - ex)), ex - 47)          # truncated to the 24-bit window
    assert np.array_equal(lo[keep], w[keep])
    assert np.any(np.abs(lo[keep]) < 2.0 ** -126) and np.all(lo[~keep] == 0)
    # dw_f2d (and so dw_to_d) drops a subnormal low part: an error below 2^-126
    assert np.all(ot[:, 1] == np.where(np.abs(lo) < 2.0 ** -126, 0.0, lo))
    # values with at most 48 significant bits round-trip exactly
    y = np.ldexp(np.random.default_rng(3).integers(2 ** 47, 2 ** 48, 1000).astype(np.float64), -40)
    oy = run_ops(host, 0, y)
    assert np.array_equal(oy[:, 0] + oy[:, 1], y)


def test_from_d_special(host):
    x = np.array([0.0, -0.0, 1e-200, -1e-200, 1e200, np.inf, -np.inf, np.nan, 2.0 ** -120])
    o = run_ops(host, 0, x)
    assert o[0, 0] == 0.0 and o[1, 0] == 0.0 and np.signbit(o[1, 0])
    assert o[2, 0] == 0.0 and o[3, 0] == 0.0          # below FP32's range: signed zero
    assert np.all(np.isnan(o[4:8, 0]))                # at or above 2^128: NaN
    assert o[8, 0] == 2.0 ** -120 and o[8, 1] == 0.0


# (op, reference as a function of the exact inputs, error scale, bound in u^2).
# The operands come from dw_from_d, whose low parts reach ulp(h) (twice a
# normalised pair's), and the product drops the low parts' product: the
# bounds are those of the header, ~16 u^2 = 2^-44 at most.
OPS = {
    "add": (1, lambda a, b, c: a + b, lambda a, b, c: abs(a) + abs(b), 4.0),
    "sub": (2, lambda a, b, c: a - b, lambda a, b, c: abs(a) + abs(b), 4.0),
    "mul": (4, lambda a, b, c: a * b, lambda a, b, c: abs(a * b), 16.0),
    "sqr": (6, lambda a, b, c: a * a, lambda a, b, c: a * a, 12.0),
    "fma": (7, lambda a, b, c: a * b + c, lambda a, b, c: abs(a * b) + abs(c), 16.0),
}


@pytest.mark.parametrize("name", sorted(OPS))
def test_ops_error_bounds(host, name):
    op, ref, scale, k = OPS[name]
    n = 3000
    x, y, z = sample(n, 11), sample(n, 12), sample(n, 13)
    # cancellation cases: y close to -x (and z close to -x y)
    y[: n // 4] = -x[: n // 4] * (1.0 + np.random.default_rng(5).normal(0, 1e-9, n // 4))
    z[: n // 4] = -(x[: n // 4] * y[: n // 4]) * (1.0 + np.random.default_rng(6).normal(0, 1e-9, n // 4))
    o = run_ops(host, op, x, y, z)
    ix, iy, iz = run_ops(host, 0, x), run_ops(host, 0, y), run_ops(host, 0, z)
    worst = 0.0
    for i in range(n):
        a, b, c = dwval(ix[i, 0], ix[i, 1]), dwval(iy[i, 0], iy[i, 1]), dwval(iz[i, 0], iz[i, 1])
        exact = ref(a, b, c)
        got = dwval(o[i, 0], o[i, 1])
        err = abs(got - exact)
        bound = Fraction(k * U2) * scale(a, b, c)
        assert err <= bound, (name, i, float(err), float(bound))
        worst = max(worst, float(err / scale(a, b, c)) if scale(a, b, c) else 0.0)
        # the result is normalised: |l| <= ulp(h)
        assert abs(o[i, 1]) <= abs(o[i, 0]) * 2.0 ** -23
    assert worst <= k * U2


@pytest.mark.parametrize("name,op", [("add_f", 3), ("mul_f", 5)])
def test_ops_with_float(host, name, op):
    n = 3000
    x, y = sample(n, 21), sample(n, 22)
    o = run_ops(host, op, x, y)
    ix, iy = run_ops(host, 0, x), run_ops(host, 0, y)
    for i in range(n):
        a, b = dwval(ix[i, 0], ix[i, 1]), Fraction(float(iy[i, 0]))  # the float operand is y's high part
        exact, scale = (a + b, abs(a) + abs(b)) if name == "add_f" else (a * b, abs(a * b))
        got = dwval(o[i, 0], o[i, 1])
        assert abs(got - exact) <= Fraction(8.0 * U2) * scale, (name, i)


def test_f2d_widens_floats_exactly(host):
    # every float exponent field 1..254 with random fractions and both signs:
    # x is a float, so h = x, l = 0, and the integer widening dw_f2d gives x
    rng = np.random.default_rng(31)
    bits = (rng.integers(0, 2, 254 * 40, dtype=np.uint32) << 31) | \
        (np.repeat(np.arange(1, 255, dtype=np.uint32), 40) << 23) | rng.integers(0, 2 ** 23, 254 * 40, dtype=np.uint32)
    x = bits.view(np.float32).astype(np.float64)
    o = run_ops(host, 0, x)
    ok = np.abs(x) >= 2.0 ** -126
    assert np.array_equal(o[ok, 0], x[ok]) and np.all(o[:, 1] == 0.0) and np.array_equal(o[:, 2], x)
    assert np.array_equal(np.signbit(o[:, 0]), np.signbit(x))
