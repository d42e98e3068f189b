"""Constants of the float-float exp in csrc/ffmath.cuh, re-derived on the CPU.

The CUDA path evaluates kept plan entries of the float-float passes with its
own exp (Tang's table-driven method in float-float arithmetic).  Its table
of 2^(j/64) and its reduction constants are checked here against values
derived independently in 60-digit decimal arithmetic; the GPU parity tests
check the resulting plan entries against the float64 oracle.
"""

import math
import os
import re
import struct
from decimal import Decimal, getcontext

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2603_07156_gb300", "csrc", "ffmath.cuh")

getcontext().prec = 60


def _ln2() -> Decimal:
    # ln 2 = 2 atanh(1/3) = 2 sum_k (1/3)^(2k+1) / (2k+1)
    x = Decimal(1) / 3
    s, k = Decimal(0), 0
    while True:
        t = x ** (2 * k + 1) / (2 * k + 1)
        if t < Decimal(10) ** -58:
            break
        s += t
        k += 1
    return 2 * s


def _f32(v: float) -> float:
    return struct.unpack("f", struct.pack("f", v))[0]


def _hexfloats(text: str):
    return [float.fromhex(h[:-1]) if h != "0.0f" else 0.0 for h in re.findall(r"-?0x[0-9a-f.]+p[+-]\d+f|0\.0f", text)]


def _source() -> str:
    with open(SRC) as f:
        return f.read()


def test_table_is_two_to_the_j_over_64_in_float_float():
    src = _source()
    body = src[src.index("kExp2Tab64[64] = {"):src.index("};", src.index("kExp2Tab64[64] = {"))]
    vals = _hexfloats(body)
    assert len(vals) == 128
    for j in range(64):
        exact = Decimal(2) ** (Decimal(j) / 64)
        hi, lo = vals[2 * j], vals[2 * j + 1]
        assert hi == _f32(float(exact))                      # hi is the float rounding
        assert abs(Decimal(hi) + Decimal(lo) - exact) <= Decimal(2) ** -46 * exact  # pair to ~2^-48


def test_reduction_constants_split_ln2_over_64():
    src = _source()
    ln2_64 = _ln2() / 64

    def const(name):
        m = re.search(name + r" = (-?0x[0-9a-f.]+p[+-]\d+f)", src)
        return float.fromhex(m.group(1)[:-1])

    L1, L2, L3 = const("L1"), const("L2"), const("L3")
    # L1 carries few bits, so k * L1 is exact in float for |k| < 2^15
    mant = Decimal(L1) / (Decimal(2) ** math.floor(math.log2(L1)))
    assert (mant * 2 ** 8) == int(mant * 2 ** 8)
    total = Decimal(L1) + Decimal(L2) + Decimal(L3)
    assert abs(total - ln2_64) <= Decimal(2) ** -70
    inv = const("kInvLn2_64")
    assert abs(Decimal(inv) - 1 / ln2_64) <= Decimal(2) ** -17
    m = re.search(r"C6h = (-?0x[0-9a-f.]+p[+-]\d+f), C6l = (-?0x[0-9a-f.]+p[+-]\d+f)", src)
    c6 = Decimal(float.fromhex(m.group(1)[:-1])) + Decimal(float.fromhex(m.group(2)[:-1]))
    assert abs(c6 - Decimal(1) / 6) <= Decimal(2) ** -50


def test_reduction_and_series_reach_float_float_accuracy():
    """The method itself in exact arithmetic: with the source's constants the
    reduced argument stays within ln2/128 and the truncated series plus the
    table reproduce exp to better than 2^-46 over the range the passes use."""
    src = _source()
    body = src[src.index("kExp2Tab64[64] = {"):src.index("};", src.index("kExp2Tab64[64] = {"))]
    vals = _hexfloats(body)

    def const(name):
        m = re.search(name + r" = (-?0x[0-9a-f.]+p[+-]\d+f)", src)
        return Decimal(float.fromhex(m.group(1)[:-1]))

    L = const("L1") + const("L2") + const("L3")
    inv = float(const("kInvLn2_64"))
    for x in [0.0, -1e-7, -0.3, -1.0, -7.25, -20.0, -44.3, -63.9, -86.0]:
        k = round(x * inv)
        e, j = k >> 6, k & 63
        r = Decimal(x) - k * L
        assert abs(r) <= Decimal(0.0055)
        poly = 1 + r + r * r / 2 + r ** 3 / 6 + r ** 4 / 24 + r ** 5 / 120 + r ** 6 / 720
        t = Decimal(vals[2 * j]) + Decimal(vals[2 * j + 1])
        approx = poly * t * Decimal(2) ** e
        exact = Decimal(x).exp()
        assert abs(approx - exact) <= Decimal(2) ** -46 * exact, x


# --- the float-float exp evaluated in float32 arithmetic (numpy emulation) ---

import numpy as np  # noqa: E402

f32 = np.float32


def _fma(a, b, c):
    # a*b is exact in float64 for float32 a, b; one rounding to float32 at the end
    return f32(float(a) * float(b) + float(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def _ff_add(a, b):
    s, e = _two_sum(a[0], b[0])
    return _fast_two_sum(s, f32(e + f32(a[1] + b[1])))


def _ff_mul(a, b):
    p = f32(a[0] * b[0])
    e = f32(_fma(a[0], b[0], -p) + _fma(a[0], b[1], f32(a[1] * b[0])))
    return _fast_two_sum(p, e)


def _consts():
    src = _source()

    def const(name):
        m = re.search(name + r" = (-?0x[0-9a-f.]+p[+-]\d+f)", src)
        return f32(float.fromhex(m.group(1)[:-1]))

    body = src[src.index("kExp2Tab64[64] = {"):src.index("};", src.index("kExp2Tab64[64] = {"))]
    vals = [f32(v) for v in _hexfloats(body)]
    m = re.search(r"C6h = (-?0x[0-9a-f.]+p[+-]\d+f), C6l = (-?0x[0-9a-f.]+p[+-]\d+f)", src)
    c6 = (f32(float.fromhex(m.group(1)[:-1])), f32(float.fromhex(m.group(2)[:-1])))
    return const("kInvLn2_64"), const("L1"), const("L2"), const("L3"), c6, vals


def _ff_exp(x, K):
    inv, L1, L2, L3, c6, tab = K
    kf = f32(np.rint(f32(x[0] * inv)))
    k = int(kf)
    e, j = k >> 6, k & 63
    if e < -125:
        return (f32(0), f32(0))
    t1 = _fma(-kf, L1, x[0])
    p2 = f32(kf * L2)
    e2 = _fma(kf, L2, -p2)
    rh, rl = _two_sum(t1, -p2)
    sh, sl = _two_sum(rh, x[1])
    r = _fast_two_sum(sh, f32(sl + f32(f32(rl - e2) - f32(kf * L3))))
    r2 = _ff_mul(r, r)
    r3 = _ff_mul(r2, r)
    h = r[0]
    tail = f32(f32(f32(h * h) * f32(h * h)) * f32(f32(1) / f32(24) + f32(h * f32(f32(1) / f32(120) + f32(h * f32(f32(1) / f32(720)))))))
    s = _ff_add(_ff_mul(r3, c6), (tail, f32(0)))
    s = _ff_add(s, (f32(r2[0] * f32(0.5)), f32(r2[1] * f32(0.5))))
    s = _ff_add(s, r)
    s = _ff_add((f32(1), f32(0)), s)
    v = _ff_mul(s, (tab[2 * j], tab[2 * j + 1]))
    sc = f32(2.0 ** e)
    return (f32(v[0] * sc), f32(v[1] * sc))


def test_ff_exp_in_float32_arithmetic_reaches_float_float_accuracy():
    """The CUDA routine's steps replayed with float32 rounding after every
    operation: relative error below 2^-45 against a 60-digit exp over the
    exponents the float-float passes evaluate.  Those are taken relative to
    the row maximum and kept only above 2^-64 of it, so x lies in
    [-44.4, 0]; the test covers [-64, 0]."""
    K = _consts()
    rng = np.random.default_rng(5)
    xs = np.concatenate([-rng.uniform(0, 64, 300), -rng.uniform(0, 1e-3, 20), [0.0, -44.4, -60.0, -64.0]])
    worst = 0.0
    for xv in xs:
        xh = f32(xv)
        xl = f32(rng.uniform(-1, 1) * 2.0 ** -24 * abs(float(xh)))  # a float-float argument
        h, l = _ff_exp((xh, xl), K)
        exact = (Decimal(float(xh)) + Decimal(float(xl))).exp()
        err = abs(Decimal(float(h)) + Decimal(float(l)) - exact) / exact
        worst = max(worst, float(err))
    assert worst < 2.0 ** -45, worst
