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
